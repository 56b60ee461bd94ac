"""Pins of the oracle on grids with a different number of points per direction
(Sec. 2 footnote: other point counts per direction; Sec. 3.1 mesh and wavenumbers).

* The library transforms equal the triple-sum DFT of Eqs. ffteq/iffteq written out on
  grids such as 6 x 4 x 8.
* The 2/3 mask keeps |k_i| < N_i/3 per direction: the kept counts are products of the
  per-direction counts, written out by hand.
* The dealiased nonlinear term of a band-limited field equals the direct convolution
  sum over triads p + q = k of u_hat(p) x omega_hat(q), masked with each direction's
  own cut-off (no FFT on the checking side).
* ABC flow (omega = u, so u x omega = 0) decays by the RK4 polynomial R(-nu dt) per
  step on any point counts.
* Swapping the x and y axes (and components) maps the run on (Nx, Ny, Nz) onto the run
  on (Ny, Nx, Nz): each count must act on its own axis.
* Grid means: u = (sin y, 0, 0) has E = 1/4 and eps = nu/2 on every grid.
"""

import numpy as np
import pytest

from oracle import brute_dft, spectral_ns as sn
from paper_1602_03638_gb300 import inputs


def _rk4_R(z):
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0


@pytest.mark.parametrize("shape", [(6, 4, 8), (4, 8, 6), (8, 6, 4)])
def test_transforms_are_the_triple_sum_dft(shape):
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(shape)
    np.testing.assert_allclose(sn.forward(u), brute_dft.forward_r2c(u), rtol=0, atol=1e-11)
    uh = sn.forward(u)
    np.testing.assert_allclose(sn.inverse(uh), brute_dft.inverse_c2r(uh), rtol=0, atol=1e-13)
    np.testing.assert_allclose(sn.inverse(uh), u, rtol=0, atol=1e-13)


def test_wavenumbers_follow_each_directions_count():
    K = sn.wavenumbers((6, 4, 8))
    assert K.shape == (3, 6, 4, 5)
    assert list(K[0, :, 0, 0]) == [0, 1, 2, -3, -2, -1]
    assert list(K[1, 0, :, 0]) == [0, 1, -2, -1]
    assert list(K[2, 0, 0, :]) == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("variant,expected", [(0, 7 * 3 * 8), (1, 9 * 5 * 9)])
def test_dealias_mask_keeps_each_directions_own_box(variant, expected):
    # (12, 6, 24). variant 0: |kx| < 4 (7 values), |ky| < 2 (3), kz < 8 (8).
    # variant 1: |kx| < 2/3 * 7 (9 values), |ky| < 2/3 * 4 (5), kz < 2/3 * 13 (9).
    m = sn.dealias_mask((12, 6, 24), variant)
    assert m.shape == (12, 6, 13) and int(m.sum()) == expected


def _band_field(shape, band, seed):
    """Full-spectrum Fourier-series coefficients c(k) of a real field with |k_i| <= band_i."""
    rng = np.random.default_rng(seed)
    modes = {}
    for kx in range(-band[0], band[0] + 1):
        for ky in range(-band[1], band[1] + 1):
            for kz in range(-band[2], band[2] + 1):
                k = (kx, ky, kz)
                if k in modes:
                    continue
                mk = (-kx, -ky, -kz)
                v = rng.standard_normal(3) + 1j * rng.standard_normal(3)
                if k == mk:
                    v = v.real.astype(np.complex128)
                modes[k] = v
                modes[mk] = np.conj(v)
    return modes


def _half_spectrum(modes, shape):
    """u_hat on the half spectrum: N^3 times the series coefficients (forward F unnormalised)."""
    nx, ny, nz = shape
    uh = np.zeros((3, nx, ny, nz // 2 + 1), dtype=np.complex128)
    for (kx, ky, kz), v in modes.items():
        if kz >= 0:
            uh[:, kx % nx, ky % ny, kz] = v * (nx * ny * nz)
    return uh


def test_nonlinear_term_equals_the_masked_triad_sum():
    shape = (16, 8, 12)
    band = (3, 1, 2)  # product modes |k_i| <= (6, 2, 4) < N_i / 2: no aliasing on this grid
    c = _band_field(shape, band, 5)
    w = {k: 1j * np.cross(np.array(k, dtype=np.float64), v) for k, v in c.items()}
    prod = {}
    for p, up in c.items():
        for q, wq in w.items():
            k = (p[0] + q[0], p[1] + q[1], p[2] + q[2])
            prod[k] = prod.get(k, 0.0) + np.cross(up, wq)
    # each direction's own cut-off: |kx| < 16/3, |ky| < 8/3, |kz| < 4
    kept = {k: v for k, v in prod.items() if 3 * abs(k[0]) < 16 and 3 * abs(k[1]) < 8 and 3 * abs(k[2]) < 12}
    assert any(abs(k[0]) == 6 for k in prod) and any(abs(k[2]) == 4 for k in prod)  # the mask acts in x and z
    expect = _half_spectrum(kept, shape)
    uh = _half_spectrum(c, shape)
    got = sn.nonlinear_hat(uh, sn.Grid(shape))
    assert np.abs(got - expect).max() < 1e-10 * np.abs(expect).max()


def test_planted_single_count_mask_is_caught(monkeypatch):
    # a mask built from the x count alone keeps |ky| = 2 on the 8-point y axis
    shape = (16, 8, 12)
    good = sn.dealias_mask(shape)
    bad = sn.dealias_mask((16, 16, 16))[:, np.r_[0:4, 12:16], :7]
    assert not np.array_equal(good, bad)
    monkeypatch.setattr(sn, "dealias_mask", lambda N, variant=0: bad)
    c = _band_field(shape, (3, 1, 2), 5)
    uh = _half_spectrum(c, shape)
    got = sn.nonlinear_hat(uh, sn.Grid(shape))
    monkeypatch.undo()
    ref = sn.nonlinear_hat(uh, sn.Grid(shape))
    assert np.abs(got - ref).max() > 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(16, 8, 12), (8, 12, 16)])
def test_abc_flow_decays_by_the_rk4_polynomial(shape):
    nu, dt, n = 0.2, 0.1, 6
    uh0 = sn.to_spectral(inputs.abc_flow(shape))
    got = sn.run(uh0, shape, nu, dt, n)
    assert np.abs(got - uh0 * _rk4_R(-nu * dt) ** n).max() < 1e-12 * np.abs(uh0).max()


def test_swapping_x_and_y_swaps_their_counts():
    shape, nu, dt, n = (16, 8, 12), 0.02, 0.01, 3
    uh = inputs.isotropic_spectral(shape, seed=4, k0=2.0).numpy()
    a = sn.run(uh, shape, nu, dt, n)
    # transpose: x <-> y axes and components 0 <-> 1
    t = np.transpose(uh, (0, 2, 1, 3))[[1, 0, 2]]
    b = sn.run(t, (8, 16, 12), nu, dt, n)
    np.testing.assert_allclose(np.transpose(b, (0, 2, 1, 3))[[1, 0, 2]], a, rtol=0, atol=1e-12 * np.abs(a).max())


def test_grid_means_of_a_shear_wave():
    nu = 0.03
    for shape in [(8, 6, 4), (4, 12, 10)]:
        X = sn.mesh(shape)
        u = np.zeros((3,) + shape)
        u[0] = np.sin(X[1])
        d = sn.diagnostics(sn.to_spectral(u), nu)
        assert abs(d["energy"] - 0.25) < 1e-14 and abs(d["dissipation"] - nu / 2) < 1e-14
        assert abs(sn.energy(sn.to_spectral(u)) - 0.25) < 1e-14
        assert abs(sn.energy_spectrum(sn.to_spectral(u)).sum() - 0.25) < 1e-14


def test_random_field_is_divergence_free_and_in_each_directions_box():
    shape = (16, 8, 12)
    uh = inputs.isotropic_spectral(shape, seed=7, k0=3.0).numpy()
    g = sn.Grid(shape)
    assert np.abs(np.sum(g.K * uh, axis=0)).max() < 1e-12 * np.abs(uh).max()
    assert np.all(uh[:, ~g.mask] == 0)
    assert abs(sn.energy(uh) - 1.0) < 1e-12


def test_zero_nyquist_clears_each_directions_own_nyquist_plane():
    uh = np.ones((3, 6, 4, 5), dtype=np.complex128)  # (Nx, Ny, Nz) = (6, 4, 8)
    z = sn.zero_nyquist(uh)
    K = sn.wavenumbers((6, 4, 8))
    nyq = (np.abs(K[0]) == 3) | (np.abs(K[1]) == 2) | (K[2] == 4)
    assert np.all(z[:, nyq] == 0) and np.all(z[:, ~nyq] == 1)
    assert int(nyq.sum()) == 6 * 4 * 5 - 5 * 3 * 4  # kept: 5 kx x 3 ky x 4 kz
