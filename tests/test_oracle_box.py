"""Pins of the oracle on boxes other than [0, 2 pi]^3 (Sec. 2 footnote: other domain
lengths; Sec. 3.1: other box sizes through scaling of the governing equations).

* A single Fourier mode u = (sin kz, cos kz, 0) with k = 2 pi / Lz is a Beltrami field
  (omega = k u, u x omega = 0): RK4 multiplies it by R(-nu k^2 dt) per step exactly.
  The same along x and along y with their own lengths.
* The curl of (0, sin(2 pi x / Lx), 0) is (0, 0, (2 pi / Lx) cos(2 pi x / Lx)).
* Scaling: on the box of side 2 pi s the coefficients after n steps with (nu, dt)
  equal those on the 2 pi box with (nu / s, dt / s) (x = s x', t = s t', u unchanged).
* Transposition: swapping the x and y axes (and the x and y components) maps the run on
  box (Lx, Ly, Lz) onto the run on box (Ly, Lx, Lz): the equations are invariant under
  this reflection, so each length must act on its own axis.
"""

import math

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import inputs


def _rk4_R(z):
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0


def _beltrami(N, lengths, axis):
    X = sn.mesh(N, lengths)
    k = 2.0 * np.pi / lengths[axis]
    a, b = (axis + 1) % 3, (axis + 2) % 3
    u = np.zeros((3, N, N, N))
    u[a] = np.sin(k * X[axis])
    u[b] = np.cos(k * X[axis])
    return u, k


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_single_mode_beltrami_decays_by_rk4_polynomial(axis):
    # dt keeps -nu k^2 dt inside RK4's real stability interval for every mode of the
    # short axis (k up to 14 on Lx = pi), so round-off in the other modes stays small
    N, nu, dt, n = 16, 0.2, 0.02, 6
    lengths = (np.pi, 3.0 * np.pi, 4.0 * np.pi)
    u, k = _beltrami(N, lengths, axis)
    g = sn.Grid(N, 0, lengths)
    uh0 = sn.to_spectral(u)
    w = sn.inverse(sn.curl_hat(uh0, g))
    np.testing.assert_allclose(w, k * u, atol=1e-12)
    uh = sn.run(uh0, N, nu, dt, n, lengths=lengths)
    assert np.abs(uh - uh0 * _rk4_R(-nu * k * k * dt) ** n).max() < 1e-13 * np.abs(uh0).max()


def test_curl_of_a_shear_wave_on_a_long_box():
    N, Lx = 16, 6.0 * np.pi
    lengths = (Lx, 2.0 * np.pi, np.pi)
    X = sn.mesh(N, lengths)
    u = np.zeros((3, N, N, N))
    u[1] = np.sin(2 * np.pi * X[0] / Lx)
    w = sn.inverse(sn.curl_hat(sn.forward(u), sn.Grid(N, 0, lengths)))
    np.testing.assert_allclose(w[0], 0, atol=1e-13)
    np.testing.assert_allclose(w[1], 0, atol=1e-13)
    np.testing.assert_allclose(w[2], (2 * np.pi / Lx) * np.cos(2 * np.pi * X[0] / Lx), atol=1e-13)


def test_uniform_box_scaling_is_a_change_of_nu_and_dt():
    N, nu, dt, n, s = 16, 0.01, 0.02, 5, 2.5
    uh0 = inputs.random_field_in_mask(N, seed=6).numpy()
    big = sn.run(uh0, N, nu, dt, n, lengths=(2 * np.pi * s,) * 3)
    ref = sn.run(uh0, N, nu / s, dt / s, n)
    assert np.abs(big - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(big - sn.run(uh0, N, nu, dt, n)).max() > 1e-6 * np.abs(ref).max()


def _transpose_xy(uh):
    t = np.swapaxes(uh, 1, 2).copy()
    return t[[1, 0, 2]]


def _run_box(uh0, lengths, N=16, nu=0.01, dt=0.01, n=4):
    return sn.run(uh0, N, nu, dt, n, lengths=lengths)


def test_swapping_x_and_y_swaps_their_lengths():
    N = 16
    uh0 = inputs.random_field_in_mask(N, seed=8).numpy()
    a = _run_box(uh0, (np.pi, 3 * np.pi, 2 * np.pi))
    b = _run_box(_transpose_xy(uh0), (3 * np.pi, np.pi, 2 * np.pi))
    assert np.abs(_transpose_xy(a) - b).max() < 1e-12 * np.abs(a).max()
    # and the lengths matter: the cubic run differs
    c = _run_box(uh0, (2 * np.pi,) * 3)
    assert np.abs(a - c).max() > 1e-4 * np.abs(a).max()


def test_projection_and_divergence_on_a_non_cubic_box():
    N = 16
    lengths = (np.pi, 2 * np.pi, 5 * np.pi)
    g = sn.Grid(N, 0, lengths)
    rng = np.random.default_rng(12)
    phi = sn.forward(rng.standard_normal((N, N, N)))
    grad = np.array([1j * g.K[i] * phi for i in range(3)])
    assert np.abs(sn.project(grad, g)).max() < 1e-12 * np.abs(grad).max()
    uh = sn.project(sn.forward(rng.standard_normal((3, N, N, N))), g)
    uh = sn.run(sn.zero_nyquist(uh), N, 0.01, 0.01, 3, lengths=lengths)
    assert sn.diagnostics(uh, 0.01, lengths)["max_div"] < 1e-12 * np.abs(uh).max()


def test_planted_swapped_axis_lengths_are_caught(monkeypatch):
    orig = sn.Grid.__post_init__

    def swapped(self):
        if self.lengths is not None:
            L = list(self.lengths)
            self.lengths = (L[1], L[0], L[2])
        orig(self)

    monkeypatch.setattr(sn.Grid, "__post_init__", swapped)
    u, k = _beltrami(16, (np.pi, 3.0 * np.pi, 4.0 * np.pi), 0)
    uh0 = sn.to_spectral(u)
    uh = sn.run(uh0, 16, 0.2, 0.02, 6, lengths=(np.pi, 3.0 * np.pi, 4.0 * np.pi))
    assert np.abs(uh - uh0 * _rk4_R(-0.2 * k * k * 0.02) ** 6).max() > 1e-3 * np.abs(uh0).max()


def test_energy_of_box_beltrami_tracks_exp_minus_2_nu_k2_t():
    N, nu, dt, n = 16, 0.05, 0.01, 20
    lengths = (2 * np.pi, 2 * np.pi, 4 * np.pi)
    u, k = _beltrami(N, lengths, 2)
    uh = sn.run(sn.to_spectral(u), N, nu, dt, n, lengths=lengths)
    assert abs(sn.energy(uh) / 0.5 - math.exp(-2 * nu * k * k * n * dt)) < 1e-10
