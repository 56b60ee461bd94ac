"""Pins of the support invariant behind the skipped-row passes (reading of Sec. 3.1 and
Eq. NSfinal): outside the 2/3 box the masked nonlinear term is zero, so there every mode
obeys du/dt = -nu |k|^2 u.

* A state that vanishes outside the box keeps vanishing there exactly (bit for bit zero)
  under the oracle's RK4, the other two-register schemes and the 2N schemes, under both
  dealias rules and on a grid with other counts per direction.
* A mode outside the box decays by the scheme's stability polynomial R(-nu |k|^2 dt) per step
  whatever the rest of the field does (to round-off), so a state with anything outside the
  box must run the full transforms.
* The right-hand side of a state inside the box vanishes outside it exactly.
"""

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import inputs


def _outside(shape, variant=0):
    return ~sn.dealias_mask(shape, variant)


def _rk4_R(z):
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0


@pytest.mark.parametrize("scheme", ["rk4", "euler", "heun", "midpoint", "williamson3", "ck45"])
@pytest.mark.parametrize("variant", [0, 1])
def test_a_state_inside_the_box_stays_inside_exactly(scheme, variant):
    N = 24
    uh = inputs.isotropic_spectral(N, seed=3, k0=4.0).numpy()
    out = _outside((N, N, N), variant)
    assert np.all(uh[:, out] == 0) and np.abs(uh).max() > 0
    got = sn.run(uh, N, 0.02, 0.01, 6, variant=variant, scheme=scheme)
    assert np.all(got[:, out] == 0)
    assert np.abs(got[:, ~out]).max() > 0


def test_a_state_inside_the_box_of_another_grid_stays_inside():
    shape = (16, 8, 12)
    uh = inputs.isotropic_spectral(shape, seed=5, k0=2.0).numpy()
    out = _outside(shape)
    got = sn.run(uh, shape, 0.02, 0.01, 5)
    assert np.all(got[:, out] == 0)


def test_a_mode_outside_the_box_decays_by_the_stability_polynomial():
    N, nu, dt, n = 24, 0.05, 0.01, 6
    uh = inputs.isotropic_spectral(N, seed=8, k0=4.0).numpy()
    K = sn.wavenumbers(N)
    # a solenoidal mode at k = (0, 9, 1): |ky| = 9 >= 24/3, outside the box (row outside)
    kx, ky, kz = 0, 9, 1
    k2 = float(kx * kx + ky * ky + kz * kz)
    amp = np.zeros(3, dtype=np.complex128)
    amp[0] = 3.0 + 1.0j  # along x, perpendicular to k = (0, 9, 1)
    uh[:, kx, ky, kz] = amp * N ** 3 * 1e-2
    assert _outside((N, N, N))[kx, ky, kz] and np.all(K[:, kx, ky, kz] == [kx, ky, kz])
    got = sn.run(uh, N, nu, dt, n)
    expect = uh[:, kx, ky, kz] * _rk4_R(-nu * k2 * dt) ** n
    np.testing.assert_allclose(got[:, kx, ky, kz], expect, rtol=1e-13, atol=0)
    # and the field's other modes outside the box, zero at the start, stay zero
    out = _outside((N, N, N))
    out[kx, ky, kz] = False
    assert np.all(got[:, out] == 0)


def test_the_right_hand_side_of_a_state_inside_the_box_vanishes_outside_it():
    N = 32
    uh = inputs.isotropic_spectral(N, seed=11, k0=6.0).numpy()
    for variant in (0, 1):
        g = sn.Grid(N, variant)
        r = sn.rhs(uh, g, 0.01)
        assert np.all(r[:, ~g.mask] == 0)
        assert np.abs(r[:, g.mask]).max() > 0


def test_a_missing_mask_is_caught():
    # without the 2/3 rule the products reach outside the box and the invariant fails
    N = 24
    uh = inputs.isotropic_spectral(N, seed=3, k0=4.0).numpy()
    out = _outside((N, N, N))
    g = sn.Grid(N)
    g.mask = np.ones_like(g.mask)
    got = sn.rk4_step(uh, g, 0.02, 0.01)
    assert np.abs(got[:, out]).max() > 1e-8 * np.abs(got).max()
