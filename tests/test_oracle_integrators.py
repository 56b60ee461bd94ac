"""Pins of the oracle's explicit Runge-Kutta schemes other than the Appendix RK4
(forward Euler of Sec. 3.1; the two-stage Heun and midpoint rules; the low-storage
2N schemes of Williamson (3 stages, order 3) and Carpenter & Kennedy (5 stages, order 4)).

* Linear decay: the ABC (Beltrami) flow has u x omega = 0, so each step multiplies
  u_hat by the scheme's stability polynomial R(z), z = -nu |k|^2 dt, exactly:
  1 + z for Euler, 1 + z + z^2/2 for both two-stage rules.
* Order on the nonlinear system: halving dt divides the error against a fine RK4
  reference by about 2 (Euler) and 4 (Heun, midpoint).
* The RK4 entry of the table is the Appendix driver itself.
"""

import math

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import inputs

R = {
    "euler": lambda z: 1.0 + z,
    "heun": lambda z: 1.0 + z + z * z / 2.0,
    "midpoint": lambda z: 1.0 + z + z * z / 2.0,
}


def _abc_error(scheme, N=16, nu=0.2, dt=0.1, n=7):
    uh0 = sn.to_spectral(inputs.abc_flow(N))
    uh = sn.run(uh0, N, nu, dt, n, scheme=scheme)
    expect = uh0 * R[scheme](-nu * 1.0 * dt) ** n
    return np.abs(uh - expect).max() / np.abs(uh0).max()


@pytest.mark.parametrize("scheme", ["euler", "heun", "midpoint"])
def test_abc_decays_by_the_scheme_stability_polynomial(scheme):
    assert _abc_error(scheme) < 1e-13


def test_rk4_entry_is_the_appendix_driver():
    N = 16
    g = sn.Grid(N)
    uh = inputs.random_field_in_mask(N, seed=5).numpy()
    np.testing.assert_array_equal(sn.rk_step(uh, g, 0.01, 0.05, "rk4"), sn.rk4_step(uh, g, 0.01, 0.05))


def _error(scheme, dt, T=0.4, N=16, nu=0.01):
    uh0 = inputs.random_field_in_mask(N, seed=7).numpy()
    ref = sn.run(uh0, N, nu, T / 64, 64)
    got = sn.run(uh0, N, nu, dt, int(round(T / dt)), scheme=scheme)
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("scheme,order", [("euler", 1), ("heun", 2), ("midpoint", 2)])
def test_order_on_the_nonlinear_system(scheme, order):
    e1, e2 = _error(scheme, 0.05), _error(scheme, 0.025)
    ratio = e1 / e2
    assert 0.75 * 2 ** order < ratio < 1.3 * 2 ** order, ratio


def test_euler_entry_is_the_sec31_loop():
    N = 16
    g = sn.Grid(N)
    uh = inputs.random_field_in_mask(N, seed=3).numpy()
    np.testing.assert_allclose(sn.rk_step(uh, g, 0.02, 0.01, "euler"), sn.euler_step(uh, g, 0.02, 0.01),
                               rtol=0, atol=1e-15 * np.abs(uh).max())


def test_planted_wrong_midpoint_tableau_is_caught(monkeypatch):
    # a = (1/2, 1/2) with b = 1/2 has R(z) = 1 + z + z^2/4: off by z^2/4 per step
    bad = dict(sn.RK_SCHEMES)
    bad["midpoint"] = ((0.5, 0.5), (0.5,))
    monkeypatch.setattr(sn, "RK_SCHEMES", bad)
    assert _abc_error("midpoint") > 1e-4


def test_energy_of_abc_under_euler_matches_closed_form():
    N, nu, dt, n = 16, 0.05, 0.01, 20
    uh = sn.run(sn.to_spectral(inputs.abc_flow(N)), N, nu, dt, n, scheme="euler")
    E0 = 1.5  # A = B = C = 1
    assert abs(sn.energy(uh) / E0 - (1.0 - nu * dt) ** (2 * n)) < 1e-12
    assert abs(sn.energy(uh) / E0 - math.exp(-2 * nu * n * dt)) > 1e-7  # Euler is not exact


# ---------------------------------------------------------------- low-storage (2N) schemes

def _butcher_from_2n(A, B):
    """Butcher matrix and weights of a 2N scheme, from the recurrence written out by hand:
    u_j = u_0 + dt sum_i k_i sum_{l=i..j} B_l prod_{m=i+1..l} A_m, stage j + 1 starts from u_j."""
    s = len(A)

    def coef(i, j):
        return sum(B[l] * math.prod(A[m] for m in range(i + 1, l + 1)) for l in range(i, j + 1))

    a = np.zeros((s, s))
    for j in range(1, s):
        for i in range(j):
            a[j, i] = coef(i, j - 1)
    return a, np.array([coef(i, s - 1) for i in range(s)])


def _stability(A, B, z):
    a, b = _butcher_from_2n(A, B)
    s = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * a, np.ones(s))


@pytest.mark.parametrize("scheme,order", [("williamson3", 3), ("ck45", 4)])
def test_2n_coefficients_satisfy_the_order_conditions(scheme, order):
    a, b = _butcher_from_2n(*sn.LSRK_SCHEMES[scheme])
    c = a.sum(1)
    conds = [b.sum() - 1, b @ c - 1 / 2, b @ c ** 2 - 1 / 3, b @ a @ c - 1 / 6]
    if order >= 4:
        conds += [b @ c ** 3 - 1 / 4, b @ (c * (a @ c)) - 1 / 8, b @ a @ c ** 2 - 1 / 12, b @ a @ a @ c - 1 / 24]
    assert max(abs(x) for x in conds) < 1e-14
    if order == 3:  # third order only: an order-four condition fails
        assert abs(b @ c ** 3 - 1 / 4) > 1e-3


@pytest.mark.parametrize("scheme", ["williamson3", "ck45"])
def test_abc_decays_by_the_2n_stability_polynomial(scheme):
    N, nu, dt, n = 16, 0.2, 0.1, 7
    uh0 = sn.to_spectral(inputs.abc_flow(N))
    uh = sn.run(uh0, N, nu, dt, n, scheme=scheme)
    A, B = sn.LSRK_SCHEMES[scheme]
    z = -nu * dt
    expect = uh0 * _stability(A, B, z) ** n
    assert np.abs(uh - expect).max() < 1e-13 * np.abs(uh0).max()
    # the polynomial agrees with exp(z) to the scheme's order: 1 + z + z^2/2 + z^3/6 (+ z^4/24)
    taylor = sum(z ** k / math.factorial(k) for k in range(4 if scheme == "williamson3" else 5))
    assert abs(_stability(A, B, z) - taylor) < 1e-5


@pytest.mark.parametrize("scheme,order", [("williamson3", 3), ("ck45", 4)])
def test_2n_order_on_the_nonlinear_system(scheme, order):
    e1, e2 = _error(scheme, 0.1), _error(scheme, 0.05)
    ratio = e1 / e2
    assert 0.75 * 2 ** order < ratio < 1.4 * 2 ** order, ratio


def test_planted_2n_mistake_is_caught(monkeypatch):
    # dropping the A_j dU term (dU = dt RHS) turns the scheme into stages of forward Euler
    bad = dict(sn.LSRK_SCHEMES)
    A, B = bad["williamson3"]
    bad["williamson3"] = ((0.0, 0.0, 0.0), B)
    monkeypatch.setattr(sn, "LSRK_SCHEMES", bad)
    N, nu, dt, n = 16, 0.2, 0.1, 7
    uh0 = sn.to_spectral(inputs.abc_flow(N))
    uh = sn.run(uh0, N, nu, dt, n, scheme="williamson3")
    assert np.abs(uh - uh0 * _stability(A, B, -nu * dt) ** n).max() > 1e-4 * np.abs(uh0).max()
