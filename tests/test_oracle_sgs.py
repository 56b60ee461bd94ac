"""Pins of the FP64 closure reference (oracle/sgs_mlp.py): closed forms and finite differences."""

import numpy as np
import pytest

from oracle import sgs_mlp as sg
from oracle import spectral_ns as sn


def _sinc(x):
    return 1.0 if x == 0 else np.sin(x) / x


def test_filter_of_single_modes_is_the_sinc_product():
    Nf, Nc = 32, 16
    X = sn.mesh(Nf)
    D = 2 * np.pi / Nc
    u = np.zeros((1, Nf, Nf, Nf))
    u[0] = np.cos(3 * X[0]) + 0.5 * np.sin(2 * X[1] + 5 * X[2]) + np.cos(9 * X[0])  # 9 >= Nc/2: truncated
    ubar = sn.inverse(sg.filter_truncate(sn.forward(u), Nc))[0]
    Xc = sn.mesh(Nc)
    exact = _sinc(3 * D / 2) * np.cos(3 * Xc[0]) + 0.5 * _sinc(2 * D / 2) * _sinc(5 * D / 2) * np.sin(2 * Xc[1] + 5 * Xc[2])
    np.testing.assert_allclose(ubar, exact, atol=1e-13)


def test_stress_of_a_cosine_has_closed_form():
    # u = (cos a x, 0, 0): tau_00 = 1/2 (1 - s^2) + 1/2 (sinc(a D) - s^2) cos 2 a x, s = sinc(a D / 2)
    Nf, Nc, a = 32, 16, 3
    X = sn.mesh(Nf)
    u = np.zeros((3, Nf, Nf, Nf))
    u[0] = np.cos(a * X[0])
    tau, _ = sg.sgs_stress(sn.forward(u), Nc)
    D = 2 * np.pi / Nc
    s = _sinc(a * D / 2)
    Xc = sn.mesh(Nc)
    exact = 0.5 * (1 - s * s) + 0.5 * (_sinc(a * D) - s * s) * np.cos(2 * a * Xc[0])
    np.testing.assert_allclose(tau[0], exact, atol=1e-13)
    np.testing.assert_allclose(tau[1:], 0, atol=1e-13)


def test_stress_force_is_minus_divergence():
    N = 16
    X = sn.mesh(N)
    tau = np.zeros((6, N, N, N))
    tau[0] = np.sin(2 * X[0])            # tau_00
    tau[5] = np.cos(X[1]) * np.sin(X[2])  # tau_12 = tau_21
    f = sn.inverse(sg.stress_force(tau))
    np.testing.assert_allclose(f[0], -2 * np.cos(2 * X[0]), atol=1e-13)
    # f_1 = -d tau_12/dz, f_2 = -d tau_21/dy
    np.testing.assert_allclose(f[1], -np.cos(X[1]) * np.cos(X[2]), atol=1e-13)
    np.testing.assert_allclose(f[2], np.sin(X[1]) * np.sin(X[2]), atol=1e-13)


def test_gradients_of_a_plane_wave():
    N = 16
    X = sn.mesh(N)
    u = np.zeros((3, N, N, N))
    u[1] = np.sin(2 * X[0] + X[2])
    A = sg.velocity_gradients(sn.forward(u))
    np.testing.assert_allclose(A[3], 2 * np.cos(2 * X[0] + X[2]), atol=1e-12)  # dv/dx
    np.testing.assert_allclose(A[5], np.cos(2 * X[0] + X[2]), atol=1e-12)      # dv/dz
    np.testing.assert_allclose(A[[0, 1, 2, 4, 6, 7, 8]], 0, atol=1e-12)


@pytest.mark.parametrize("round_bf16", [False, True])
def test_network_gradient_matches_central_differences(round_bf16):
    rng = np.random.default_rng(3)
    p = sg.init_params(1)
    p["b1"] = rng.normal(size=sg.N_HID) * 0.1
    p["in_scale"] = rng.uniform(0.5, 2.0, size=sg.N_IN)
    X = rng.normal(size=(37, sg.N_IN))
    T = rng.normal(size=(37, sg.N_OUT))
    _, g = sg.loss_and_grads(p, X, T)  # exact FP64 gradient
    eps = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        idx = tuple(rng.integers(0, s) for s in p[name].shape)
        q = {k: v.copy() for k, v in p.items()}
        q[name][idx] += eps
        lp, _ = sg.loss_and_grads(q, X, T)
        q[name][idx] -= 2 * eps
        lm, _ = sg.loss_and_grads(q, X, T)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[name][idx]) < 1e-7 * max(1.0, abs(fd)), name
    if round_bf16:
        lr, gr = sg.loss_and_grads(p, X, T, round_bf16=True)
        l0, g0 = sg.loss_and_grads(p, X, T)
        assert abs(lr - l0) < 0.05 * l0  # bfloat16 inputs move the loss by well under 5 %
        for name in g0:
            assert np.linalg.norm(gr[name] - g0[name]) <= 0.05 * np.linalg.norm(g0[name]) + 1e-12


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.14159265], dtype=np.float32)
    r = sg.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0          # tie -> even (mantissa 0)
    assert r[2] == 1.0 + 2 ** -6                 # tie -> even (round up)
    assert r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12


def test_param_vector_round_trip():
    p = sg.init_params(4)
    v = sg.flatten(p)
    assert v.size == 10 + 10 + 640 + 64 + 4096 + 64 + 384 + 6 + 6 + 6
    q = sg.unflatten(v)
    for k in p:
        assert np.array_equal(p[k], q[k])


def test_forced_rhs_reduces_to_plain_rhs_without_force():
    N = 16
    uh = sn.to_spectral(np.random.default_rng(0).standard_normal((3, N, N, N)) * 0.1)
    g = sn.Grid(N)
    np.testing.assert_allclose(sg.rhs_forced(uh, g, 0.01, np.zeros_like(uh)), sn.rhs(uh, g, 0.01), atol=1e-12)
