"""Pins of the FP64 closure reference (oracle/sgs_mlp.py): closed forms and finite differences."""

import math

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


# ---------------------------------------------------------------- hand-computed pins

def _sparse_net():
    """One active path: x0 -> hidden unit 5 -> hidden unit 7 -> output 2 (all other weights zero).

    in_shift[0] = 1, in_scale[0] = 0.5 and x0 = 3 give xn0 = 1; W1[0, 5] = 2, b1[5] = 0 give
    z1 = 2; W2[5, 7] = 1, b2[7] = -1 give z2 = SiLU(2) - 1; W3[7, 2] = -3, b3[2] = 0.25 give
    y2; out_scale[2] = 4, out_shift[2] = -1 give tau2. Outputs 0 and 4 carry only their biases
    and shifts. Every hidden unit other than 5 and 7 has pre-activation 0 and SiLU(0) = 0.
    """
    p = {k: np.zeros_like(v) for k, v in sg.init_params(0).items()}
    p["in_scale"][:] = 1.0
    p["out_scale"][:] = 1.0
    p["in_shift"][0], p["in_scale"][0] = 1.0, 0.5
    p["W1"][0, 5] = 2.0
    p["W2"][5, 7], p["b2"][7] = 1.0, -1.0
    p["W3"][7, 2], p["b3"][2] = -3.0, 0.25
    p["out_scale"][2], p["out_shift"][2] = 4.0, -1.0
    p["b3"][4], p["out_shift"][0] = 0.5, 2.0
    X = np.array([[3.0, 7.0, -2.0, 0.5, 1.5, -4.0, 2.5, 0.25, -1.0, 0.098]])
    return p, X


def test_forward_of_a_sparse_network_is_a_hand_computed_composition():
    p, X = _sparse_net()
    a = sg.forward(p, X)
    # SiLU(z) = z / (1 + e^-z):  SiLU(2) = 2 e^2 / (1 + e^2), so z2 = SiLU(2) - 1 = tanh(1)
    h1 = 2.0 * math.e ** 2 / (1.0 + math.e ** 2)
    assert abs(h1 - 1.7615941559557646) < 1e-15
    t = math.tanh(1.0)
    h2 = t / (1.0 + math.exp(-t))  # SiLU(tanh 1)
    assert abs(h2 - 0.5191785397719028) < 1e-15
    y2 = -3.0 * h2 + 0.25
    np.testing.assert_allclose(a["h1"][0, 5], h1, rtol=0, atol=1e-15)
    np.testing.assert_allclose(a["z2"][0, 7], t, rtol=0, atol=1e-15)
    np.testing.assert_allclose(a["y"][0], [0, 0, y2, 0, 0.5, 0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(a["tau"][0], [2.0, 0, 4.0 * y2 - 1.0, 0, 0.5, 0], rtol=0, atol=1e-14)
    # the other hidden units are exactly zero (SiLU(0) = 0)
    assert np.count_nonzero(a["h1"]) == 1 and np.count_nonzero(a["h2"]) == 1


def test_forward_rounds_features_weights_and_activations_to_bf16():
    p, X = _sparse_net()
    a = sg.forward(p, X, round_bf16=True)
    # xn = 1 and the weights 2, 1, -3 are exact in bfloat16; SiLU(2) = 1.76159... rounds to
    # 225/128 = 1.7578125 (8 significant bits), so z2 = 0.7578125; its SiLU 0.51598 rounds
    # to 132/256 = 0.515625 before the last product
    z2 = 225.0 / 128.0 - 1.0
    np.testing.assert_allclose(a["z2"][0, 7], z2, rtol=0, atol=1e-15)
    h2 = z2 / (1.0 + math.exp(-z2))
    assert abs(h2 - 0.5159783258600358) < 1e-15
    np.testing.assert_allclose(a["y"][0, 2], -3.0 * (132.0 / 256.0) + 0.25, rtol=0, atol=1e-15)


def test_adam_two_hand_computed_steps_on_a_scalar():
    # Kingma & Ba (2015), Algorithm 1 with beta1 = 0.9, beta2 = 0.999, eps = 1e-8, lr = 0.1
    p = {k: np.zeros_like(v) for k, v in sg.init_params(0).items()}
    p["b3"][1] = 1.0
    st = sg.adam_init(p)
    g = {k: np.zeros_like(p[k]) for k in sg.TRAINABLE}
    # step 1, g = 2: m = 0.2, v = 0.004, m_hat = 0.2 / 0.1 = 2, v_hat = 0.004 / 0.001 = 4
    g["b3"][1] = 2.0
    q, st = sg.adam_step(p, g, st, lr=0.1)
    assert abs(st["m"]["b3"][1] - 0.2) < 1e-16 and abs(st["v"]["b3"][1] - 0.004) < 1e-17
    assert abs(q["b3"][1] - (1.0 - 0.1 * 2.0 / (2.0 + 1e-8))) < 1e-15
    # step 2, g = -1: m = 0.18 - 0.1 = 0.08, v = 0.003996 + 0.001 = 0.004996,
    # m_hat = 0.08 / 0.19, v_hat = 0.004996 / 0.001999
    g["b3"][1] = -1.0
    q2, st = sg.adam_step(q, g, st, lr=0.1)
    assert st["t"] == 2
    assert abs(st["m"]["b3"][1] - 0.08) < 1e-16 and abs(st["v"]["b3"][1] - 0.004996) < 1e-17
    m_hat, v_hat = 0.08 / 0.19, 0.004996 / 0.001999
    assert abs(m_hat - 0.42105263157894735) < 1e-15 and abs(v_hat - 2.499249624812406) < 1e-14
    expect = q["b3"][1] - 0.1 * m_hat / (math.sqrt(v_hat) + 1e-8)
    assert abs(q2["b3"][1] - expect) < 1e-15
    assert abs(q2["b3"][1] - 0.8733662967024313) < 1e-14
    # entries with zero gradient and zero moments do not move; normalisation entries are fixed
    for k in p:
        if k != "b3":
            assert np.array_equal(q2[k], p[k]), k


def test_adam_without_bias_correction_would_fail_the_first_step():
    # a planted omission (no 1 - beta^t factors) moves the scalar by 0.1 * 0.2 / sqrt(0.004) = 0.316
    p = {k: np.zeros_like(v) for k, v in sg.init_params(0).items()}
    g = {k: np.zeros_like(p[k]) for k in sg.TRAINABLE}
    g["W1"][3, 4] = 2.0
    q, _ = sg.adam_step(p, g, sg.adam_init(p), lr=0.1)
    assert abs(q["W1"][3, 4] + 0.1) < 1e-8
    wrong = 0.1 * 0.2 / (math.sqrt(0.004) + 1e-8)
    assert abs(abs(q["W1"][3, 4]) - wrong) > 0.2


def _gradient_force_error(rhs_forced):
    N, nu = 16, 0.02
    X = sn.mesh(N)
    g = sn.Grid(N)
    uh = sn.to_spectral(np.random.default_rng(1).standard_normal((3, N, N, N)) * 0.1)
    # f = grad phi with phi = cos(2y) sin(z) + sin(x + y) (inside the 2/3 box)
    f = np.stack([np.cos(X[0] + X[1]),
                  -2 * np.sin(2 * X[1]) * np.sin(X[2]) + np.cos(X[0] + X[1]),
                  np.cos(2 * X[1]) * np.cos(X[2])])
    fh = sn.forward(f)
    return np.abs(rhs_forced(uh, g, nu, fh) - sn.rhs(uh, g, nu)).max() / np.abs(fh).max()


def _outside_box_error(rhs_forced):
    N, nu = 16, 0.02
    X = sn.mesh(N)
    g = sn.Grid(N)
    uh = sn.to_spectral(np.random.default_rng(2).standard_normal((3, N, N, N)) * 0.1)
    # solenoidal force whose modes all have some |k_i| >= 6 > N/3: removed by the mask
    f = np.stack([np.cos(6 * X[1]), np.sin(7 * X[2] + X[0]), np.cos(6 * X[0])])
    fh = sn.forward(f)
    return np.abs(rhs_forced(uh, g, nu, fh) - sn.rhs(uh, g, nu)).max() / np.abs(fh).max()


def _solenoidal_mode_error(rhs_forced):
    N, nu = 16, 0.02
    X = sn.mesh(N)
    g = sn.Grid(N)
    # f = (0, 3 sin x, 0) + grad cos(2y): the projection keeps exactly (0, 3 sin x, 0)
    f = np.stack([np.zeros_like(X[0]), 3 * np.sin(X[0]) - 2 * np.sin(2 * X[1]), np.zeros_like(X[0])])
    keep = np.stack([np.zeros_like(X[0]), 3 * np.sin(X[0]), np.zeros_like(X[0])])
    zero = np.zeros((3, N, N, N // 2 + 1), dtype=np.complex128)
    e0 = np.abs(sn.inverse(rhs_forced(zero, g, nu, sn.forward(f))) - keep).max()
    # superposition on a non-zero state: forced minus unforced is the same mode
    uh = sn.to_spectral(np.random.default_rng(3).standard_normal((3, N, N, N)) * 0.1)
    e1 = np.abs(sn.inverse(rhs_forced(uh, g, nu, sn.forward(f)) - sn.rhs(uh, g, nu)) - keep).max()
    return max(e0, e1)


def test_forced_rhs_removes_a_gradient_force():
    assert _gradient_force_error(sg.rhs_forced) < 1e-12


def test_forced_rhs_masks_a_force_outside_the_dealiasing_box():
    assert _outside_box_error(sg.rhs_forced) < 1e-12


def test_forced_rhs_passes_a_solenoidal_mode_and_drops_its_gradient_part():
    assert _solenoidal_mode_error(sg.rhs_forced) < 1e-12


def test_forced_rhs_pins_catch_planted_mistakes():
    def force_after_projection(uh, g, nu, fh):
        return sn.project(sn.nonlinear_hat(uh, g), g) + fh * g.mask - nu * g.K2 * uh

    def force_unmasked(uh, g, nu, fh):
        return sn.project(sn.nonlinear_hat(uh, g) + fh, g) - nu * g.K2 * uh

    def force_sign_flipped(uh, g, nu, fh):
        return sn.project(sn.nonlinear_hat(uh, g) - fh * g.mask, g) - nu * g.K2 * uh

    assert _gradient_force_error(force_after_projection) > 0.1
    assert _outside_box_error(force_unmasked) > 0.1
    assert _solenoidal_mode_error(force_sign_flipped) > 1.0


def test_forward_pins_catch_a_planted_activation(monkeypatch):
    p, X = _sparse_net()
    t = math.tanh(1.0)
    expect = 4.0 * (-3.0 * t / (1.0 + math.exp(-t)) + 0.25) - 1.0
    assert abs(sg.forward(p, X)["tau"][0, 2] - expect) < 1e-14
    for wrong in (np.tanh, lambda z: 1.0 / (1.0 + np.exp(-z)), lambda z: np.maximum(z, 0.0)):
        monkeypatch.setattr(sg, "_silu", wrong)
        assert abs(sg.forward(p, X)["tau"][0, 2] - expect) > 1e-3
