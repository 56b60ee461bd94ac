"""FP64 reference of the learned subgrid-stress (SGS) closure (TEST INFRASTRUCTURE).

Imported only by the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py``. The paper itself has no closure model: this restates the
closure chosen for the coarse-grid runs, built on the solver's own transforms
(Sec. 2 conventions, see spectral_ns):

  * box filter of width D = 2 pi / Nc applied in spectral space with the
    transfer function G(k) = prod_i sinc(k_i D / 2), sinc(x) = sin(x)/x,
    followed by truncation to the modes |k_i| < Nc/2 of an Nc^3 grid;
    coarse coefficients are (Nc/Nf)^3 G(k) u_hat_fine(k) (unnormalised DFTs);
  * resolved velocity gradients A_ij = d ubar_i / d x_j = F^{-1}(i k_j ubar_hat_i),
    order (i, j) row-major: du/dx, du/dy, du/dz, dv/dx, ...;
  * SGS stress tau_ij = filter(u_i u_j) - ubar_i ubar_j, components
    (00, 11, 22, 01, 02, 12);
  * the pointwise network: 10 inputs (the 9 A_ij and D) -> 64 SiLU -> 64 SiLU ->
    6 linear outputs, with per-feature input standardisation and per-component
    output scaling, loss = mean squared error of the standardised stress;
  * the force the closure adds to the coarse right-hand side before the 2/3
    mask and the projection: f_i = -i k_j tau_hat_ij (= -d tau_ij / d x_j);
  * training by Adam (Kingma & Ba 2015, Algorithm 1: first and second moment
    estimates with bias correction, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on
    the weights and biases; the normalisation entries stay fixed.

Parity: pinned by closed forms (single-mode filter, stress of cos(a x), force
of sin(2x)), by a sparse network whose output is a hand-computed composition of
logistic functions (forward), by forces that the projection or the mask must
remove and a solenoidal single-mode force that must pass unchanged (rhs_forced),
by two hand-computed Adam steps on a scalar (adam_step), and by central finite
differences of the network gradient.
"""

from __future__ import annotations

import numpy as np

from . import spectral_ns as sn

TAU_INDEX = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
N_IN, N_HID, N_OUT = 10, 64, 6


def _fft_k(N):
    return np.array([j if j < N // 2 else j - N for j in range(N)], dtype=np.int64)


def _sinc(x):
    return np.where(np.abs(x) < 1e-12, 1.0, np.sin(x) / np.where(np.abs(x) < 1e-12, 1.0, x))


def filter_truncate(uh_f: np.ndarray, Nc: int) -> np.ndarray:
    """Box-filter (width 2 pi/Nc) a fine half spectrum (..., Nf, Nf, Nf/2+1) and keep |k_i| < Nc/2."""
    Nf = uh_f.shape[-3]
    D = 2.0 * np.pi / Nc
    kc = _fft_k(Nc)
    out = np.zeros(uh_f.shape[:-3] + (Nc, Nc, Nc // 2 + 1), dtype=np.complex128)
    for a, kx in enumerate(kc):
        if abs(kx) >= Nc // 2:
            continue
        for b, ky in enumerate(kc):
            if abs(ky) >= Nc // 2:
                continue
            kz = np.arange(Nc // 2)
            g = _sinc(kx * D / 2) * _sinc(ky * D / 2) * _sinc(kz * D / 2)
            out[..., a, b, : Nc // 2] = uh_f[..., kx % Nf, ky % Nf, : Nc // 2] * g
    return out * (Nc / Nf) ** 3


def velocity_gradients(uh: np.ndarray) -> np.ndarray:
    """A_ij = F^{-1}(i k_j u_hat_i), shape (9, N, N, N), (i, j) row-major."""
    N = uh.shape[-3]
    K = sn.wavenumbers(N)
    out = np.empty((9, N, N, N))
    for i in range(3):
        for j in range(3):
            out[3 * i + j] = sn.inverse(1j * K[j] * uh[i])
    return out


def sgs_stress(uh_f: np.ndarray, Nc: int) -> tuple[np.ndarray, np.ndarray]:
    """(tau (6,Nc,Nc,Nc), ubar_hat (3,Nc,Nc,Nc/2+1)) from a fine spectral velocity."""
    u = sn.inverse(uh_f)
    ubh = filter_truncate(uh_f, Nc)
    ub = sn.inverse(ubh)
    tau = np.empty((6, Nc, Nc, Nc))
    for c, (i, j) in enumerate(TAU_INDEX):
        pbar = sn.inverse(filter_truncate(sn.forward(u[i] * u[j]), Nc))
        tau[c] = pbar - ub[i] * ub[j]
    return tau, ubh


def stress_force(tau: np.ndarray) -> np.ndarray:
    """f_hat_i = -i k_j tau_hat_ij for a physical stress (6, N, N, N)."""
    N = tau.shape[-1]
    K = sn.wavenumbers(N)
    th = sn.forward(tau)
    full = {}
    for c, (i, j) in enumerate(TAU_INDEX):
        full[(i, j)] = th[c]
        full[(j, i)] = th[c]
    f = np.zeros((3,) + th.shape[1:], dtype=np.complex128)
    for i in range(3):
        for j in range(3):
            f[i] += -1j * K[j] * full[(i, j)]
    return f


def rhs_forced(uh: np.ndarray, g: sn.Grid, nu: float, fh: np.ndarray) -> np.ndarray:
    """Eq. NSfinal with an extra force added to the nonlinear term before the mask and the projection."""
    nh = sn.nonlinear_hat(uh, g) + fh * g.mask
    return sn.project(nh, g) - nu * g.K2 * uh


# --------------------------------------------------------------------------
# Pointwise network
# --------------------------------------------------------------------------

def bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16 (nearest, ties to even) and return them as float64."""
    a = np.asarray(x, dtype=np.float32).copy()
    bits = a.view(np.uint32).astype(np.uint64)
    rounding = ((bits >> 16) & 1) + 0x7FFF
    bits = ((bits + rounding) >> 16) << 16
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int = 0) -> dict:
    """Glorot-uniform weights, zero biases, identity normalisation."""
    rng = np.random.default_rng(seed)

    def glorot(n_in, n_out):
        lim = np.sqrt(6.0 / (n_in + n_out))
        return rng.uniform(-lim, lim, size=(n_in, n_out))

    return {
        "in_shift": np.zeros(N_IN), "in_scale": np.ones(N_IN),
        "W1": glorot(N_IN, N_HID), "b1": np.zeros(N_HID),
        "W2": glorot(N_HID, N_HID), "b2": np.zeros(N_HID),
        "W3": glorot(N_HID, N_OUT), "b3": np.zeros(N_OUT),
        "out_scale": np.ones(N_OUT), "out_shift": np.zeros(N_OUT),
    }


PARAM_ORDER = ("in_shift", "in_scale", "W1", "b1", "W2", "b2", "W3", "b3", "out_scale", "out_shift")


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in PARAM_ORDER])


def unflatten(v: np.ndarray) -> dict:
    shapes = {"in_shift": (N_IN,), "in_scale": (N_IN,), "W1": (N_IN, N_HID), "b1": (N_HID,),
              "W2": (N_HID, N_HID), "b2": (N_HID,), "W3": (N_HID, N_OUT), "b3": (N_OUT,),
              "out_scale": (N_OUT,), "out_shift": (N_OUT,)}
    out, o = {}, 0
    for k in PARAM_ORDER:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shapes[k])
        o += n
    return out


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p: dict, X: np.ndarray, round_bf16: bool = False) -> dict:
    """X: (P, 10) raw features. Returns the activations and y (P, 6, standardised) and tau (P, 6).

    round_bf16 mimics tensor-core inputs: the standardised features, the
    weights and the hidden activations are rounded to bfloat16 before each
    product; sums and the nonlinearity stay in float64.
    """
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    xn = (X - p["in_shift"]) * p["in_scale"]
    z1 = r(xn) @ r(p["W1"]) + p["b1"]
    h1 = _silu(z1)
    z2 = r(h1) @ r(p["W2"]) + p["b2"]
    h2 = _silu(z2)
    y = r(h2) @ r(p["W3"]) + p["b3"]
    tau = y * p["out_scale"] + p["out_shift"]
    return {"xn": xn, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "y": y, "tau": tau}


def loss_and_grads(p: dict, X: np.ndarray, T: np.ndarray, round_bf16: bool = False) -> tuple[float, dict]:
    """Mean squared error of the standardised stress and its gradients w.r.t. W1, b1, W2, b2, W3, b3.

    T: (P, 6) target stress; the standardised target is (T - out_shift) / out_scale.
    """
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    a = forward(p, X, round_bf16)
    P = X.shape[0]
    tn = (T - p["out_shift"]) / p["out_scale"]
    d = a["y"] - tn
    loss = float(np.mean(d * d))
    dy = 2.0 * d / (P * N_OUT)
    g = {"W3": r(a["h2"]).T @ dy, "b3": dy.sum(0)}
    dh2 = dy @ r(p["W3"]).T
    dz2 = dh2 * _dsilu(a["z2"])
    g["W2"] = r(a["h1"]).T @ dz2
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ r(p["W2"]).T
    dz1 = dh1 * _dsilu(a["z1"])
    g["W1"] = r(a["xn"]).T @ dz1
    g["b1"] = dz1.sum(0)
    return loss, g


# --------------------------------------------------------------------------
# Optimiser
# --------------------------------------------------------------------------

TRAINABLE = ("W1", "b1", "W2", "b2", "W3", "b3")


def adam_init(p: dict) -> dict:
    """Zero first and second moments for the trainable entries, step counter 0."""
    return {"t": 0, "m": {k: np.zeros_like(np.asarray(p[k], dtype=np.float64)) for k in TRAINABLE},
            "v": {k: np.zeros_like(np.asarray(p[k], dtype=np.float64)) for k in TRAINABLE}}


def adam_step(p: dict, g: dict, state: dict, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> tuple[dict, dict]:
    """One Adam update of the trainable entries (Kingma & Ba 2015, Algorithm 1), in float64.

    With t the new step count: m <- beta1 m + (1 - beta1) g, v <- beta2 v + (1 - beta2) g^2,
    p <- p - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps). Entries not in
    TRAINABLE are copied unchanged. Returns (new parameters, new state).
    """
    t = state["t"] + 1
    q = {k: np.array(v, dtype=np.float64, copy=True) for k, v in p.items()}
    m_new, v_new = {}, {}
    for k in TRAINABLE:
        gk = np.asarray(g[k], dtype=np.float64)
        m_new[k] = beta1 * state["m"][k] + (1.0 - beta1) * gk
        v_new[k] = beta2 * state["v"][k] + (1.0 - beta2) * gk * gk
        m_hat = m_new[k] / (1.0 - beta1 ** t)
        v_hat = v_new[k] / (1.0 - beta2 ** t)
        q[k] = q[k] - lr * m_hat / (np.sqrt(v_hat) + eps)
    return q, {"t": t, "m": m_new, "v": v_new}
