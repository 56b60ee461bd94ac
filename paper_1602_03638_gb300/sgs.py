"""Learned subgrid-stress closure for coarse-grid runs (argument marshalling over the C ABI).

Every array operation of the closure runs in the library's CUDA kernels:
transforms (dns_transform_r2c/c2r), box filter and truncation
(dns_spectral_filter), gradient features (dns_spectral_gradient), stress
(dns_pointwise_products, dns_subtract_products), the network
(dns_mlp_forward/train_step on BF16 tensor cores) and the closure force
(dns_stress_force + dns_set_forcing). torch only provides device buffers.

Workflow
  1. fine DNS (this solver) -> snapshots
  2. filtered_training_data(): ubar, gradient features X (10 x P), stress T (6 x P)
  3. MLP.fit(): Adam on the standardised stress, BF16 products, FP32 weights
  4. set_closure_force(): before each coarse step, f = -div(MLP(grad ubar))
"""

from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib
from .solver import Solver

N_IN, N_OUT = 10, 6


def _p(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _code(dtype: str) -> int:
    return _lib.DNS_F32 if dtype == "f32" else _lib.DNS_F64


def _cdt(dtype: str):
    return torch.complex64 if dtype == "f32" else torch.complex128


def _rdt(dtype: str):
    return torch.float32 if dtype == "f32" else torch.float64


# ------------------------------------------------------------------ primitives

def spectral_filter(fine_hat: torch.Tensor, Nc: int, dtype: str = "f32") -> torch.Tensor:
    Nf = fine_hat.shape[-3]
    out = torch.empty((fine_hat.shape[0], Nc, Nc, Nc // 2 + 1), dtype=_cdt(dtype), device=fine_hat.device)
    assert fine_hat.shape[0] == 3
    _lib.check(_lib.lib().dns_spectral_filter(_p(fine_hat), Nf, _p(out), Nc, _code(dtype), _stream()),
               "dns_spectral_filter")
    return out


def spectral_gradient(uhat: torch.Tensor, dtype: str = "f32") -> torch.Tensor:
    N = uhat.shape[-3]
    out = torch.empty((9, N, N, N // 2 + 1), dtype=_cdt(dtype), device=uhat.device)
    _lib.check(_lib.lib().dns_spectral_gradient(_p(uhat), N, _p(out), _code(dtype), _stream()), "dns_spectral_gradient")
    return out


def stress_force(tauhat: torch.Tensor, dtype: str = "f32") -> torch.Tensor:
    N = tauhat.shape[-3]
    out = torch.empty((3, N, N, N // 2 + 1), dtype=_cdt(dtype), device=tauhat.device)
    _lib.check(_lib.lib().dns_stress_force(_p(tauhat), N, _p(out), _code(dtype), _stream()), "dns_stress_force")
    return out


def pointwise_products(u: torch.Tensor, dtype: str = "f32") -> torch.Tensor:
    N = u.shape[-1]
    out = torch.empty((6, N, N, N), dtype=_rdt(dtype), device=u.device)
    _lib.check(_lib.lib().dns_pointwise_products(_p(u), N, _p(out), _code(dtype), _stream()), "dns_pointwise_products")
    return out


def subtract_products(tau: torch.Tensor, ubar: torch.Tensor, dtype: str = "f32") -> torch.Tensor:
    N = ubar.shape[-1]
    _lib.check(_lib.lib().dns_subtract_products(_p(tau), _p(ubar), N, _code(dtype), _stream()), "dns_subtract_products")
    return tau


def r2c(solver: Solver, phys: torch.Tensor) -> torch.Tensor:
    """F of a (3k, N, N, N) device tensor, k fields at a time through the solver's transforms."""
    N = solver.N
    n = phys.shape[0]
    out = torch.empty((n, N, N, N // 2 + 1), dtype=_cdt(solver.dtype), device=phys.device)
    for i in range(0, n, 3):
        _lib.check(_lib.lib().dns_transform_r2c(solver.handle, _p(phys[i:i + 3]), _p(out[i:i + 3])), "dns_transform_r2c")
    return out


def c2r(solver: Solver, spec: torch.Tensor) -> torch.Tensor:
    N = solver.N
    n = spec.shape[0]
    out = torch.empty((n, N, N, N), dtype=_rdt(solver.dtype), device=spec.device)
    for i in range(0, n, 3):
        _lib.check(_lib.lib().dns_transform_c2r(solver.handle, _p(spec[i:i + 3]), _p(out[i:i + 3])), "dns_transform_c2r")
    return out


def on_torch_stream(*solvers: Solver):
    """Puts the solvers on torch's current stream, so that their transforms and the
    closure kernels (launched on that stream) are ordered without host waits."""
    st = torch.cuda.current_stream()
    for s in solvers:
        s.set_stream(st)


# ------------------------------------------------------------------ data

def gradient_features(coarse: Solver, ubar_hat: torch.Tensor) -> torch.Tensor:
    """X (10, P): the 9 resolved gradients d ubar_i / d x_j and the filter width 2 pi/N."""
    Nc = coarse.N
    g9 = c2r(coarse, spectral_gradient(ubar_hat, coarse.dtype))
    torch.cuda.synchronize()
    X = torch.empty((N_IN, Nc ** 3), dtype=torch.float32, device=ubar_hat.device)
    X[:9] = g9.reshape(9, -1).to(torch.float32)
    X[9] = 2.0 * math.pi / Nc
    return X


def filtered_training_data(fine: Solver, coarse: Solver):
    """(X (10,P), T (6,P), ubar_hat) from the fine solver's current state.

    ubar = box filter (width 2 pi/Nc) + truncation of u; T = filter(u_i u_j) - ubar_i ubar_j
    on the coarse grid. The fine solver's state is not changed.
    """
    Nf, Nc, dt = fine.N, coarse.N, fine.dtype
    dev = "cuda"
    on_torch_stream(fine, coarse)
    uh = torch.empty(fine.spec_shape, dtype=_cdt(dt), device=dev)
    fine.get_state_spectral(uh)
    u = torch.empty(fine.phys_shape, dtype=_rdt(dt), device=dev)
    fine.get_state(u)
    torch.cuda.synchronize()
    prod = pointwise_products(u, dt)
    del u
    torch.cuda.synchronize()
    pbar_hat = torch.empty((6, Nc, Nc, Nc // 2 + 1), dtype=_cdt(dt), device=dev)
    for i in (0, 3):
        spec = r2c(fine, prod[i:i + 3])
        torch.cuda.synchronize()
        pbar_hat[i:i + 3] = spectral_filter(spec, Nc, dt)
        del spec
    del prod
    ubar_hat = spectral_filter(uh, Nc, dt)
    torch.cuda.synchronize()
    tau = c2r(coarse, pbar_hat)
    ubar = c2r(coarse, ubar_hat)
    torch.cuda.synchronize()
    subtract_products(tau, ubar, dt)
    X = gradient_features(coarse, ubar_hat)
    T = tau.reshape(6, -1).to(torch.float32)
    torch.cuda.synchronize()
    return X, T.contiguous(), ubar_hat


# ------------------------------------------------------------------ network

class MLP:
    """The BF16 tensor-core network (dns_mlp)."""

    PARAM_COUNT = 5286

    def __init__(self, params: np.ndarray | None = None, seed: int = 0):
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().dns_mlp_create(ctypes.byref(h)), "dns_mlp_create")
        self._h = h
        assert _lib.lib().dns_mlp_param_count() == self.PARAM_COUNT
        self.set_params(params if params is not None else init_params(seed))

    def set_params(self, v: np.ndarray):
        v = np.ascontiguousarray(v, dtype=np.float32)
        _lib.check(_lib.lib().dns_mlp_set_params(self._h, v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), v.size),
                   "dns_mlp_set_params")

    def get_params(self) -> np.ndarray:
        v = np.empty(self.PARAM_COUNT, dtype=np.float32)
        _lib.check(_lib.lib().dns_mlp_get_params(self._h, v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), v.size),
                   "dns_mlp_get_params")
        return v

    def set_normalisation(self, X: torch.Tensor, T: torch.Tensor):
        """in_shift/in_scale and out_scale/out_shift from the mean and unbiased std of the rows of
        the device arrays X (10, P) and T (6, P), computed by a device kernel (constant features
        keep scale 1); the Adam state is kept."""
        _lib.check(_lib.lib().dns_mlp_set_normalisation(self._h, _p(X), _p(T), X.shape[1], _stream()),
                   "dns_mlp_set_normalisation")

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        P = X.shape[1]
        Y = torch.empty((N_OUT, P), dtype=torch.float32, device=X.device)
        _lib.check(_lib.lib().dns_mlp_forward(self._h, _p(X), _p(Y), P, _stream()), "dns_mlp_forward")
        return Y

    def loss_grad(self, X: torch.Tensor, T: torch.Tensor):
        g = np.empty(self.PARAM_COUNT, dtype=np.float32)
        loss = ctypes.c_float()
        _lib.check(_lib.lib().dns_mlp_loss_grad(self._h, _p(X), _p(T), X.shape[1],
                                                g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                ctypes.byref(loss), _stream()), "dns_mlp_loss_grad")
        return float(loss.value), g

    def train_step(self, X: torch.Tensor, T: torch.Tensor, lr: float, want_loss: bool = True):
        loss = ctypes.c_float()
        _lib.check(_lib.lib().dns_mlp_train_step(self._h, _p(X), _p(T), X.shape[1], float(lr),
                                                 ctypes.byref(loss) if want_loss else None, _stream()),
                   "dns_mlp_train_step")
        return float(loss.value) if want_loss else None

    def fit(self, X: torch.Tensor, T: torch.Tensor, iters: int, lr: float = 1e-3, batch: int = 65536,
            seed: int = 0, log_every: int = 0):
        """Adam on random minibatches (index gathers on the device); returns the loss history."""
        g = torch.Generator(device=X.device)
        g.manual_seed(seed)
        P = X.shape[1]
        hist = []
        for it in range(iters):
            idx = torch.randint(0, P, (min(batch, P),), device=X.device, generator=g)
            xb, tb = X[:, idx].contiguous(), T[:, idx].contiguous()
            want = log_every > 0 and (it % log_every == 0 or it == iters - 1)
            loss = self.train_step(xb, tb, lr, want_loss=want)
            if want:
                hist.append((it, loss))
        return hist

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().dns_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases, identity normalisation (the layout of include/dns.h)."""
    rng = np.random.default_rng(seed)

    def glorot(n_in, n_out):
        lim = math.sqrt(6.0 / (n_in + n_out))
        return rng.uniform(-lim, lim, size=(n_in, n_out))

    parts = [np.zeros(10), np.ones(10), glorot(10, 64), np.zeros(64), glorot(64, 64), np.zeros(64),
             glorot(64, 6), np.zeros(6), np.ones(6), np.zeros(6)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def with_normalisation(params: np.ndarray, X: torch.Tensor, T: torch.Tensor) -> np.ndarray:
    """The parameter vector with in_shift/in_scale and out_scale/out_shift set from the data
    statistics (MLP.set_normalisation on a temporary network)."""
    m = MLP(params)
    m.set_normalisation(X.contiguous(), T.contiguous())
    v = m.get_params()
    m.close()
    return v


# ------------------------------------------------------------------ coarse runs

def set_closure_force(coarse: Solver, mlp: MLP):
    """Forcing f = -i k_j tau_hat_ij with tau = MLP(grad ubar) from the coarse solver's current state,
    composed from the library's separate calls (public layout, host waits between them): the
    reference the in-step closure of dns_set_closure is tested against."""
    dev = "cuda"
    on_torch_stream(coarse)
    uh = torch.empty(coarse.spec_shape, dtype=_cdt(coarse.dtype), device=dev)
    coarse.get_state_spectral(uh)
    X = gradient_features(coarse, uh)
    tau = mlp.forward(X).reshape(6, coarse.N, coarse.N, coarse.N)
    if coarse.dtype != "f32":
        tau = tau.to(_rdt(coarse.dtype))
    torch.cuda.synchronize()
    tauhat = r2c(coarse, tau.contiguous())
    torch.cuda.synchronize()
    f = stress_force(tauhat, coarse.dtype)
    torch.cuda.synchronize()
    _lib.check(_lib.lib().dns_set_forcing(coarse.handle, _p(f), 1), "dns_set_forcing")
    torch.cuda.synchronize()


def run_coarse(coarse: Solver, steps: int, mlp: MLP | None = None):
    """Advance the coarse solver; with a network, the closure force is evaluated by the solver
    itself at the start of every step (dns_set_closure: features, network, stress force and
    forcing inside the step graph, held over its four RK4 stages); None detaches it."""
    coarse.set_closure(mlp)
    coarse.step(steps)
    torch.cuda.synchronize()


def energy_spectrum(uhat: np.ndarray) -> np.ndarray:
    """Shell spectrum E(k), k = round(|k|), of a public-layout half spectrum (evaluation helper)."""
    N = uhat.shape[-3]
    k = np.array([j if j < N // 2 else j - N for j in range(N)])
    kz = np.arange(N // 2 + 1)
    KX, KY, KZ = np.meshgrid(k, k, kz, indexing="ij")
    kk = np.rint(np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)).astype(int)
    w = np.where((KZ == 0) | (KZ == N // 2), 1.0, 2.0)
    e = 0.5 * w * np.sum(np.abs(uhat) ** 2, axis=0) / float(N) ** 6
    return np.bincount(kk.ravel(), weights=e.ravel())


def spectrum_error(uh_model: np.ndarray, uh_ref: np.ndarray, kmax: int) -> float:
    """Relative L2 error of the shell spectra over 1 <= k < kmax."""
    a = energy_spectrum(uh_model)[1:kmax]
    b = energy_spectrum(uh_ref)[1:kmax]
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def eddy_turnover(s: Solver) -> dict:
    """Large-eddy turnover time T_e = L / u' of a solver state (evaluation helper):
    u' = sqrt(2E/3), L = pi / (2 u'^2) * sum_k E(k)/k over the shell spectrum, k = round(|k|) >= 1."""
    N = s.N
    uh = torch.empty(s.spec_shape, dtype=torch.complex64 if s.dtype == "f32" else torch.complex128, device="cuda")
    s.get_state_spectral(uh)
    k = torch.fft.fftfreq(N, 1.0 / N, device="cuda")
    kz = torch.arange(N // 2 + 1, device="cuda", dtype=k.dtype)
    kk = torch.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + kz[None, None, :] ** 2).round().long()
    w = torch.where((kz == 0) | (kz == N // 2), 1.0, 2.0).to(torch.float64)
    e = (0.5 / float(N) ** 6) * w * (uh.abs() ** 2).sum(0).to(torch.float64)
    spec = torch.bincount(kk.reshape(-1), weights=e.reshape(-1)).cpu().numpy()
    energy = float(spec.sum())
    up = math.sqrt(2.0 * energy / 3.0)
    shells = np.arange(1, spec.size)
    L = math.pi / (2.0 * up * up) * float(np.sum(spec[1:] / shells))
    return {"energy": energy, "u_rms": up, "integral_scale": L, "T_e": L / up}


def _device_ms(fn) -> float:
    """Milliseconds between CUDA events on torch's current stream around fn()."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    e0.record(st)
    fn()
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1)


def closure_experiment(Nf: int = 512, Nc: int = 64, nu: float = 2e-3, dt_f: float = 1e-3, dt_c: float = 4e-3,
                       k0: float = 4.0, seed: int = 0, t_dev: float = 0.3, t_run: float | None = None, snaps: int = 3,
                       checkpoints: int = 4, iters: int = 600, batch: int = 65536, lr: float = 2e-3) -> dict:
    """Fine DNS -> filtered training data -> GPU training -> coarse runs with and without the closure.

    The fine field (FP32, isotropic, energy 1, spectrum k^4 exp(-2 (k/k0)^2)) develops until t_dev;
    training snapshots are taken at t_dev * i / snaps (i = 1..snaps). Both coarse runs start from
    the filtered fine state at t_dev and are compared with the filtered DNS at `checkpoints` equally
    spaced times up to t_dev + t_run: relative L2 error of the shell spectrum over 1 <= k < Nc/3 and
    relative error of the resolved dissipation nu <|curl ubar|^2>. t_run = None runs two large-eddy
    turnover times of the fine field at t_dev.
    """
    import time

    from . import inputs

    dev = "cuda"
    out = {"Nf": Nf, "Nc": Nc, "nu": nu, "dt_fine": dt_f, "dt_coarse": dt_c, "k0": k0, "t_dev": t_dev, "t_run": t_run}
    fine = Solver(Nf, nu, dt_f, "f32")
    tool = Solver(Nc, nu, dt_c, "f32")
    on_torch_stream(fine, tool)
    fine.set_state_spectral(inputs.isotropic_spectral(Nf, seed=seed, k0=k0, energy=1.0, device=dev).to(torch.complex64))
    Xs, Ts = [], []
    n_dev = int(round(t_dev / dt_f))
    t0 = time.perf_counter()
    done = 0
    for i in range(1, snaps + 1):
        target = int(round(n_dev * i / snaps))
        fine.step(target - done)
        done = target
        X, T, ubh = filtered_training_data(fine, tool)
        Xs.append(X)
        Ts.append(T)
    torch.cuda.synchronize()
    out["dns_develop_s"] = time.perf_counter() - t0
    X = torch.cat(Xs, dim=1).contiguous()
    T = torch.cat(Ts, dim=1).contiguous()
    out["training_points"] = int(X.shape[1])
    out["eddy"] = eddy_turnover(fine)
    if t_run is None:
        t_run = 2.0 * out["eddy"]["T_e"]
    out["t_run"] = t_run
    net = MLP(seed=seed)
    net.set_normalisation(X, T)
    t0 = time.perf_counter()
    hist = net.fit(X, T, iters=iters, lr=lr, batch=batch, seed=seed, log_every=max(1, iters // 5))
    torch.cuda.synchronize()
    out["train_s"] = time.perf_counter() - t0
    out["train_loss"] = hist
    ub0 = ubh.clone()

    def coarse_from(uh):
        s = Solver(Nc, nu, dt_c, "f32")
        on_torch_stream(s)
        s.set_state_spectral(uh)
        return s

    plain, model = coarse_from(ub0), coarse_from(ub0)
    n_c = max(1, int(round(t_run / dt_c / checkpoints)))
    n_f = int(round(n_c * dt_c / dt_f))  # the same physical time per checkpoint
    rec = []
    t_plain = t_model = t_dns = 0.0
    for c in range(1, checkpoints + 1):
        t0 = time.perf_counter()
        fine.step(n_f)
        torch.cuda.synchronize()
        t_dns += time.perf_counter() - t0
        _, _, ref = filtered_training_data(fine, tool)
        t_plain += _device_ms(lambda: run_coarse(plain, n_c, None))
        t_model += _device_ms(lambda: run_coarse(model, n_c, net))
        tool.set_state_spectral(ref)
        d_ref = tool.diagnostics()["dissipation"]
        refn = ref.cpu().numpy()
        row = {"t": t_dev + c * n_f * dt_f}
        for name, s in (("no_model", plain), ("model", model)):
            uh = torch.empty(s.spec_shape, dtype=torch.complex64, device=dev)
            s.get_state_spectral(uh)
            d = s.diagnostics()["dissipation"]
            row[name] = {"spectrum_err": spectrum_error(uh.cpu().numpy(), refn, Nc // 3),
                         "dissipation_err": abs(d - d_ref) / d_ref}
        rec.append(row)
    out["checkpoints"] = rec
    out["final"] = rec[-1]
    out["coarse_ms_per_step_no_model"] = t_plain / (checkpoints * n_c)
    out["coarse_ms_per_step_model"] = t_model / (checkpoints * n_c)
    out["coarse_timing"] = "CUDA events on the solvers' stream around each checkpoint's steps"
    out["dns_ms_per_step"] = 1e3 * t_dns / (checkpoints * n_f)
    for s in (plain, model, tool, fine):
        s.close()
    net.close()
    return out
