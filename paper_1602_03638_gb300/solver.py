"""Python handle over the C ABI (argument marshalling only).

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA).
Every computation runs in the library's CUDA kernels; this module only
checks shapes/dtypes and passes pointers.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the runtime image
    torch = None


def _ptr(arr, shape, real_dtype_bytes, complex_):
    """(pointer, on_device) for a C-contiguous numpy array or torch tensor of the expected shape."""
    if torch is not None and isinstance(arr, torch.Tensor):
        if not arr.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if tuple(arr.shape) != tuple(shape):
            raise ValueError(f"expected shape {tuple(shape)}, got {tuple(arr.shape)}")
        want = {(4, False): torch.float32, (8, False): torch.float64, (4, True): torch.complex64, (8, True): torch.complex128}
        if arr.dtype != want[(real_dtype_bytes, complex_)]:
            raise ValueError(f"expected dtype {want[(real_dtype_bytes, complex_)]}, got {arr.dtype}")
        return ctypes.c_void_p(arr.data_ptr()), 1 if arr.is_cuda else 0
    if isinstance(arr, np.ndarray):
        if not arr.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        if tuple(arr.shape) != tuple(shape):
            raise ValueError(f"expected shape {tuple(shape)}, got {tuple(arr.shape)}")
        want = {(4, False): np.float32, (8, False): np.float64, (4, True): np.complex64, (8, True): np.complex128}
        if arr.dtype != want[(real_dtype_bytes, complex_)]:
            raise ValueError(f"expected dtype {np.dtype(want[(real_dtype_bytes, complex_)])}, got {arr.dtype}")
        return ctypes.c_void_p(arr.ctypes.data), 0
    raise TypeError("expected a numpy array or a torch tensor")


# explicit Runge-Kutta schemes of dns_step ("integrator" option of the C ABI)
INTEGRATORS = {"rk4": 0, "euler": 1, "heun": 2, "midpoint": 3, "williamson3": 4, "ck45": 5}


def set_tune_cache(path) -> None:
    """Keep the tuners' choices in a text file across runs (dns_set_tune_cache); None turns it off."""
    _lib.check(_lib.lib().dns_set_tune_cache(None if path is None else str(path).encode()), "dns_set_tune_cache")


def tune_cache_lookup(device: str, shape, dtype: str):
    """The stored tiles entry for (device, (Nx, Ny, Nz), dtype), or None:
    {"y_inverse", "y_forward", "z", "plan"}."""
    nx, ny, nz = _shape(shape)
    v = [ctypes.c_int() for _ in range(4)]
    rc = _lib.lib().dns_tune_cache_lookup(device.encode(), nx, ny, nz, {"f32": 0, "f64": 1}[dtype],
                                          *[ctypes.byref(x) for x in v])
    if rc < 0:
        _lib.check(rc, "dns_tune_cache_lookup")
    if rc == 0:
        return None
    return dict(zip(("y_inverse", "y_forward", "z", "plan"), (x.value for x in v)))


def _shape(N) -> tuple:
    """(Nx, Ny, Nz) from one point count or three."""
    if np.ndim(N) == 0:
        return (int(N),) * 3
    n = tuple(int(v) for v in N)
    if len(n) != 3:
        raise ValueError("N must be one point count or three (Nx, Ny, Nz)")
    return n


class Solver:
    """One dns_handle: N^3 grid (or N = (Nx, Ny, Nz), a compiled grid with other point
    counts per direction), viscosity nu, time step dt, 'f32' or 'f64'; integrator
    'rk4' (the Appendix driver, default), 'euler', 'heun' or 'midpoint'; box lengths
    (Lx, Ly, Lz), default (2 pi, 2 pi, 2 pi). ``shape`` is (Nx, Ny, Nz); ``N`` the count
    along x."""

    def __init__(self, N, nu: float, dt: float, dtype: str = "f32", dealias_variant: int = 0,
                 integrator: str = "rk4", lengths=None):
        if integrator not in INTEGRATORS:
            raise ValueError(f"integrator must be one of {sorted(INTEGRATORS)}, got {integrator!r}")
        self.shape = _shape(N)
        self.N = self.shape[0]
        self.dtype = dtype
        self._code = {"f32": _lib.DNS_F32, "f64": _lib.DNS_F64}[dtype]
        self._rb = 4 if dtype == "f32" else 8
        self._owned = True
        h = ctypes.c_void_p()
        nx, ny, nz = self.shape
        _lib.check(_lib.lib().dns_create3(nx, ny, nz, float(nu), float(dt), self._code, ctypes.byref(h)), "dns_create")
        self._h = h
        if dealias_variant:
            self.set_option("dealias_variant", dealias_variant)
        if integrator != "rk4":
            self.set_option("integrator", INTEGRATORS[integrator])
        if lengths is not None:  # box lengths (Lx, Ly, Lz); default 2 pi each
            for key, L in zip(("Lx", "Ly", "Lz"), lengths):
                self.set_option(key, float(L))

    @classmethod
    def _borrow(cls, handle: ctypes.c_void_p, N: int, dtype: str):
        """Wrap a handle owned elsewhere (an ensemble member); close() does not free it."""
        obj = cls.__new__(cls)
        obj.N, obj.dtype = int(N), dtype
        obj.shape = (obj.N,) * 3
        obj._code = {"f32": _lib.DNS_F32, "f64": _lib.DNS_F64}[dtype]
        obj._rb = 4 if dtype == "f32" else 8
        obj._owned = False
        obj._h = handle
        return obj

    # -- life cycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if getattr(self, "_owned", True):
                _lib.lib().dns_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- shapes ---------------------------------------------------------------
    @property
    def phys_shape(self):
        return (3,) + self.shape

    @property
    def spec_shape(self):
        nx, ny, nz = self.shape
        return (3, nx, ny, nz // 2 + 1)

    # -- calls ----------------------------------------------------------------
    def set_stream(self, stream=None):
        s = None
        if stream is not None:
            s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        _lib.check(_lib.lib().dns_set_stream(self._h, s), "dns_set_stream")

    def set_option(self, key: str, value: float):
        _lib.check(_lib.lib().dns_set_option(self._h, key.encode(), float(value)), "dns_set_option")

    def get_option(self, key: str) -> float:
        v = ctypes.c_double()
        _lib.check(_lib.lib().dns_get_option(self._h, key.encode(), ctypes.byref(v)), "dns_get_option")
        return v.value

    def set_closure(self, net=None, delta: float | None = None):
        """Attach a closure network (sgs.MLP) that every step evaluates on the device before its
        stages (dns_set_closure; FP32, 2 pi box); None detaches. delta: the filter-width feature
        (default 2 pi / N). The solver keeps a reference to the network while attached."""
        import math

        h = net._h if net is not None else None
        d = float(delta) if delta is not None else 2.0 * math.pi / self.N
        _lib.check(_lib.lib().dns_set_closure(self._h, h, d), "dns_set_closure")
        self._closure = net

    def set_rk_tableau(self, form: int, a, b=()):
        """A user-supplied explicit RK scheme (dns_set_rk_tableau): form 0 = the Appendix
        two-register form (weights a, offsets b), form 1 = Williamson's 2N form (A = a, B = b)."""
        av = (ctypes.c_double * max(1, len(a)))(*[float(x) for x in a])
        bv = (ctypes.c_double * max(1, len(b)))(*[float(x) for x in b])
        _lib.check(_lib.lib().dns_set_rk_tableau(self._h, int(form), len(a), av, bv), "dns_set_rk_tableau")

    def tune_tiles(self, steps: int = 5) -> tuple:
        """Time dns_step with each radix plan and y- and z-pass tile width the grid offers;
        keep the fastest plan (option "fft_plan") and (y_inverse, y_forward, z) widths
        (0 = default), returned. The state and time are left unchanged."""
        ti, tf, tz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(_lib.lib().dns_tune_tiles(self._h, int(steps), ctypes.byref(ti), ctypes.byref(tf), ctypes.byref(tz)),
                   "dns_tune_tiles")
        return ti.value, tf.value, tz.value

    def set_state(self, u):
        p, dev = _ptr(u, self.phys_shape, self._rb, False)
        _lib.check(_lib.lib().dns_set_state(self._h, p, dev), "dns_set_state")

    def set_state_spectral(self, uhat):
        p, dev = _ptr(uhat, self.spec_shape, self._rb, True)
        _lib.check(_lib.lib().dns_set_state_spectral(self._h, p, dev), "dns_set_state_spectral")

    def step(self, n: int = 1):
        _lib.check(_lib.lib().dns_step(self._h, int(n)), "dns_step")

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.phys_shape, dtype=np.float32 if self._rb == 4 else np.float64)
        p, dev = _ptr(out, self.phys_shape, self._rb, False)
        _lib.check(_lib.lib().dns_get_state(self._h, p, dev), "dns_get_state")
        return out

    def get_state_spectral(self, out=None):
        if out is None:
            out = np.empty(self.spec_shape, dtype=np.complex64 if self._rb == 4 else np.complex128)
        p, dev = _ptr(out, self.spec_shape, self._rb, True)
        _lib.check(_lib.lib().dns_get_state_spectral(self._h, p, dev), "dns_get_state_spectral")
        return out

    def rhs(self, out=None):
        if out is None:
            out = np.empty(self.spec_shape, dtype=np.complex64 if self._rb == 4 else np.complex128)
        p, dev = _ptr(out, self.spec_shape, self._rb, True)
        _lib.check(_lib.lib().dns_rhs(self._h, p, dev), "dns_rhs")
        return out

    def set_forcing(self, fhat=None):
        """A force (3, Nx, Ny, Nz/2+1) complex, paper order, added to the nonlinear term of every
        stage before the mask and the projection (dns_set_forcing); None removes it."""
        if fhat is None:
            _lib.check(_lib.lib().dns_set_forcing(self._h, None, 0), "dns_set_forcing")
            return
        p, dev = _ptr(fhat, self.spec_shape, self._rb, True)
        _lib.check(_lib.lib().dns_set_forcing(self._h, p, dev), "dns_set_forcing")

    def transform_r2c(self, phys, out):
        """The solver's forward 3D transform of 3 device fields (dns_transform_r2c): phys
        (3, Nx, Ny, Nz) real -> out (3, Nx, Ny, Nz/2+1) complex, unnormalised, Nyquist zeroed."""
        p, dev = _ptr(phys, self.phys_shape, self._rb, False)
        q, dev2 = _ptr(out, self.spec_shape, self._rb, True)
        if not (dev and dev2):
            raise ValueError("transform_r2c takes device arrays")
        _lib.check(_lib.lib().dns_transform_r2c(self._h, p, q), "dns_transform_r2c")
        return out

    def transform_c2r(self, spec, out):
        """The solver's inverse 3D transform of 3 device fields (dns_transform_c2r), with the
        1/(Nx Ny Nz) factor."""
        p, dev = _ptr(spec, self.spec_shape, self._rb, True)
        q, dev2 = _ptr(out, self.phys_shape, self._rb, False)
        if not (dev and dev2):
            raise ValueError("transform_c2r takes device arrays")
        _lib.check(_lib.lib().dns_transform_c2r(self._h, p, q), "dns_transform_c2r")
        return out

    def diagnostics(self, check_finite: bool = True) -> dict:
        d = _lib.dns_diag()
        rc = _lib.lib().dns_diagnostics(self._h, ctypes.byref(d))
        if check_finite or rc != _lib.DNS_ERR_NONFINITE:
            _lib.check(rc, "dns_diagnostics")
        return {k: getattr(d, k) for k, _ in d._fields_}

    KERNEL_CLASSES = ("y_inverse", "z_pass", "y_forward", "x_stage")

    def profile_steps(self, n: int) -> dict:
        """Advance n steps eagerly; per kernel class (total ms, launches)."""
        ms = (ctypes.c_double * 4)()
        ln = (ctypes.c_int * 4)()
        _lib.check(_lib.lib().dns_profile_steps(self._h, int(n), ms, ln, 4), "dns_profile_steps")
        return {k: (ms[i], ln[i]) for i, k in enumerate(self.KERNEL_CLASSES)}

    def device_bytes(self) -> int:
        return int(_lib.lib().dns_device_bytes(self._h))


class Ensemble:
    """dns_ensemble: independent members of mixed grid sizes stepped by one graph per step."""

    def __init__(self, Ns, nus, dts, dtype: str = "f32"):
        n = len(Ns)
        if not (len(nus) == len(dts) == n) or n == 0:
            raise ValueError("Ns, nus and dts must have the same non-zero length")
        code = {"f32": _lib.DNS_F32, "f64": _lib.DNS_F64}[dtype]
        e = ctypes.c_void_p()
        _lib.check(_lib.lib().dns_ensemble_create(n, (ctypes.c_int * n)(*[int(x) for x in Ns]),
                                                  (ctypes.c_double * n)(*[float(x) for x in nus]),
                                                  (ctypes.c_double * n)(*[float(x) for x in dts]), code,
                                                  ctypes.byref(e)), "dns_ensemble_create")
        self._e = e
        self.members = []
        for i, N in enumerate(Ns):
            h = ctypes.c_void_p()
            _lib.check(_lib.lib().dns_ensemble_member(e, i, ctypes.byref(h)), "dns_ensemble_member")
            self.members.append(Solver._borrow(h, N, dtype))

    def __len__(self):
        return len(self.members)

    def step(self, n: int = 1):
        _lib.check(_lib.lib().dns_ensemble_step(self._e, int(n)), "dns_ensemble_step")

    def tune(self) -> dict:
        """Pick the radix plan and the y- and z-pass tile widths per grid size and the
        schedule (batching, branch count) by timing; advances every member (see
        include/dns.h)."""
        k = ctypes.c_int()
        _lib.check(_lib.lib().dns_ensemble_tune(self._e, ctypes.byref(k)), "dns_ensemble_tune")
        tiles = {}
        for m in self.members:
            tiles.setdefault(m.N, {"y_inverse": int(m.get_option("y_tile_inverse")),
                                   "y_forward": int(m.get_option("y_tile_forward")),
                                   "z": int(m.get_option("z_tile")),
                                   "plan": int(m.get_option("fft_plan"))})
        return {"batching": self.batching, "streams": k.value, "tiles": tiles}

    def set_batching(self, max_batch: int):
        """0: every member runs its own kernels; n >= 1: up to n equal-size members share each launch."""
        _lib.check(_lib.lib().dns_ensemble_set_batching(self._e, int(max_batch)), "dns_ensemble_set_batching")

    @property
    def batching(self) -> int:
        return int(_lib.lib().dns_ensemble_batching(self._e))

    def set_streams(self, k: int):
        _lib.check(_lib.lib().dns_ensemble_set_streams(self._e, int(k)), "dns_ensemble_set_streams")

    @property
    def streams(self) -> int:
        return int(_lib.lib().dns_ensemble_streams(self._e))

    def time_steps(self, n: int) -> float:
        """n ensemble steps timed with CUDA events on the ensemble's stream; milliseconds."""
        ms = ctypes.c_double()
        _lib.check(_lib.lib().dns_ensemble_time_steps(self._e, int(n), ctypes.byref(ms)), "dns_ensemble_time_steps")
        return float(ms.value)

    def synchronize(self):
        _lib.check(_lib.lib().dns_ensemble_synchronize(self._e), "dns_ensemble_synchronize")

    def close(self):
        if getattr(self, "_e", None) is not None and self._e.value:
            for m in self.members:
                m._h = None
            _lib.lib().dns_ensemble_destroy(self._e)
            self._e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
