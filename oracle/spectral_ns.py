"""Plain FP64 pseudo-spectral Navier-Stokes solver (the oracle).

TEST INFRASTRUCTURE: imported only by the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``. The GPU library never calls it.

Every function follows one passage of Mortensen & Langtangen (arXiv
1602.03638) and says which. No blocking, fusion or reordering is done beyond
what the paper states; the library FFT (scipy.fft, pocketfft) is used as the
transform primitive, exactly as the paper's solver uses numpy.fft/pyFFTW.

Array conventions (Sec. 3.1)
----------------------------
physical   u[c, i, j, k] = u_c(x_i, y_j, z_k),  x_i = 2*pi*i/N       (Eq. realmesh)
spectral  uh[c, l, m, n]: kx = fftfreq order over l, ky = fftfreq order
           over m, kz = n = 0..N/2 with the last entry stored as +N/2
           (the wavenumber listing of Sec. 3.1; Eq. kmesh)
Every function also takes per-direction point counts (Nx, Ny, Nz) (the Sec. 2
footnote: other numbers of points per direction); N then stands for the count of
the direction in question, and N^3 for Nx Ny Nz.

Readings of the paper that this module takes (each is stated where used):
  * F is the unnormalised forward transform with e^{-ik.x}; F^{-1} carries
    1/N^3 (Sec. 2: the labels of Eqs. ffteq/iffteq are swapped relative to
    the formulas; rfftn/irfftn of Sec. 3.1 fix the convention).
  * The state is kept free of Nyquist modes (any |k_i| = N/2 zeroed on input);
    the RHS keeps them zero because they lie outside the dealiasing box.
  * The complex-to-real step along z ignores the imaginary parts of the kz=0
    and kz=N/2 coefficients (pocketfft/FFTW c2r semantics).
  * Dealiasing cut-off |k_i| < N/3 (Sec. 3.1 text); the Appendix script's
    2/3*(N/2+1) is dealias_variant=1.
"""

from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

WORKERS = max(1, len(os.sched_getaffinity(0))) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)

# Classical RK4 weights of the Appendix driver: a = stage weights, b = stage offsets.
RK4_A = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)
RK4_B = (0.5, 0.5, 1.0)

# Explicit Runge-Kutta schemes in the same two-register form (stage s + 1 starts
# from u0 + b_s dt dU_s, the new state is u0 + sum_s a_s dt dU_s): the Appendix's
# RK4, the forward Euler loop of Sec. 3.1, and the two-stage Heun and midpoint
# rules (textbook Butcher tableaux with c = (0, 1) and (0, 1/2)).
RK_SCHEMES = {
    "rk4": (RK4_A, RK4_B),
    "euler": ((1.0,), ()),
    "heun": ((0.5, 0.5), (1.0,)),
    "midpoint": ((0.0, 1.0), (0.5,)),
}


# Low-storage explicit Runge-Kutta schemes in Williamson's 2N form (Williamson 1980,
# J. Comput. Phys. 35): two registers u and dU; stage j does dU <- A_j dU + dt RHS(u),
# then u <- u + B_j dU, with A_1 = 0. The Sec. 3.1 remark that more advanced
# integrators may be added is read as this family (the paper names none).
# "williamson3": Williamson's three-stage third-order scheme; "ck45": the five-stage
# fourth-order scheme of Carpenter & Kennedy (1994, NASA TM-109112).
LSRK_SCHEMES = {
    "williamson3": ((0.0, -5.0 / 9.0, -153.0 / 128.0), (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)),
    "ck45": ((0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
              -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0),
             (1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
              1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
              2277821191437.0 / 14882151754819.0)),
}


def set_workers(n: int) -> None:
    """Thread count for the library FFT (the CPU baseline reports it)."""
    global WORKERS
    WORKERS = max(1, int(n))


# --------------------------------------------------------------------------
# Mesh and wavenumbers (Eq. realmesh, Eq. kmesh, Sec. 3.1)
# --------------------------------------------------------------------------

def dims(N) -> tuple:
    """(Nx, Ny, Nz) from one point count or three (Sec. 2 footnote: the number of points
    may differ per direction); each must be even."""
    n = (int(N),) * 3 if np.ndim(N) == 0 else tuple(int(v) for v in N)
    if len(n) != 3 or any(v < 2 or v % 2 for v in n):
        raise ValueError("N must be even in every direction")
    return n


def shape_of(uh: np.ndarray) -> tuple:
    """(Nx, Ny, Nz) of a half spectrum (..., Nx, Ny, Nz/2+1)."""
    return (uh.shape[-3], uh.shape[-2], 2 * (uh.shape[-1] - 1))


def mesh(N, lengths=None) -> np.ndarray:
    """Physical mesh x_i = 2*pi*i/N in each direction (Eq. realmesh); shape (3,Nx,Ny,Nz).
    With box lengths (Lx, Ly, Lz) (Sec. 2 footnote) x_i = Lx*i/Nx, and so on; N may be
    one point count or three (Nx, Ny, Nz)."""
    n = dims(N)
    L = (2.0 * np.pi,) * 3 if lengths is None else tuple(float(v) for v in lengths)
    xs = [L[d] * np.arange(n[d], dtype=np.float64) / n[d] for d in range(3)]
    return np.array(np.meshgrid(*xs, indexing="ij"))


def wavenumbers(N) -> np.ndarray:
    """Integer wavenumber mesh K of shape (3, Nx, Ny, Nz/2+1) (Sec. 3.1).

    kx and ky follow the FFT ordering (0..N/2-1, -N/2..-1) of their own point
    counts; kz is the real-transform axis with entries 0..Nz/2, the last one stored
    as +Nz/2.
    """
    nx, ny, nz = dims(N)
    kx = np.rint(sfft.fftfreq(nx, 1.0 / nx)).astype(np.int64)
    ky = np.rint(sfft.fftfreq(ny, 1.0 / ny)).astype(np.int64)
    kz = np.rint(sfft.fftfreq(nz, 1.0 / nz)).astype(np.int64)[: nz // 2 + 1].copy()
    kz[-1] *= -1
    return np.array(np.meshgrid(kx, ky, kz, indexing="ij"), dtype=np.int64)


def dealias_mask(N, variant: int = 0) -> np.ndarray:
    """2/3-rule box mask on the half spectrum (Sec. 3.1, dealiasing paragraph).

    variant 0: keep modes with |k_i| < N_i/3 ("2/3 of the Nyquist mode") in each
    direction i, with that direction's point count.
    variant 1: the Appendix script's cut-off 2/3*(N_i/2+1), also strict.
    """
    K = wavenumbers(N)
    keep = np.ones(K.shape[1:], dtype=bool)
    for d, n in enumerate(dims(N)):
        kmax = n / 3.0 if variant == 0 else 2.0 / 3.0 * (n // 2 + 1)
        keep &= np.abs(K[d]) < kmax
    return keep


@dataclass
class Grid:
    """Precomputed K, |K|^2, K/|K|^2 and the dealias mask (Sec. 3.1).

    With box lengths (Lx, Ly, Lz) the wavenumber of index l along x is 2*pi*l/Lx
    (Sec. 2 footnote; Sec. 3.1: other box sizes by scaling); the 2/3 mask stays on
    the integer indices. N is one point count or three (Nx, Ny, Nz).
    """

    N: int | tuple
    variant: int = 0
    lengths: tuple | None = None

    def __post_init__(self):
        self.K = wavenumbers(self.N)
        if self.lengths is not None:
            scale = np.array([2.0 * np.pi / float(v) for v in self.lengths]).reshape(3, 1, 1, 1)
            self.K = self.K * scale
        self.K2 = np.sum(self.K * self.K, axis=0)
        # K/|K|^2 with the k=0 entry set to 0 (Sec. 3.1: where(K2 == 0, 1, K2)).
        self.K_over_K2 = self.K.astype(np.float64) / np.where(self.K2 == 0, 1, self.K2).astype(np.float64)
        self.mask = dealias_mask(self.N, self.variant)


# --------------------------------------------------------------------------
# Transforms (Eqs. ffteq/iffteq, fft/ifft; Sec. 3.1 fftn_mpi/ifftn_mpi serial form)
# --------------------------------------------------------------------------

def forward(u: np.ndarray) -> np.ndarray:
    """F: unnormalised real-to-complex 3D DFT with e^{-ik.x} over the last 3 axes.

    The real transform is taken along z (last axis), then complex ones along
    y and x (Eq. fft). Output shape (..., Nx, Ny, Nz/2+1).
    """
    return sfft.rfftn(np.asarray(u, dtype=np.float64), axes=(-3, -2, -1), workers=WORKERS)


def inverse(uh: np.ndarray) -> np.ndarray:
    """F^{-1}: complex-to-real 3D inverse DFT including the 1/(Nx Ny Nz) factor (Eq. ifft).

    Complex inverse transforms along x and y, then the real one along z; the
    z step uses only the real parts of the kz=0 and kz=Nz/2 coefficients.
    """
    return sfft.irfftn(np.asarray(uh, dtype=np.complex128), s=shape_of(uh), axes=(-3, -2, -1), workers=WORKERS)


def zero_nyquist(uh: np.ndarray) -> np.ndarray:
    """Zero every mode with |kx| = Nx/2, |ky| = Ny/2 or kz = Nz/2 (Sec. 3.3 drops these)."""
    nx, ny, nz = shape_of(uh)
    uh = uh.copy()
    uh[..., nx // 2, :, :] = 0.0
    uh[..., :, ny // 2, :] = 0.0
    uh[..., :, :, nz // 2] = 0.0
    return uh


def to_spectral(u: np.ndarray) -> np.ndarray:
    """State from a physical velocity (3,Nx,Ny,Nz): F of each component, Nyquist zeroed."""
    return zero_nyquist(forward(u))


# --------------------------------------------------------------------------
# Right-hand side (Eq. curl_convection, Eq. NSfinal, computeRHS of Sec. 3.1)
# --------------------------------------------------------------------------

def curl_hat(uh: np.ndarray, g: Grid) -> np.ndarray:
    """omega_hat = i k x u_hat (the curl in spectral space, Sec. 3.1)."""
    K = g.K
    w = np.empty_like(uh)
    w[0] = 1j * (K[1] * uh[2] - K[2] * uh[1])
    w[1] = 1j * (K[2] * uh[0] - K[0] * uh[2])
    w[2] = 1j * (K[0] * uh[1] - K[1] * uh[0])
    return w


def cross(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Pointwise c = a x b over the first axis (Eq. curl_convection)."""
    c = np.empty_like(a)
    c[0] = a[1] * b[2] - a[2] * b[1]
    c[1] = a[2] * b[0] - a[0] * b[2]
    c[2] = a[0] * b[1] - a[1] * b[0]
    return c


def nonlinear_hat(uh: np.ndarray, g: Grid, u_phys: np.ndarray | None = None) -> np.ndarray:
    """Dealiased N_hat = mask * F(u x omega) with u = F^{-1}(u_hat), omega = F^{-1}(ik x u_hat).

    Eq. curl_convection plus the 2/3-rule mask. ``u_phys`` lets the caller
    supply u in physical space (the Appendix reuses it at RK stage 0).
    """
    u = inverse(uh) if u_phys is None else u_phys
    w = inverse(curl_hat(uh, g))
    return forward(cross(u, w)) * g.mask


def project(nh: np.ndarray, g: Grid) -> np.ndarray:
    """N_hat - k (k . N_hat)/|k|^2, with K/|K|^2 = 0 at k = 0 (Eq. NSfinal, pressure of Eq. mod_pressure)."""
    p = np.sum(nh * g.K_over_K2, axis=0)
    return nh - p * g.K


def rhs(uh: np.ndarray, g: Grid, nu: float, u_phys: np.ndarray | None = None) -> np.ndarray:
    """du_hat/dt = P(mask*F(u x omega)) - nu |k|^2 u_hat (Eq. NSfinal; computeRHS of Sec. 3.1)."""
    return project(nonlinear_hat(uh, g, u_phys), g) - nu * g.K2 * uh


def rk4_step(uh: np.ndarray, g: Grid, nu: float, dt: float, u_phys: np.ndarray | None = None) -> np.ndarray:
    """One classical RK4 step exactly as the Appendix driver orders it.

    u0 = u1 = u; for s = 0..3: dU = RHS(u); if s < 3: u = u0 + b_s dt dU;
    u1 += a_s dt dU; the new state is u1. If ``u_phys`` is given it is used as
    the physical velocity at stage 0 (the Appendix keeps U in sync).
    """
    u0 = uh.copy()
    u1 = uh.copy()
    cur = uh
    for s in range(4):
        dU = rhs(cur, g, nu, u_phys if s == 0 else None)
        if s < 3:
            cur = u0 + RK4_B[s] * dt * dU
        u1 = u1 + RK4_A[s] * dt * dU
    return u1


def euler_step(uh: np.ndarray, g: Grid, nu: float, dt: float) -> np.ndarray:
    """Forward Euler step u += dt * RHS(u) (the integrator loop of Sec. 3.1)."""
    return uh + dt * rhs(uh, g, nu)


def rk_step(uh: np.ndarray, g: Grid, nu: float, dt: float, scheme: str = "rk4") -> np.ndarray:
    """One step of an explicit RK scheme of RK_SCHEMES, stage by stage as the
    Appendix driver orders RK4: dU_s = RHS(stage state); stage s + 1 starts from
    u0 + b_s dt dU_s; the new state is u0 + sum_s a_s dt dU_s."""
    a, b = RK_SCHEMES[scheme]
    u0 = uh.copy()
    u1 = uh.copy()
    cur = uh
    for s in range(len(a)):
        dU = rhs(cur, g, nu)
        if s < len(b):
            cur = u0 + b[s] * dt * dU
        u1 = u1 + a[s] * dt * dU
    return u1


def lsrk_step(uh: np.ndarray, g: Grid, nu: float, dt: float, A, B) -> np.ndarray:
    """One step of a low-storage scheme in Williamson's 2N form: for each stage j,
    dU <- A_j dU + dt RHS(u); u <- u + B_j dU (A_1 multiplies a zero register)."""
    u = uh.copy()
    dU = np.zeros_like(uh)
    for Aj, Bj in zip(A, B):
        dU = Aj * dU + dt * rhs(u, g, nu)
        u = u + Bj * dU
    return u


def run(uh: np.ndarray, N, nu: float, dt: float, nsteps: int, variant: int = 0,
        paper_reuse_u: bool = False, u0_phys: np.ndarray | None = None, scheme: str = "rk4",
        lengths=None) -> np.ndarray:
    """Advance ``nsteps`` steps (the step count is round(T/dt), reading of the while loop)
    of the Appendix's RK4, or of another scheme of RK_SCHEMES or LSRK_SCHEMES.

    paper_reuse_u=True mimics the Appendix: the physical U used at stage 0 is
    the one computed at the end of the previous step (the initial physical
    field ``u0_phys`` at step one) instead of F^{-1}(u_hat); RK4 only. ``lengths``:
    box lengths (Lx, Ly, Lz), default 2 pi each.
    """
    g = Grid(N, variant, lengths)
    if scheme in LSRK_SCHEMES:
        if paper_reuse_u:
            raise ValueError("paper_reuse_u applies to the Appendix RK4 driver only")
        A, B = LSRK_SCHEMES[scheme]
        for _ in range(nsteps):
            uh = lsrk_step(uh, g, nu, dt, A, B)
        return uh
    if scheme != "rk4":
        if paper_reuse_u:
            raise ValueError("paper_reuse_u applies to the Appendix RK4 driver only")
        for _ in range(nsteps):
            uh = rk_step(uh, g, nu, dt, scheme)
        return uh
    u_phys = u0_phys if paper_reuse_u else None
    for _ in range(nsteps):
        uh = rk4_step(uh, g, nu, dt, u_phys)
        if paper_reuse_u:
            u_phys = inverse(uh)
    return uh


# --------------------------------------------------------------------------
# Diagnostics (Appendix energy; workshop quantities of Sec. 4 "Verification")
# --------------------------------------------------------------------------

def energy(uh: np.ndarray) -> float:
    """E = 1/2 * sum(U*U) / (Nx Ny Nz) on the physical mesh (the Appendix's final reduce)."""
    u = inverse(uh)
    return float(0.5 * np.sum(u * u) / float(np.prod(shape_of(uh))))


def diagnostics(uh: np.ndarray, nu: float, lengths=None) -> dict:
    """Energy, dissipation, max|div u|, helicity and enstrophy as grid means.

    E = 1/2 <|u|^2>, eps = nu <|omega|^2> (the paper names "energy dissipation"
    without defining it; this is the standard form for periodic incompressible
    flow), H = <u . omega>, Z = 1/2 <|omega|^2>, div = max_x |F^{-1}(i k . u_hat)|.
    """
    n = shape_of(uh)
    g = Grid(n, 0, lengths)
    u = inverse(uh)
    w = inverse(curl_hat(uh, g))
    n3 = float(np.prod(n))
    div = inverse(1j * np.sum(g.K * uh, axis=0))
    return {
        "energy": float(0.5 * np.sum(u * u) / n3),
        "dissipation": float(nu * np.sum(w * w) / n3),
        "max_div": float(np.max(np.abs(div))),
        "helicity": float(np.sum(u * w) / n3),
        "enstrophy": float(0.5 * np.sum(w * w) / n3),
    }


def energy_spectrum(uh: np.ndarray) -> np.ndarray:
    """Shell-summed energy spectrum E(k), k = round(|k|) (for closure and decay checks).

    Uses the half-spectrum weight 1 at kz = 0 and kz = Nz/2 and 2 otherwise,
    so that sum(E(k)) equals the grid-mean energy.
    """
    n = shape_of(uh)
    K = wavenumbers(n)
    kmag = np.rint(np.sqrt(np.sum(K * K, axis=0).astype(np.float64))).astype(np.int64)
    w = np.full(K.shape[1:], 2.0)
    w[:, :, 0] = 1.0
    w[:, :, n[2] // 2] = 1.0
    e = 0.5 * w * np.sum(np.abs(uh) ** 2, axis=0) / float(np.prod(n)) ** 2
    return np.bincount(kmag.ravel(), weights=e.ravel())
