"""Seeded synthetic initial conditions (shared by the GPU tests, the oracle tests and the bench).

This module holds no arithmetic of the solver itself (no transforms, no
right-hand side, no time stepping): it only builds velocity fields.

* Taylor-Green vortex, u = (sin x cos y cos z, -cos x sin y cos z, 0)
  (the initial condition of the Appendix script and of Sec. 4 "Verification"), on the
  mesh or as its exact Fourier coefficients.
* ABC (Arnold-Beltrami-Childress) flow with |k| = 1, for which omega = u.
* Decaying-isotropic random field in spectral form (Rogallo-style random
  phases): divergence-free, Hermitian in the kz = 0 plane, no Nyquist modes,
  all modes inside the 2/3 box, spectrum E(k) ~ k^4 exp(-2 (k/k0)^2),
  rescaled to a prescribed energy.

Layouts: physical fields are (3, N, N, N) with x slowest (Eq. realmesh);
spectral fields are (3, N, N, N/2+1) complex in the order [c][kx][ky][kz]
with kx, ky in FFT order (Sec. 3.1).
"""

from __future__ import annotations

import math

import numpy as np
import torch


def _axis(N: int, device=None, dtype=torch.float64) -> torch.Tensor:
    return torch.arange(N, device=device, dtype=dtype) * (2.0 * math.pi / N)


def taylor_green(N: int, dtype=np.float64) -> np.ndarray:
    """Taylor-Green velocity on the N^3 mesh as a numpy array (3, N, N, N)."""
    x = 2.0 * np.pi * np.arange(N) / N
    sx, cx = np.sin(x), np.cos(x)
    u = np.zeros((3, N, N, N), dtype=dtype)
    u[0] = (sx[:, None, None] * cx[None, :, None] * cx[None, None, :]).astype(dtype)
    u[1] = (-cx[:, None, None] * sx[None, :, None] * cx[None, None, :]).astype(dtype)
    return u


def taylor_green_spectral(N: int, device="cpu", dtype=torch.complex128) -> torch.Tensor:
    """Taylor-Green velocity in the half spectrum (3, N, N, N/2+1), paper order, written out
    exactly: sin x cos y cos z has the Fourier coefficient s_x / (8i) at k = (s_x, s_y, s_z),
    s_i = +-1, and -cos x sin y cos z the coefficient -s_y / (8i); the unnormalised forward
    transform multiplies them by N^3. Only kz = +1 is stored (kz = -1 is its conjugate) and
    every other mode is exactly zero."""
    uh = torch.zeros((3, N, N, N // 2 + 1), device=device, dtype=dtype)
    c = float(N) ** 3 / 8.0
    for sx in (1, -1):
        for sy in (1, -1):
            uh[0, sx % N, sy % N, 1] = -1j * c * sx
            uh[1, sx % N, sy % N, 1] = 1j * c * sy
    return uh


def taylor_green_torch(N: int, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """Taylor-Green velocity built directly in device memory (large grids)."""
    x = _axis(N, device=device, dtype=torch.float64)
    sx, cx = torch.sin(x).to(dtype), torch.cos(x).to(dtype)
    u = torch.zeros((3, N, N, N), device=device, dtype=dtype)
    u[0] = sx[:, None, None] * cx[None, :, None] * cx[None, None, :]
    u[1] = -cx[:, None, None] * sx[None, :, None] * cx[None, None, :]
    return u


def abc_flow(N, A: float = 1.0, B: float = 1.0, C: float = 1.0, dtype=np.float64) -> np.ndarray:
    """ABC flow u = (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x); curl u = u.
    N: one point count or three (Nx, Ny, Nz)."""
    n = _dims(N)
    X, Y, Z = np.meshgrid(*(2.0 * np.pi * np.arange(v) / v for v in n), indexing="ij")
    u = np.empty((3,) + n, dtype=dtype)
    u[0] = A * np.sin(Z) + C * np.cos(Y)
    u[1] = B * np.sin(X) + A * np.cos(Z)
    u[2] = C * np.sin(Y) + B * np.cos(X)
    return u


def _dims(N) -> tuple:
    return (int(N),) * 3 if np.ndim(N) == 0 else tuple(int(v) for v in N)


def _freq(n: int, device, dtype):
    k = torch.arange(n, device=device)
    return torch.where(k < n // 2, k, k - n).to(dtype)


def isotropic_spectral(N, seed: int = 0, k0: float = 4.0, energy: float = 1.0,
                       device="cpu", dtype=torch.complex128) -> torch.Tensor:
    """Random divergence-free field in the half spectrum (3, Nx, Ny, Nz/2+1), paper order.

    N is one point count or three (Nx, Ny, Nz). Each mode with 0 < |k| and
    |k_i| < N_i/3 gets amplitude sqrt(E(|k|)/(4 pi |k|^2)), E(k) = k^4 exp(-2 (k/k0)^2),
    along a random direction perpendicular to k, with uniform random phases (Rogallo
    1981 style). The kz = 0 plane is made Hermitian by averaging each mode with the
    conjugate of its mirror, Nyquist modes are zero, and the field is scaled so that
    1/2 (Nx Ny Nz)^-2 sum_k w_k |u_hat_k|^2 = ``energy`` (w = 1 at kz = 0, else 2).
    Random numbers come from a seeded torch generator on ``device``.
    """
    nx, ny, nz = _dims(N)
    h = nz // 2 + 1
    rdt = torch.float64 if dtype == torch.complex128 else torch.float32
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    KX = _freq(nx, device, rdt)[:, None, None].expand(nx, ny, h)
    KY = _freq(ny, device, rdt)[None, :, None].expand(nx, ny, h)
    KZ = torch.arange(h, device=device).to(rdt)[None, None, :].expand(nx, ny, h)
    kk = torch.sqrt(KX * KX + KY * KY + KZ * KZ)
    inside = (KX.abs() < nx / 3.0) & (KY.abs() < ny / 3.0) & (KZ < nz / 3.0) & (kk > 0)
    kk_safe = torch.where(kk > 0, kk, torch.ones_like(kk))
    spec = kk_safe ** 4 * torch.exp(-2.0 * (kk_safe / k0) ** 2)
    amp = torch.sqrt(spec / (4.0 * math.pi * kk_safe ** 2)) * inside

    # Two unit vectors spanning the plane perpendicular to k.
    # e1 = k x a / |k x a| with a = z-hat unless k is parallel to z (then a = x-hat).
    par = (KX == 0) & (KY == 0)
    ax = torch.where(par, torch.ones_like(KX), torch.zeros_like(KX))
    az = torch.where(par, torch.zeros_like(KX), torch.ones_like(KX))
    e1x = KY * az
    e1y = KZ * ax - KX * az
    e1z = -KY * ax
    n1 = torch.sqrt(e1x ** 2 + e1y ** 2 + e1z ** 2)
    n1 = torch.where(n1 > 0, n1, torch.ones_like(n1))
    e1x, e1y, e1z = e1x / n1, e1y / n1, e1z / n1
    e2x = (KY * e1z - KZ * e1y) / kk_safe
    e2y = (KZ * e1x - KX * e1z) / kk_safe
    e2z = (KX * e1y - KY * e1x) / kk_safe

    shape = (nx, ny, h)
    th1 = torch.rand(shape, generator=gen, device=device, dtype=rdt) * (2.0 * math.pi)
    th2 = torch.rand(shape, generator=gen, device=device, dtype=rdt) * (2.0 * math.pi)
    phi = torch.rand(shape, generator=gen, device=device, dtype=rdt) * (2.0 * math.pi)
    a1 = amp * torch.cos(phi) * torch.exp(1j * th1)
    a2 = amp * torch.sin(phi) * torch.exp(1j * th2)
    uh = torch.stack([a1 * e1x + a2 * e2x, a1 * e1y + a2 * e2y, a1 * e1z + a2 * e2z]).to(dtype)

    # Hermitian kz = 0 plane: u(-kx,-ky,0) = conj(u(kx,ky,0)).
    ix = (-torch.arange(nx, device=device)) % nx
    iy = (-torch.arange(ny, device=device)) % ny
    p0 = uh[:, :, :, 0]
    mirror = p0[:, ix][:, :, iy]
    uh[:, :, :, 0] = 0.5 * (p0 + mirror.conj())
    uh[:, nx // 2, :, :] = 0
    uh[:, :, ny // 2, :] = 0
    uh[:, :, :, nz // 2] = 0
    uh[:, 0, 0, 0] = 0

    w = torch.full((h,), 2.0, device=device, dtype=rdt)
    w[0] = 1.0
    w[nz // 2] = 1.0
    e = 0.5 * torch.sum(w * torch.sum(uh.real ** 2 + uh.imag ** 2, dim=0)) / (float(nx) * ny * nz) ** 2
    uh *= math.sqrt(energy / float(e))
    return uh


def random_field_in_mask(N: int, seed: int = 0, device="cpu") -> torch.Tensor:
    """Isotropic field with k0 = N/8 (all energy well inside the 2/3 box), FP64 spectral."""
    return isotropic_spectral(N, seed=seed, k0=max(1.0, N / 8.0), energy=0.5, device=device)
