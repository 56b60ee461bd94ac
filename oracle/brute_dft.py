"""Brute-force triple-sum DFT (TEST INFRASTRUCTURE).

Writes out the definition of the discrete Fourier pair of Sec. 2
(Eqs. ffteq/iffteq) as explicit sums over the physical mesh of Eq. realmesh
and the wavenumbers of Eq. kmesh, with no FFT factorisation. O(N^6): only for
the tiny grids (6^3, 8^3, 12^3, and a few with other point counts per direction)
that pin the oracle's library transforms.
"""

from __future__ import annotations

import numpy as np


def _k_axis(N: int) -> np.ndarray:
    """Wavenumbers in FFT storage order 0..N/2-1, -N/2..-1, built by a plain loop."""
    return np.array([j if j < N // 2 else j - N for j in range(N)], dtype=np.float64)


def forward_r2c(u: np.ndarray) -> np.ndarray:
    """u_hat(kx, ky, kz) = sum_x u(x) exp(-i k.x), kz = 0..Nz/2 (Eq. iffteq, forward direction).

    u has shape (Nx, Ny, Nz); the point counts may differ per direction (Sec. 2 footnote).
    """
    nx, ny, nz = u.shape
    X, Y, Z = np.meshgrid(*(2.0 * np.pi * np.arange(n) / n for n in (nx, ny, nz)), indexing="ij")
    kx, ky = _k_axis(nx), _k_axis(ny)
    kz = np.arange(nz // 2 + 1, dtype=np.float64)
    out = np.zeros((nx, ny, nz // 2 + 1), dtype=np.complex128)
    for a in range(nx):
        for b in range(ny):
            for c in range(nz // 2 + 1):
                out[a, b, c] = np.sum(u * np.exp(-1j * (kx[a] * X + ky[b] * Y + kz[c] * Z)))
    return out


def inverse_c2r(uh: np.ndarray) -> np.ndarray:
    """u(x) = (Nx Ny Nz)^-1 sum over the full spectrum of u_hat(k) exp(+i k.x) (Eq. ffteq).

    uh has shape (Nx, Ny, Nz/2+1). The half spectrum is extended to all kz by
    Hermitian symmetry u_hat(-k) = conj(u_hat(k)) applied to kz = 1..Nz/2-1; the
    kz = 0 and kz = Nz/2 planes enter once each, through their real part only along
    z, which is what a real-valued result requires.
    """
    nx, ny, h = uh.shape
    nz = 2 * (h - 1)
    X, Y, Z = np.meshgrid(*(2.0 * np.pi * np.arange(n) / n for n in (nx, ny, nz)), indexing="ij")
    kx, ky = _k_axis(nx), _k_axis(ny)
    u = np.zeros((nx, ny, nz), dtype=np.float64)
    for a in range(nx):
        for b in range(ny):
            phxy = kx[a] * X + ky[b] * Y
            for c in range(h):
                if c == 0 or c == nz // 2:
                    u += _xy_then_real_z(uh[a, b, c], phxy, c * Z)
                else:
                    u += 2.0 * np.real(uh[a, b, c] * np.exp(1j * (phxy + c * Z)))
    return u / (float(nx) * float(ny) * float(nz))


def _xy_then_real_z(coef: complex, phxy: np.ndarray, phz: np.ndarray) -> np.ndarray:
    """Term of a kz = 0 or kz = N/2 coefficient in the order x, y complex then z real.

    After the complex inverse sums along x and y the coefficient becomes
    g = coef * exp(i(kx x + ky y)); the real z-transform then uses Re(g) times
    cos(kz z) (sin(kz z) vanishes on the mesh at kz = 0 and kz = N/2).
    """
    g = coef * np.exp(1j * phxy)
    return np.real(g) * np.cos(phz)
