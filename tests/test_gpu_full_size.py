"""Full-spectrum checks of the right-hand side at the bench sizes, where the z-pass
kernels are size-specific (N = 256: full-warp lines; 512: the pipelined half-warp
kernel; 1024: the pipelined canonical kernel).

256^3 and 512^3 compare every mode with the FP64 oracle (a random physical field
with energy in all modes, the oracle run in full on the host cores). At 1024^3
the oracle is too large for a test. There, first, a dense random divergence-free
field band-limited to |k_i| <= 85 is compared mode by mode with the oracle at
512^3: its products reach |k_i| <= 170, which neither grid aliases (170 < 256)
nor masks (3 * 170 < 512), so the right-hand side is the same trigonometric
polynomial on both grids and its unnormalised coefficients differ by the factor
(1024/512)^3 = 8. Second, the right-hand side of a random divergence-free field
filling the 2/3 box is checked against what holds at any
size (Eq. NSfinal, Sec. 2): the projected, dealiased nonlinear term transfers no
energy and no helicity (u.(u x w) = w.(u x w) = 0 pointwise, and the mask and the
projection are the identity on the state), it is divergence-free, and the
viscous part is exactly -nu |k|^2 u_hat.
"""

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import Solver, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()


@pytest.mark.parametrize("N,dtype,tol", [(256, "f64", 1e-12), (256, "f32", 2e-5), (512, "f32", 2e-5),
                                         (512, "f64", 1e-12)])
def test_rhs_of_random_full_spectrum_field_matches_oracle(N, dtype, tol):
    rng = np.random.default_rng(4000 + N)
    u = rng.standard_normal((3, N, N, N)).astype(np.float32 if dtype == "f32" else np.float64)
    nu = 0.004
    with Solver(N, nu, 1e-3, dtype) as s:
        s.set_state(u)
        got = s.rhs()
    ref = sn.rhs(sn.to_spectral(u.astype(np.float64)), sn.Grid(N), nu)
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    assert err < tol, err


def _kvecs(N, dev):
    k = torch.fft.fftfreq(N, 1.0 / N, device=dev, dtype=torch.float64)
    kz = torch.arange(N // 2 + 1, device=dev, dtype=torch.float64)
    return k, kz


def _slabs(N, step=64):
    for a in range(0, N, step):
        yield slice(a, min(N, a + step))


@pytest.fixture(autouse=True)
def _release_cached_memory():
    yield
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _embed(src, N, dev, dtype):
    """Half spectrum (3, n, n, n/2+1) of |k_i| <= kb modes placed into an N grid (N > 2 n)."""
    n = src.shape[1]
    out = torch.zeros((3, N, N, N // 2 + 1), dtype=dtype, device=dev)
    lo, hi = n // 2, n - n // 2  # indices 0..lo-1 are k >= 0, lo..n-1 are k < 0
    s = src.to(device=dev, dtype=dtype)
    kz = min(n // 2 + 1, N // 2 + 1)
    for a_src, a_dst in ((slice(0, lo), slice(0, lo)), (slice(lo, n), slice(N - hi, N))):
        for b_src, b_dst in ((slice(0, lo), slice(0, lo)), (slice(lo, n), slice(N - hi, N))):
            out[:, a_dst, b_dst, :kz] = s[:, a_src, b_src, :kz]
    return out


@pytest.fixture(scope="module")
def band_limited_case():
    """A dense divergence-free field with |k_i| <= 85 (the 2/3 box of a 256 grid) and the FP64
    oracle's right-hand side of it on the 512 grid (nu = 0.004)."""
    nu = 0.004
    u256 = inputs.isotropic_spectral(256, seed=31, k0=256 / 5.0, energy=1.0)
    u512 = _embed(u256, 512, "cpu", torch.complex128) * 8.0
    ref = sn.rhs(u512.numpy(), sn.Grid(512), nu)
    return u256, torch.from_numpy(ref), nu


@pytest.mark.parametrize("dtype,tol", [("f32", 3e-5), ("f64", 1e-12)])
def test_rhs_of_band_limited_field_at_1024_matches_oracle_at_512(band_limited_case, dtype, tol):
    u256, ref512, nu = band_limited_case
    N, dev = 1024, "cuda"
    cdt = torch.complex64 if dtype == "f32" else torch.complex128
    uh = _embed(u256, N, dev, cdt) * 64.0
    out = torch.empty_like(uh)
    with Solver(N, nu, 1e-3, dtype) as s:
        s.set_state_spectral(uh)
        del uh
        s.rhs(out)
    torch.cuda.synchronize()
    expect = _embed(ref512, N, dev, torch.complex128)  # modes |k_i| <= 255, zero beyond
    scale = 8.0 * float(ref512.abs().max())
    err = 0.0
    for sl in _slabs(N):
        e = (out[:, sl].to(torch.complex128) - 8.0 * expect[:, sl]).abs().max()
        err = max(err, float(e) / scale)
    assert err < tol, err


def test_rhs_invariants_at_1024():
    N, dev = 1024, "cuda"
    uh = inputs.isotropic_spectral(N, seed=17, k0=N / 5.0, energy=1.0, device=dev).to(torch.complex64)
    rhs0 = torch.empty_like(uh)
    rhs1 = torch.empty_like(uh)
    nu = 0.01
    for visc, out in ((0.0, rhs0), (nu, rhs1)):
        with Solver(N, visc, 1e-3, "f32") as s:
            s.set_state_spectral(uh)
            s.rhs(out)
        torch.cuda.synchronize()
    k, kz = _kvecs(N, dev)
    w = torch.where(kz == 0, 1.0, 2.0).to(torch.float64)[None, None, :]
    e_tr = h_tr = e_sc = h_sc = 0.0
    div_max = div_sc = visc_max = nl_max = visc_sc = 0.0
    for sl in _slabs(N):  # slabs of kx, everything in FP64
        kx, ky, kzz = k[sl][:, None, None], k[None, :, None], kz[None, None, :]
        u = [uh[c, sl].to(torch.complex128) for c in range(3)]
        r0 = [rhs0[c, sl].to(torch.complex128) for c in range(3)]
        om = [1j * (ky * u[2] - kzz * u[1]), 1j * (kzz * u[0] - kx * u[2]), 1j * (kx * u[1] - ky * u[0])]
        e_tr += sum(float((w * (u[c].conj() * r0[c]).real).sum()) for c in range(3))
        h_tr += sum(float((w * (om[c].conj() * r0[c]).real).sum()) for c in range(3))
        e_sc += sum(float((w * u[c].abs() * r0[c].abs()).sum()) for c in range(3))
        h_sc += sum(float((w * om[c].abs() * r0[c].abs()).sum()) for c in range(3))
        kmag = torch.sqrt(kx ** 2 + ky ** 2 + kzz ** 2)
        div_max = max(div_max, float((kx * r0[0] + ky * r0[1] + kzz * r0[2]).abs().max()))
        div_sc = max(div_sc, float((kmag * torch.stack([r.abs() for r in r0]).max(dim=0).values).max()))
        k2 = kmag ** 2
        for c in range(3):
            d = rhs1[c, sl].to(torch.complex128) - r0[c] + nu * k2 * u[c]
            visc_max = max(visc_max, float(d.abs().max()))
            visc_sc = max(visc_sc, float((nu * k2 * u[c].abs()).max()))
            nl_max = max(nl_max, float(r0[c].abs().max()))
    # no energy or helicity transfer, divergence-free
    assert abs(e_tr) < 1e-5 * e_sc
    assert abs(h_tr) < 1e-5 * h_sc
    assert div_max < 1e-5 * div_sc
    # the nonlinear term is not trivially small next to the viscous one
    assert nl_max > 1e-3 * visc_sc
    # both right-hand sides round the same nonlinear term in FP32: the difference is
    # -nu |k|^2 u_hat up to one rounding of each
    assert visc_max < 1e-5 * (nl_max + visc_sc)
