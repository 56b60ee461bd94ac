"""GPU test of dns_spectral_sums_noalloc, the entry point for callers that cannot allocate.

Callers whose device memory belongs to another allocator (or that must not take
cudaMalloc's synchronisation) get the diagnostics sums through this call
without any allocation. The test calls it through the C ABI on device buffers
the test itself owns, twice in a row on different fields, and checks each
result against dns_diagnostics (the handle-based path) on the same state and
against the FP64 oracle's grid-mean diagnostics of the same field. A third
check shows the documented scope: the sums take the wavenumber of index k as k
(the [0, 2 pi]^3 box), so for a handle whose box has other lengths the
dissipation differs from dns_diagnostics by the square of the length ratio.
It lives in a file of its own, collected last, and needs nothing from the
other test files.
"""

import ctypes

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import Solver, _lib, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# Both paths sum in FP64 over the same values; only the summation order differs.
REL_TOL = 1e-12
# The oracle sums the same field on the physical grid (Parseval), in FP64.
ORACLE_TOL = 1e-11


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()
    return _lib.lib()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_sums_match_diagnostics_on_two_calls(L, dtype):
    N, nu = 32, 0.017
    code = _lib.DNS_F32 if dtype == "f32" else _lib.DNS_F64
    cdt = torch.complex64 if dtype == "f32" else torch.complex128
    stream = torch.cuda.current_stream()
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    with Solver(N, nu, 0.01, dtype) as s:
        for call, seed in enumerate((3, 4)):
            uh = inputs.isotropic_spectral(N, seed=seed, k0=3.0 + call).to(cdt).cuda()
            s.set_state_spectral(uh)
            ref = s.diagnostics()
            state = torch.empty((3, N, N, N // 2 + 1), dtype=cdt, device="cuda")
            s.get_state_spectral(state)
            rc = L.dns_spectral_sums_noalloc(ctypes.c_void_p(state.data_ptr()), N, code, nu,
                                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
            assert rc == _lib.DNS_OK, _lib.last_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            orc = sn.diagnostics(state.cpu().numpy().astype(np.complex128), nu)
            for i, key in enumerate(("energy", "dissipation", "helicity", "enstrophy")):
                assert abs(got[i] - ref[key]) <= REL_TOL * max(abs(ref[key]), 1e-30), (call, key, got[i], ref[key])
                scale = max(abs(orc[key]), abs(orc["energy"]) if key == "helicity" else 0.0, 1e-30)
                assert abs(got[i] - orc[key]) <= ORACLE_TOL * scale, (call, key, got[i], orc[key])
            assert got[4] == 0.0


def test_noalloc_sums_take_the_2pi_box(L):
    """On a box of side pi (wavenumbers 2 k) the handle's dissipation is 4x the fixed-box sum."""
    N, nu = 16, 0.01
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    uh = inputs.isotropic_spectral(N, seed=8, k0=2.0).cuda()
    with Solver(N, nu, 0.01, "f64") as s:
        for key in ("Lx", "Ly", "Lz"):
            s.set_option(key, np.pi)
        s.set_state_spectral(uh)
        ref = s.diagnostics()
        rc = L.dns_spectral_sums_noalloc(ctypes.c_void_p(uh.data_ptr()), N, _lib.DNS_F64, nu,
                                         ctypes.c_void_p(out.data_ptr()), None)
        assert rc == _lib.DNS_OK, _lib.last_error()
        torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert abs(got[0] - ref["energy"]) <= REL_TOL * ref["energy"]
    assert abs(4.0 * got[1] - ref["dissipation"]) <= REL_TOL * ref["dissipation"]


def test_noalloc_rejects_oversize_and_bad_arguments(L):
    buf = torch.zeros(64, dtype=torch.complex128, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    p, o = ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(out.data_ptr())
    rc = L.dns_spectral_sums_noalloc(p, 4096, _lib.DNS_F64, 0.01, o, None)
    assert rc == _lib.DNS_ERR_ARG and "maximum" in _lib.last_error()
    assert L.dns_spectral_sums_noalloc(p, 31, _lib.DNS_F64, 0.01, o, None) == _lib.DNS_ERR_ARG
    assert L.dns_spectral_sums_noalloc(None, 32, _lib.DNS_F64, 0.01, o, None) == _lib.DNS_ERR_ARG
    assert L.dns_spectral_sums_noalloc(p, 32, 5, 0.01, o, None) == _lib.DNS_ERR_ARG
    assert np.all(out.cpu().numpy() == 0)  # nothing was launched
