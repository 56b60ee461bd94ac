"""GPU test of dns_spectral_sums_noalloc, the entry point for callers that cannot allocate.

Callers whose device memory belongs to another allocator (or that must not take
cudaMalloc's synchronisation) get the diagnostics sums through this call
without any allocation. The test calls it through the C ABI on device buffers
the test itself owns, twice in a row on different fields, and checks each
result against dns_diagnostics (the handle-based path) on the same state.
It lives in a file of its own, collected last, and needs nothing from the
other test files.
"""

import ctypes

import numpy as np
import pytest

from paper_1602_03638_gb300 import Solver, _lib, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# Both paths sum in FP64 over the same values; only the summation order differs.
REL_TOL = 1e-12


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
            for i, key in enumerate(("energy", "dissipation", "helicity", "enstrophy")):
                assert abs(got[i] - ref[key]) <= REL_TOL * max(abs(ref[key]), 1e-30), (call, key, got[i], ref[key])
            assert got[4] == 0.0


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
