"""GPU tests of the plane-pass schedule (option "fused_planes" = 1, N >= 256): each RK stage as the
z-pass plus one persistent launch that walks the kz planes doing the y-forward, x-stage and
y-inverse of each plane (they are local to a plane; Eq. NSfinal's transforms in the order of
Sec. 3.2 with the transposes replaced by changes of pass direction).

The plane pass runs the same per-column and per-line arithmetic as the four-pass schedule, so
after the same steps from the same state the two states agree to the last bit (checked), and
both agree with the FP64 oracle (FP64 1e-12, FP32 1e-5 relative L2). The bounded waits are exercised by
a debug hook whose waits cannot be met: they give up after 1 s, the host reads
DNS_ERR_TIMEOUT, and the handle keeps working.
"""

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import Solver, _lib, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()


@pytest.fixture(autouse=True)
def _release_cached_memory():
    yield
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _run(N, dtype, fused, uh, steps, **opts):
    with Solver(N, 0.004, 2e-3, dtype, **opts) as s:
        s.set_option("fused_planes", fused)
        assert s.get_option("fused_planes") == fused
        s.set_state_spectral(uh)
        s.step(steps)
        return s.get_state_spectral(), s.diagnostics()


@pytest.mark.parametrize("N,dtype,steps", [(256, "f32", 3), (256, "f64", 3), (512, "f32", 2), (512, "f64", 1),
                                           (1024, "f32", 1)])
def test_plane_pass_equals_four_pass(N, dtype, steps):
    cdt = torch.complex64 if dtype == "f32" else torch.complex128
    uh = inputs.isotropic_spectral(N, seed=50 + N, k0=N / 8.0, device="cuda").to(cdt)
    a, da = _run(N, dtype, 1, uh, steps)
    b, db = _run(N, dtype, 0, uh, steps)
    diff = float(np.abs(a - b).max() / np.abs(b).max())
    assert diff == 0.0, f"plane pass differs from the four-pass schedule by {diff:.3e} (relative max)"
    assert da["energy"] == db["energy"]


_ORACLE = {}


def _oracle_256(variant, integrator, nu, dt):
    """(initial state, FP64 oracle after one step) at 256^3, computed once per scheme."""
    key = (variant, integrator)
    if key not in _ORACLE:
        uh = inputs.isotropic_spectral(256, seed=7, k0=12.0).numpy()
        _ORACLE[key] = (uh, sn.run(uh, 256, nu, dt, 1, variant=variant, scheme=integrator))
    return _ORACLE[key]


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("variant,integrator", [(0, "rk4"), (1, "rk4"), (0, "euler"), (0, "heun"), (0, "williamson3")])
def test_plane_pass_matches_oracle_at_256(dtype, tol, variant, integrator):
    N, nu, dt = 256, 0.004, 2e-3
    uh, ref = _oracle_256(variant, integrator, nu, dt)
    with Solver(N, nu, dt, dtype, dealias_variant=variant, integrator=integrator) as s:
        assert s.get_option("fused_planes") == 0  # the default
        s.set_option("fused_planes", 1)
        s.set_state_spectral(uh.astype(np.complex64) if dtype == "f32" else uh)
        s.step(1)
        got = s.get_state_spectral()
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert err < tol, err


def test_bounded_waits_give_up_and_the_handle_recovers():
    N = 256
    uh = inputs.isotropic_spectral(N, seed=3, k0=20.0, device="cuda").to(torch.complex64)
    with Solver(N, 0.004, 2e-3, "f32") as s:
        s.set_option("fused_planes", 1)
        s.set_state_spectral(uh)
        s.step(1)
        before = s.get_state_spectral()
        rc = s.plane_wait_timeout_test()
        assert rc == _lib.DNS_ERR_TIMEOUT, (rc, _lib.last_error())
        assert "gave up" in _lib.last_error()
        # the state is untouched and the next steps are those of a fresh run from it
        np.testing.assert_array_equal(s.get_state_spectral(), before)
        s.step(2)
        got = s.get_state_spectral()
        d = s.diagnostics()
    with Solver(N, 0.004, 2e-3, "f32") as r:
        r.set_option("fused_planes", 1)
        r.set_state_spectral(before)
        r.step(2)
        ref = r.get_state_spectral()
    np.testing.assert_array_equal(got, ref)
    assert np.isfinite(d["energy"])


def test_tuner_times_the_plane_schedule_and_keeps_the_state():
    N = 256
    uh = inputs.isotropic_spectral(N, seed=77, k0=N / 8.0, device="cuda").to(torch.complex64)
    with Solver(N, 0.004, 2e-3, "f32") as s:
        s.set_state_spectral(uh)
        assert s.tune_tiles(1) == (0, 0, 0)  # no widths or plans at this size: the schedule only
        fused = int(s.get_option("fused_planes"))
        assert fused in (0, 1)
        assert torch.equal(s.get_state_spectral(torch.empty_like(uh)), uh) and s.diagnostics()["t"] == 0.0
        s.step(2)
        got = s.get_state_spectral(torch.empty_like(uh))
    ref, _ = _run(N, "f32", 1 - fused, uh, 2)  # the two schedules agree to the last bit
    assert np.array_equal(got.cpu().numpy(), ref)
