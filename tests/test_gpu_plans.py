"""GPU tests of the radix plan variants of the small grids (option "fft_plan"; the
ensemble row's tuned radix schedule).

The option is a bit mask over the passes of a stage (x, y-inverse, z, y-forward); a set
bit runs that pass's line transforms (per-member and batched kernels) with radix 3 first
and radix-4 passes instead of the default radix-8/16 schedule. The transforms are the same
DFTs, so the bounds against the FP64 oracle are those of the default plan (FP64 1e-12, FP32
1e-5 relative L2 after 20 RK4 steps); the plans differ by rounding (not bit for bit) wherever
their radix sequences differ (N >= 12). Ensemble members on other plans equal standalone
runs on the same plans bit for bit, batched or not.
"""

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import Ensemble, Solver, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CPLX = {"f32": np.complex64, "f64": np.complex128}
SIZES = [8, 12, 16, 24, 32, 48, 64, 96, 128]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _iso(N, seed, dtype):
    return inputs.isotropic_spectral(N, seed=seed, k0=max(2.0, N / 8.0)).numpy().astype(CPLX[dtype])


def _run(N, dtype, uh, plan, steps=20, nu=0.01, dt=0.004, graph=1):
    with Solver(N, nu, dt, dtype) as s:
        s.set_option("fft_plan", plan)
        s.set_option("use_graph", graph)
        s.set_state_spectral(uh)
        s.step(steps)
        return s.get_state_spectral()


@pytest.mark.parametrize("dtype,bound", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("N", SIZES)
def test_alternative_plans_match_oracle(N, dtype, bound):
    uh = _iso(N, 100 + N, dtype)
    ref = sn.run(uh.astype(np.complex128), N, 0.01, 0.004, 20)
    for mask in (15, 5, 10):  # every pass; x and z; the two y-passes
        assert rel_l2(_run(N, dtype, uh, mask), ref) <= bound, f"plan mask {mask}"


@pytest.mark.parametrize("N", [12, 32, 96])
def test_each_pass_bit_changes_the_rounding_only(N):
    uh = _iso(N, 7, "f64")
    a = _run(N, "f64", uh, 0)
    for bit in range(4):
        b = _run(N, "f64", uh, 1 << bit)
        assert not np.array_equal(a, b), f"bit {bit}"
        assert rel_l2(a, b) < 1e-13


def test_rhs_follows_the_plan():
    N = 48
    uh = _iso(N, 9, "f64")
    ref = sn.rhs(uh, sn.Grid(N), 0.01)
    for plan in (0, 15):
        with Solver(N, 0.01, 0.004, "f64") as s:
            s.set_option("fft_plan", plan)
            s.set_state_spectral(uh)
            assert rel_l2(s.rhs(), ref) <= 1e-12


def test_graph_and_eager_agree_bitwise_on_alternative_plans():
    uh = _iso(64, 3, "f32")
    assert np.array_equal(_run(64, "f32", uh, 15, steps=4, graph=1), _run(64, "f32", uh, 15, steps=4, graph=0))


def test_plan_option_is_validated():
    with Solver(32, 0.01, 0.004, "f32") as s:
        s.set_option("fft_plan", 9)
        assert s.get_option("fft_plan") == 9
        for bad in (16, -1, 0.5):
            with pytest.raises(RuntimeError):
                s.set_option("fft_plan", bad)
    with Solver(256, 0.01, 0.004, "f32") as s:  # the default plan only above the ensemble sizes
        s.set_option("fft_plan", 0)
        with pytest.raises(RuntimeError):
            s.set_option("fft_plan", 1)
    with Solver((32, 16, 24), 0.01, 0.004, "f32") as s:
        with pytest.raises(RuntimeError):
            s.set_option("fft_plan", 1)


def test_tuner_picks_a_plan_and_keeps_the_state():
    N, dtype = 48, "f32"
    uh = _iso(N, 5, dtype)
    with Solver(N, 0.01, 0.004, dtype) as s:
        s.set_state_spectral(uh)
        s.tune_tiles(3)
        plan = int(s.get_option("fft_plan"))
        assert 0 <= plan < 16
        assert s.diagnostics()["t"] == 0.0
        assert np.array_equal(s.get_state_spectral(), uh)
        s.step(6)
        got = s.get_state_spectral()
        tiles = [s.get_option(k) for k in ("y_tile_inverse", "y_tile_forward", "z_tile")]
    with Solver(N, 0.01, 0.004, dtype) as s:
        s.set_option("fft_plan", plan)
        for k, v in zip(("y_tile_inverse", "y_tile_forward", "z_tile"), tiles):
            s.set_option(k, v)
        s.set_state_spectral(uh)
        s.step(6)
        assert np.array_equal(s.get_state_spectral(), got)


@pytest.mark.parametrize("batching", [0, 1 << 30])
def test_ensemble_members_on_other_plans_equal_solo_runs(batching):
    Ns = [32, 32, 48, 32, 48, 96]
    plans = [15, 0, 6, 15, 6, 9]
    dtype, nu, dt = "f32", 0.01, 0.004
    ics = [_iso(N, 60 + i, dtype) for i, N in enumerate(Ns)]
    with Ensemble(Ns, [nu] * len(Ns), [dt] * len(Ns), dtype) as ens:
        ens.set_batching(batching)
        for m, uh, p in zip(ens.members, ics, plans):
            m.set_option("fft_plan", p)
            m.set_state_spectral(uh)
        ens.step(3)
        ens.step(2)
        got = [m.get_state_spectral() for m in ens.members]
    for i, N in enumerate(Ns):
        solo = _run(N, dtype, ics[i], plans[i], steps=5, nu=nu, dt=dt)
        assert np.array_equal(got[i], solo), f"member {i} (N={N}, plan {plans[i]})"


def test_tune_cache_applies_stored_choices_without_timing(tmp_path):
    from paper_1602_03638_gb300 import set_tune_cache

    path = tmp_path / "tune.txt"
    set_tune_cache(path)
    try:
        N, dtype = 32, "f32"
        uh = _iso(N, 11, dtype)
        picks = []
        for _ in range(2):
            with Solver(N, 0.01, 0.004, dtype) as s:
                s.set_state_spectral(uh)
                picks.append((s.tune_tiles(2), s.get_option("fft_plan")))
                assert np.array_equal(s.get_state_spectral(), uh) and s.diagnostics()["t"] == 0.0
        assert picks[0] == picks[1]
        lines = path.read_text().splitlines()
        assert len(lines) == 1 and lines[0].split()[0] == "tiles"  # the second tune read, not timed
        Ns = [16, 24, 16]
        ics = [_iso(n, 30 + i, dtype) for i, n in enumerate(Ns)]
        scheds = []
        for k in range(2):
            with Ensemble(Ns, [0.01] * 3, [0.004] * 3, dtype) as ens:
                for m, u in zip(ens.members, ics):
                    m.set_state_spectral(u)
                scheds.append(ens.tune())
                t = [m.diagnostics()["t"] for m in ens.members]
                assert (min(t) > 0.0) if k == 0 else (max(t) == 0.0)  # a stored schedule takes no steps
        assert scheds[0] == scheds[1]
        kinds = [ln.split()[0] for ln in path.read_text().splitlines()]
        assert kinds.count("ensemble") == 1 and kinds.count("tiles") == 3
    finally:
        set_tune_cache(None)


def test_new_handles_start_with_the_measured_default_masks():
    # the masks measured fastest on GB300 (dns_get_option reads them); one plan above 128
    expect = {(16, "f64"): 11, (64, "f64"): 11, (32, "f64"): 0, (96, "f64"): 0, (128, "f32"): 11,
              (48, "f32"): 9, (64, "f32"): 3, (96, "f32"): 0, (24, "f32"): 0, (256, "f32"): 0}
    for (N, dtype), mask in expect.items():
        with Solver(N, 0.01, 0.004, dtype) as s:
            assert s.get_option("fft_plan") == mask, (N, dtype)
    with Solver((32, 16, 24), 0.01, 0.004, "f32") as s:
        assert s.get_option("fft_plan") == 0
