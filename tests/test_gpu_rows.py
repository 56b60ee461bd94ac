"""GPU tests of the row pruning of a state that vanishes outside the 2/3 box (option
"prune_rows", the row flag of the stage launches).

The 2/3 rule (Sec. 3.1) removes the nonlinear term on every mode with 3|k_i| >= N_i; there
the right-hand side of Eq. NSfinal is -nu |k|^2 u_hat. A state that vanishes on every row
(kz, ky) outside the box therefore keeps vanishing there under any explicit RK stage, and
the transforms of those rows are transforms of zeros. The solver checks the state on the
device whenever it is set (or the dealias rule changes) and then skips those rows: the
x-stage and the x inverse leave them alone, the y-inverse transforms only the planes
kz < N/3 and reads the other rows as zeros, the z-pass reads only kz < N/3; where the state
also vanishes at |kx| >= N/3 (flag "box_vanish"), the x-stage reads and writes its rows at the
kept columns only. Skipping zeros
changes no nonzero sum, so the pruned steps must equal the full ones (prune_rows = 0) bit
for bit (exact zeros of either sign compare equal) on every z-pass kernel, integrator,
dealias rule and schedule; a state with modes outside the box must take the full path.
"""

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import Ensemble, Solver, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CPLX = {"f32": np.complex64, "f64": np.complex128}
TCPLX = {"f32": torch.complex64, "f64": torch.complex128}


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


def _full_spectrum(N, seed, dtype):
    rng = np.random.default_rng(seed)
    return sn.to_spectral(rng.standard_normal((3, N, N, N))).astype(CPLX[dtype])


def _run(N, dtype, uh, steps, prune, nu=0.01, dt=0.004, **opts):
    with Solver(N, nu, dt, dtype) as s:
        s.set_option("prune_rows", prune)
        for k, v in opts.items():
            s.set_option(k, v)
        s.set_state_spectral(uh)
        vanish = s.get_option("rows_vanish")
        s.step(steps)
        return s.get_state_spectral(), vanish


def test_flag_follows_the_state():
    N = 48
    with Solver(N, 0.01, 0.004, "f32") as s:
        assert s.get_option("rows_vanish") == 1.0  # a new handle holds the zero state
        assert s.get_option("box_vanish") == 1.0
        assert s.get_option("prune_rows") == 1.0
        s.set_state_spectral(_iso(N, 1, "f32"))
        assert s.get_option("rows_vanish") == 1.0 and s.get_option("box_vanish") == 1.0
        s.set_state_spectral(_full_spectrum(N, 2, "f32"))
        assert s.get_option("rows_vanish") == 0.0 and s.get_option("box_vanish") == 0.0
        # one mode at ky = N/3: outside the box of 3|k| < N, inside the one of 3|k| < N + 2
        uh = np.zeros((3, N, N, N // 2 + 1), np.complex64)
        uh[0, 1, N // 3, 1] = 1.0
        s.set_state_spectral(uh)
        assert s.get_option("rows_vanish") == 0.0
        s.set_option("dealias_variant", 1)
        assert s.get_option("rows_vanish") == 1.0
        s.set_option("dealias_variant", 0)
        assert s.get_option("rows_vanish") == 0.0
        # kz = N/3 likewise; kx = N/3 is inside a kept row and does not matter
        uh[:] = 0
        uh[0, 1, 1, N // 3] = 1.0
        s.set_state_spectral(uh)
        assert s.get_option("rows_vanish") == 0.0
        uh[:] = 0
        uh[1, N // 3, 1, 1] = 1.0
        s.set_state_spectral(uh)
        assert s.get_option("rows_vanish") == 1.0 and s.get_option("box_vanish") == 0.0
        uh[1, N // 3, 1, 1] = 0.0
        uh[1, N // 3 - 1, 1, 1] = 1.0
        s.set_state_spectral(uh)
        assert s.get_option("box_vanish") == 1.0
        uh[:] = 0
        uh[2, 3, N // 2 - 1, 2] = np.nan  # NaN counts as nonzero
        s.set_state_spectral(uh)
        assert s.get_option("rows_vanish") == 0.0
        for bad in (2, -1, 0.5):
            with pytest.raises(RuntimeError):
                s.set_option("prune_rows", bad)


# every z-pass kernel: generic shared-memory (16, 48, 96, 512 FP64), canonical register
# (256 FP64), quarter-warp (256 FP32), half-warp pipelined (512 and 1024 FP32)
CASES = [(16, "f64", 20), (48, "f32", 20), (96, "f32", 8), (256, "f32", 3), (256, "f64", 2), (512, "f32", 2),
         (512, "f64", 1)]


@pytest.mark.parametrize("N,dtype,steps", CASES)
def test_pruned_steps_equal_full_steps(N, dtype, steps):
    dev = torch.device("cuda")
    uh = inputs.isotropic_spectral(N, seed=N, k0=max(2.0, N / 8.0), device=dev, dtype=TCPLX[dtype])
    out = []
    for prune in (1, 0):
        with Solver(N, 0.002, 0.002, dtype) as s:
            s.set_option("prune_rows", prune)
            s.set_state_spectral(uh)
            assert s.get_option("rows_vanish") == 1.0
            s.step(steps)
            o = torch.empty_like(uh)
            s.get_state_spectral(o)
            torch.cuda.synchronize()
            out.append(o)
    assert torch.equal(out[0], out[1])
    assert float(out[0].abs().max()) > 0.0


def test_pruned_steps_equal_full_steps_1024_f32():
    N, dev = 1024, torch.device("cuda")
    # Taylor-Green in its exact spectral form: every mode outside (+-1, +-1, 1) is zero
    uh = inputs.taylor_green_spectral(N, device=dev, dtype=torch.complex64)
    out = []
    for prune in (1, 0):
        with Solver(N, 1.0 / 1600, 1e-3, "f32") as s:
            s.set_option("prune_rows", prune)
            s.set_state_spectral(uh)
            assert s.get_option("rows_vanish") == 1.0
            s.step(2)
            o = torch.empty_like(uh)
            s.get_state_spectral(o)
            torch.cuda.synchronize()
            out.append(o)
    assert torch.equal(out[0], out[1])


def test_pruned_taylor_green_matches_oracle():
    N, nu, dt, steps = 32, 0.01, 0.01, 100  # the oracle's first configuration
    uh = inputs.taylor_green_spectral(N).numpy()
    ref = sn.run(uh, N, nu, dt, steps)
    for dtype, bound in (("f64", 1e-12), ("f32", 1e-5)):
        got, vanish = _run(N, dtype, uh.astype(CPLX[dtype]), steps, 1, nu=nu, dt=dt)
        assert vanish == 1.0
        assert rel_l2(got, ref) <= bound, dtype


@pytest.mark.parametrize("N,dtype", [(48, "f32"), (96, "f64"), (512, "f32")])
def test_columns_outside_the_box_in_kept_rows(N, dtype):
    # modes at |kx| >= N/3 on rows inside the box: the rows are pruned, the columns are not
    rng = np.random.default_rng(N)
    uh = inputs.isotropic_spectral(N, seed=11, k0=max(2.0, N / 8.0), device="cuda", dtype=TCPLX[dtype])
    for kx in (N // 3 + 1, N - N // 3 - 1, N // 2 - 1):
        uh[0, kx, 3, 2] = complex(rng.standard_normal(), rng.standard_normal())
        uh[2, kx, N - 2, 1] = complex(rng.standard_normal(), rng.standard_normal())
    out = []
    for prune in (1, 0):
        with Solver(N, 0.01, 0.004, dtype) as s:
            s.set_option("prune_rows", prune)
            s.set_state_spectral(uh)
            assert s.get_option("rows_vanish") == 1.0 and s.get_option("box_vanish") == 0.0
            s.step(3)
            o = torch.empty_like(uh)
            s.get_state_spectral(o)
            torch.cuda.synchronize()
            out.append(o)
    assert torch.equal(out[0], out[1])


def test_out_of_box_state_takes_the_full_path():
    N = 32
    uh = _full_spectrum(N, 3, "f64")
    a, va = _run(N, "f64", uh, 5, 1)
    b, vb = _run(N, "f64", uh, 5, 0)
    assert va == 0.0 and np.array_equal(a, b)
    assert rel_l2(a, sn.run(uh, N, 0.01, 0.004, 5)) <= 1e-12


@pytest.mark.parametrize("integrator", [1, 2, 4, 5])
def test_pruned_integrators(integrator):
    N = 32
    uh = _iso(N, 4, "f64")
    a, _ = _run(N, "f64", uh, 6, 1, integrator=integrator)
    b, _ = _run(N, "f64", uh, 6, 0, integrator=integrator)
    assert np.array_equal(a, b)


def test_pruned_dealias_variant_and_rhs():
    N = 48
    uh = _iso(N, 5, "f32")
    # a mode at ky = N/3, inside the box of the Appendix rule (3|k| < N + 2) only, with
    # kx u + ky v = 0 (divergence-free)
    uh[0, 1, N // 3, 2] = 0.5
    uh[1, 1, N // 3, 2] = -0.5 / (N // 3)
    a, va = _run(N, "f32", uh, 10, 1, dealias_variant=1)
    b, _ = _run(N, "f32", uh, 10, 0, dealias_variant=1)
    assert va == 1.0 and np.array_equal(a, b)
    rhs = []
    for prune in (1, 0):
        with Solver(N, 0.01, 0.004, "f32") as s:
            s.set_option("prune_rows", prune)
            s.set_option("dealias_variant", 1)
            s.set_state_spectral(uh)
            s.step(2)
            rhs.append(s.rhs())
    assert np.array_equal(rhs[0], rhs[1])


def test_new_state_after_pruned_steps_reads_no_stale_rows():
    # pruned steps leave the rows outside the box of the RK registers and of the work
    # arrays unwritten; a state with modes there must then run exactly like a fresh handle
    N = 64
    with Solver(N, 0.01, 0.004, "f32") as s:
        s.set_state_spectral(_iso(N, 6, "f32"))
        s.step(3)
        assert s.get_option("rows_vanish") == 1.0
        full = _full_spectrum(N, 7, "f32")
        s.set_state_spectral(full)
        assert s.get_option("rows_vanish") == 0.0
        s.step(4)
        got = s.get_state_spectral()
        s.set_state_spectral(full)
        rhs_got = s.rhs()
    ref, _ = _run(N, "f32", full, 4, 0)
    assert np.array_equal(got, ref)
    with Solver(N, 0.01, 0.004, "f32") as s:
        s.set_option("prune_rows", 0)
        s.set_state_spectral(full)
        assert np.array_equal(rhs_got, s.rhs())
    # and a switch of the dealias rule in the middle of a run: a mode at ky = 16 of 48 is
    # kept by 3|k| < N + 2 and not by 3|k| < N
    N = 48
    uh = _iso(N, 8, "f32")
    uh[0, 2, N // 3, 1] = 0.25
    outs = []
    for prune in (1, 0):
        with Solver(N, 0.01, 0.004, "f32") as s:
            s.set_option("prune_rows", prune)
            s.set_option("dealias_variant", 1)
            s.set_state_spectral(uh)
            s.step(3)
            s.set_option("dealias_variant", 0)  # the state now has a row outside the box
            assert s.get_option("rows_vanish") == 0.0
            s.step(3)
            outs.append(s.get_state_spectral())
    assert np.array_equal(outs[0], outs[1])


def test_tuner_with_the_flag():
    # the tuner times pruned steps from a saved state and restores it: the flag still holds
    N = 48
    uh = _iso(N, 9, "f32")
    with Solver(N, 0.01, 0.004, "f32") as s:
        s.set_state_spectral(uh)
        tiles = s.tune_tiles(2)
        plan = s.get_option("fft_plan")
        assert s.get_option("rows_vanish") == 1.0 and np.array_equal(s.get_state_spectral(), uh)
        s.step(4)
        got = s.get_state_spectral()
    with Solver(N, 0.01, 0.004, "f32") as s:
        s.set_option("prune_rows", 0)
        s.set_option("fft_plan", plan)
        for k, v in zip(("y_tile_inverse", "y_tile_forward", "z_tile"), tiles):
            s.set_option(k, v)
        s.set_state_spectral(uh)
        s.step(4)
        assert np.array_equal(s.get_state_spectral(), got)


@pytest.mark.parametrize("batching", [0, 1 << 30])
def test_ensemble_members_pruned(batching):
    Ns = [32, 48, 32, 64, 48, 96]
    ics = [_iso(n, 20 + i, "f32") for i, n in enumerate(Ns)]
    ics[2] = _full_spectrum(32, 30, "f32")  # one member outside the box, batched with a pruned one
    got = {}
    for prune in (1, 0):
        with Ensemble(Ns, [0.01] * len(Ns), [0.004] * len(Ns), "f32") as ens:
            ens.set_batching(batching)
            for m, u in zip(ens.members, ics):
                m.set_option("prune_rows", prune)
                m.set_state_spectral(u)
            flags = [m.get_option("rows_vanish") for m in ens.members]
            ens.step(3)
            got[prune] = [m.get_state_spectral() for m in ens.members]
    assert flags == [1.0, 1.0, 0.0, 1.0, 1.0, 1.0]
    for i in range(len(Ns)):
        assert np.array_equal(got[1][i], got[0][i]), f"member {i}"
