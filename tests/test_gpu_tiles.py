"""GPU tests of the y- and z-pass tile widths and their tuner (options
"y_tile_inverse", "y_tile_forward", "z_tile", dns_tune_tiles, and the tile step of
dns_ensemble_tune).

A tile width only decides how many x columns one block of a pass transforms; each
column's arithmetic is the same, so every offered width must give the default's
result bit for bit, and tuning must not change the state or the time.
"""

import math

import numpy as np
import pytest

from paper_1602_03638_gb300 import Ensemble, Solver, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CPLX = {"f32": np.complex64, "f64": np.complex128}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()


def _offered(s, key="y_tile_inverse"):
    out = []
    for t in (4, 8, 16, 32):
        try:
            s.set_option(key, t)
            out.append(t)
        except RuntimeError:
            pass
    s.set_option(key, 0)
    return out


def _steps(N, dtype, uh, ti=0, tf=0, tz=0, n=3):
    with Solver(N, 0.01, 0.004, dtype) as s:
        s.set_option("y_tile_inverse", ti)
        s.set_option("y_tile_forward", tf)
        s.set_option("z_tile", tz)
        s.set_state_spectral(uh)
        s.step(n)
        return s.get_state_spectral()


@pytest.mark.parametrize("N,dtype", [(32, "f32"), (48, "f32"), (64, "f32"), (96, "f32"), (32, "f64"), (64, "f64")])
def test_every_offered_tile_width_gives_the_default_result(N, dtype):
    uh = inputs.isotropic_spectral(N, seed=N, k0=3.0).numpy().astype(CPLX[dtype])
    with Solver(N, 0.01, 0.004, dtype) as s:
        tiles = _offered(s)
        ztiles = _offered(s, "z_tile")
    assert tiles and ztiles, "the small grids offer tile widths"
    ref = _steps(N, dtype, uh)
    for t in tiles:
        assert np.array_equal(_steps(N, dtype, uh, ti=t), ref), f"inverse width {t}"
        assert np.array_equal(_steps(N, dtype, uh, tf=t), ref), f"forward width {t}"
    for t in ztiles:
        assert np.array_equal(_steps(N, dtype, uh, tz=t), ref), f"z width {t}"


def test_large_grids_offer_only_the_default():
    with Solver(256, 0.01, 0.004, "f32") as s:
        assert _offered(s) == [] and _offered(s, "z_tile") == []
        s.set_option("y_tile_forward", 0)
        assert s.tune_tiles(2) == (0, 0, 0)


def test_tuner_keeps_state_and_time_and_picks_an_offered_width():
    N, dtype = 64, "f32"
    uh = inputs.isotropic_spectral(N, seed=3, k0=3.0).numpy().astype(CPLX[dtype])
    with Solver(N, 0.01, 0.004, dtype) as s:
        s.set_state_spectral(uh)
        s.step(2)
        before = s.get_state_spectral()
        t_before = s.diagnostics()["t"]
        offered, zoffered = _offered(s), _offered(s, "z_tile")
        ti, tf, tz = s.tune_tiles(3)
        assert ti in [0] + offered and tf in [0] + offered and tz in [0] + zoffered
        assert (s.get_option("y_tile_inverse"), s.get_option("y_tile_forward"), s.get_option("z_tile")) == (ti, tf, tz)
        assert np.array_equal(s.get_state_spectral(), before)
        assert s.diagnostics()["t"] == t_before
        s.step(3)
        got = s.get_state_spectral()
        plan = s.get_option("fft_plan")  # the tuner's radix plans change the rounding, not the widths
    with Solver(N, 0.01, 0.004, dtype) as r:
        r.set_state_spectral(uh)
        r.step(2)
        r.set_option("fft_plan", plan)
        r.step(3)
        assert np.array_equal(got, r.get_state_spectral())


def test_get_option_round_trips():
    with Solver(32, 0.02, 0.005, "f64", integrator="heun", lengths=(math.pi, 2 * math.pi, 3 * math.pi)) as s:
        assert s.get_option("integrator") == 2
        assert s.get_option("Lx") == math.pi and s.get_option("Lz") == 3 * math.pi
        assert s.get_option("nu") == 0.02 and s.get_option("dt") == 0.005
        s.set_option("y_tile_forward", 8)
        assert s.get_option("y_tile_forward") == 8
        with pytest.raises(RuntimeError):
            s.get_option("no_such_key")


def test_tuned_ensemble_members_match_solo_runs():
    Ns = [32, 48, 64, 32, 64]
    nu, dt, dtype = 0.005, 0.002, "f32"
    ics = [inputs.isotropic_spectral(N, seed=80 + i, k0=3.0).numpy().astype(CPLX[dtype]) for i, N in enumerate(Ns)]
    with Ensemble(Ns, [nu] * len(Ns), [dt] * len(Ns), dtype) as ens:
        for m, uh in zip(ens.members, ics):
            m.set_state_spectral(uh)
        sched = ens.tune()
        assert set(sched["tiles"]) == set(Ns)
        taken = [m.diagnostics()["t"] for m in ens.members]
        plans = [m.get_option("fft_plan") for m in ens.members]
        assert all(p == sched["tiles"][N]["plan"] for p, N in zip(plans, Ns))
        ens.step(3)
        got = [m.get_state_spectral() for m in ens.members]
    for i, N in enumerate(Ns):
        steps = int(round(taken[i] / dt)) + 3
        with Solver(N, nu, dt, dtype) as s:
            s.set_option("fft_plan", plans[i])
            s.set_state_spectral(ics[i])
            s.step(steps)
            ref = s.get_state_spectral()
        assert np.array_equal(got[i], ref), f"member {i} (N={N})"
