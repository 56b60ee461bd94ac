"""GPU tests of the ensemble (many independent members of mixed grid sizes).

An ensemble step is one CUDA graph launch whose member kernel chains are
parallel branches; each member must end bit-for-bit where the same member
stepped alone ends (same kernels, same order of operations), and agree with
the FP64 oracle like a single solver does.
"""

import numpy as np
import pytest

from oracle import spectral_ns as sn
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


def _ics(Ns, dtype):
    return [inputs.isotropic_spectral(N, seed=100 + i, k0=2.0 + i % 4).numpy().astype(CPLX[dtype]) for i, N in enumerate(Ns)]


def _alone(N, nu, dt, dtype, uh, steps, plan=None):
    with Solver(N, nu, dt, dtype) as s:
        if plan is not None:  # else the handle's default plan, as the members'
            s.set_option("fft_plan", plan)
        s.set_state_spectral(uh)
        s.step(steps)
        return s.get_state_spectral()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("batching,streams", [(0, 0), (0, 1), (0, 3), (1 << 30, 0), (2, 0), (2, 2)])
def test_ensemble_members_match_solo_runs_bitwise(dtype, batching, streams):
    # equal sizes with different nu and dt share batched launches (per-member arguments)
    Ns = [16, 24, 32, 48, 64, 32, 16, 32]
    nus = [5e-3 + 1e-3 * i for i in range(len(Ns))]
    dts = [2e-3 * (1 + i % 2) for i in range(len(Ns))]
    ics = _ics(Ns, dtype)
    with Ensemble(Ns, nus, dts, dtype) as ens:
        ens.set_batching(batching)
        ens.set_streams(streams)
        for m, uh in zip(ens.members, ics):
            m.set_state_spectral(uh)
        ens.step(4)
        ens.step(3)
        got = [m.get_state_spectral() for m in ens.members]
        times = [m.diagnostics()["t"] for m in ens.members]
    for i, N in enumerate(Ns):
        ref = _alone(N, nus[i], dts[i], dtype, ics[i], 7)
        assert np.array_equal(got[i], ref), f"member {i} (N={N})"
        assert abs(times[i] - 7 * dts[i]) < 1e-12


def test_ensemble_member_matches_oracle():
    Ns = [32, 48]
    ics = _ics(Ns, "f64")
    with Ensemble(Ns, [0.01, 0.01], [0.01, 0.01], "f64") as ens:
        for m, uh in zip(ens.members, ics):
            m.set_state_spectral(uh)
        ens.step(10)
        got = [m.get_state_spectral() for m in ens.members]
    for i, N in enumerate(Ns):
        ref = sn.run(ics[i].astype(np.complex128), N, 0.01, 0.01, 10)
        assert np.linalg.norm(got[i] - ref) / np.linalg.norm(ref) < 1e-12


def test_batched_groups_split_by_dealias_rule_and_size_limit():
    # a member with the Appendix dealias rule and a 256^3 member (never batched)
    # among batchable 32^3 members: every member still matches its solo run
    Ns = [32, 32, 256, 32]
    ics = _ics(Ns, "f32")
    with Ensemble(Ns, [0.01] * 4, [0.004] * 4, "f32") as ens:
        ens.members[1].set_option("dealias_variant", 1)
        for m, uh in zip(ens.members, ics):
            m.set_state_spectral(uh)
        ens.step(3)
        got = [m.get_state_spectral() for m in ens.members]
    for i, N in enumerate(Ns):
        with Solver(N, 0.01, 0.004, "f32") as s:
            if i == 1:
                s.set_option("dealias_variant", 1)
            s.set_state_spectral(ics[i])
            s.step(3)
            assert np.array_equal(got[i], s.get_state_spectral()), f"member {i} (N={N})"


def test_ensemble_tune_advances_and_keeps_identity():
    Ns = [16, 32, 24, 32]
    ics = _ics(Ns, "f32")
    with Ensemble(Ns, [0.01] * 4, [0.005] * 4, "f32") as ens:
        for m, uh in zip(ens.members, ics):
            m.set_state_spectral(uh)
        pick = ens.tune()
        assert pick["batching"] == ens.batching and pick["streams"] == ens.streams
        assert pick["batching"] > 0 or 1 <= pick["streams"] <= len(Ns)
        taken = int(round(ens.members[0].diagnostics()["t"] / 0.005))
        assert taken >= 2 and taken % 2 == 0
        plans = [int(m.get_option("fft_plan")) for m in ens.members]  # chosen by the tuner
        ens.step(2)
        got = [m.get_state_spectral() for m in ens.members]
    for i, N in enumerate(Ns):
        assert np.array_equal(got[i], _alone(N, 0.01, 0.005, "f32", ics[i], taken + 2, plans[i]))


def test_ensemble_argument_errors():
    from paper_1602_03638_gb300 import _lib

    with pytest.raises(ValueError):
        Ensemble([16], [0.01, 0.02], [0.01], "f32")
    with pytest.raises(_lib.DnsError):
        Ensemble([16, 10], [0.01, 0.01], [0.01, 0.01], "f32")
    with Ensemble([16], [0.01], [0.01], "f32") as ens:
        with pytest.raises(_lib.DnsError):
            ens.step(-1)
        with pytest.raises(_lib.DnsError):
            ens.set_streams(-2)
        with pytest.raises(_lib.DnsError):
            ens.set_batching(-1)
