"""GPU tests of the explicit Runge-Kutta schemes selected by the "integrator"
option (forward Euler of Sec. 3.1, the two-stage Heun and midpoint rules, the
low-storage 2N schemes of Williamson and of Carpenter & Kennedy; RK4 of the
Appendix is the default and is covered by test_gpu_parity.py) and of schemes set
through dns_set_rk_tableau.

Each scheme runs through the same x-stage kernel as RK4, with the stage roles
(first / between / last) taken from the scheme's stage count; a one-stage step
updates the state in place. Parity bounds as for RK4: FP64 1e-12, FP32 1e-5
relative L2 after 100 steps at 32^3 against the FP64 oracle.
"""

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import Ensemble, Solver, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCHEMES = ["euler", "heun", "midpoint"]
CPLX = {"f32": np.complex64, "f64": np.complex128}
R = {"euler": lambda z: 1 + z, "heun": lambda z: 1 + z + z * z / 2, "midpoint": lambda z: 1 + z + z * z / 2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _iso(N, seed, dtype):
    return inputs.isotropic_spectral(N, seed=seed, k0=4.0).numpy().astype(CPLX[dtype])


def _run(N, nu, dt, steps, dtype, uh, scheme, graph=1):
    with Solver(N, nu, dt, dtype, integrator=scheme) as s:
        s.set_option("use_graph", graph)
        s.set_state_spectral(uh)
        s.step(steps)
        return s.get_state_spectral(), s.diagnostics()


@pytest.mark.parametrize("dtype,bound", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_isotropic_32_100_steps_match_oracle(scheme, dtype, bound):
    N, nu, dt, steps = 32, 0.01, 0.005, 100
    uh = _iso(N, 31, dtype)
    got, diag = _run(N, nu, dt, steps, dtype, uh, scheme)
    ref = sn.run(uh.astype(np.complex128), N, nu, dt, steps, scheme=scheme)
    assert rel_l2(got, ref) <= bound
    assert abs(diag["t"] - steps * dt) < 1e-12


@pytest.mark.parametrize("scheme", SCHEMES)
def test_abc_flow_decays_by_the_scheme_polynomial(scheme):
    N, nu, dt, n = 16, 0.2, 0.1, 7
    u = inputs.abc_flow(N)
    with Solver(N, nu, dt, "f64", integrator=scheme) as s:
        s.set_state(u)
        s.step(n)
        got = s.get_state_spectral()
    uh0 = sn.to_spectral(u)
    assert np.abs(got - uh0 * R[scheme](-nu * dt) ** n).max() < 1e-12 * np.abs(uh0).max()


@pytest.mark.parametrize("scheme", SCHEMES)
def test_graph_and_eager_launches_agree_bitwise(scheme):
    uh = _iso(32, 8, "f32")
    a, _ = _run(32, 0.01, 0.005, 5, "f32", uh, scheme, graph=1)
    b, _ = _run(32, 0.01, 0.005, 5, "f32", uh, scheme, graph=0)
    assert np.array_equal(a, b)


def test_switching_the_integrator_between_steps():
    N, nu, dt = 24, 0.01, 0.005
    uh = _iso(N, 12, "f64")
    with Solver(N, nu, dt, "f64") as s:
        s.set_state_spectral(uh)
        s.step(3)
        s.set_option("integrator", 1)
        s.step(4)
        s.set_option("integrator", 3)
        s.step(2)
        got = s.get_state_spectral()
    ref = sn.run(uh.astype(np.complex128), N, nu, dt, 3)
    ref = sn.run(ref, N, nu, dt, 4, scheme="euler")
    ref = sn.run(ref, N, nu, dt, 2, scheme="midpoint")
    assert rel_l2(got, ref) <= 1e-12


@pytest.mark.parametrize("scheme,stages", [("euler", 1), ("heun", 2), ("rk4", 4)])
def test_profiled_steps_launch_four_kernels_per_stage(scheme, stages):
    with Solver(32, 0.01, 0.005, "f32", integrator=scheme) as s:
        s.set_state_spectral(_iso(32, 2, "f32"))
        prof = s.profile_steps(3)
    assert all(n == 3 * stages for _, n in prof.values())


def test_unknown_integrator_is_an_argument_error():
    with Solver(16, 0.01, 0.01, "f32") as s:
        with pytest.raises(RuntimeError):
            s.set_option("integrator", 6)
        with pytest.raises(RuntimeError):
            s.set_option("integrator", 2.5)
    with pytest.raises(ValueError):
        Solver(16, 0.01, 0.01, "f32", integrator="rk3")


@pytest.mark.parametrize("batching", [0, 1 << 30])
def test_ensemble_members_with_other_integrators_match_solo_runs(batching):
    # equal sizes with different schemes: batched launches group members by scheme
    Ns = [16, 16, 16, 24, 24, 16]
    schemes = ["euler", "rk4", "euler", "heun", "midpoint", "heun"]
    nu, dt, dtype = 0.01, 0.004, "f32"
    ics = [inputs.isotropic_spectral(N, seed=40 + i, k0=3.0).numpy().astype(CPLX[dtype]) for i, N in enumerate(Ns)]
    with Ensemble(Ns, [nu] * len(Ns), [dt] * len(Ns), dtype) as ens:
        ens.set_batching(batching)
        for m, uh, sc in zip(ens.members, ics, schemes):
            m.set_option("integrator", {"rk4": 0, "euler": 1, "heun": 2, "midpoint": 3}[sc])
            m.set_state_spectral(uh)
        ens.step(3)
        ens.step(2)
        got = [m.get_state_spectral() for m in ens.members]
    for i, N in enumerate(Ns):
        ref, _ = _run(N, nu, dt, 5, dtype, ics[i], schemes[i])
        assert np.array_equal(got[i], ref), f"member {i} ({schemes[i]})"


# ---------------------------------------------------------------- low-storage 2N schemes

@pytest.mark.parametrize("dtype,bound", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("scheme", ["williamson3", "ck45"])
def test_2n_schemes_32_100_steps_match_oracle(scheme, dtype, bound):
    N, nu, dt, steps = 32, 0.01, 0.005, 100
    uh = _iso(N, 33, dtype)
    got, diag = _run(N, nu, dt, steps, dtype, uh, scheme)
    ref = sn.run(uh.astype(np.complex128), N, nu, dt, steps, scheme=scheme)
    assert rel_l2(got, ref) <= bound
    assert abs(diag["t"] - steps * dt) < 1e-12


def _stability_2n(A, B, z):
    # u_j = u_{j-1} + B_j dU_j, dU_j = A_j dU_{j-1} + z u_{j-1} for du/dt = lambda u, z = lambda dt
    u, d = 1.0, 0.0
    for a, b in zip(A, B):
        d = a * d + z * u
        u = u + b * d
    return u


@pytest.mark.parametrize("scheme", ["williamson3", "ck45"])
def test_2n_abc_decay_on_gpu(scheme):
    N, nu, dt, n = 16, 0.2, 0.1, 9
    uh0 = sn.to_spectral(inputs.abc_flow(N))
    got, _ = _run(N, nu, dt, n, "f64", uh0, scheme)
    A, B = sn.LSRK_SCHEMES[scheme]
    assert np.abs(got - uh0 * _stability_2n(A, B, -nu * dt) ** n).max() < 1e-12 * np.abs(uh0).max()


def test_custom_tableau_through_the_c_abi():
    N, nu, dt, steps = 32, 0.01, 0.005, 20
    uh = _iso(N, 35, "f64")
    # the built-in schemes given as custom coefficients run bit for bit the same
    A, B = sn.LSRK_SCHEMES["williamson3"]
    with Solver(N, nu, dt, "f64") as s:
        s.set_rk_tableau(1, A, B)
        assert s.get_option("integrator") == 4
        s.set_state_spectral(uh)
        s.step(steps)
        custom = s.get_state_spectral()
    builtin, _ = _run(N, nu, dt, steps, "f64", uh, "williamson3")
    np.testing.assert_array_equal(custom, builtin)
    # a scheme with no built-in entry: Heun's third-order method in the Appendix form
    # (Butcher A[1][0] = 1/3, A[2][1] = 2/3, weights 1/4, 0, 3/4)
    a, b = (0.25, 0.0, 0.75), (1.0 / 3.0, 2.0 / 3.0)
    with Solver(N, nu, dt, "f64") as s:
        s.set_rk_tableau(0, a, b)
        assert s.get_option("integrator") == -1
        s.set_state_spectral(uh)
        s.step(steps)
        got = s.get_state_spectral()
    g = sn.Grid(N)
    ref = uh.copy()
    for _ in range(steps):
        u0, acc, cur = ref.copy(), ref.copy(), ref
        for st in range(3):
            d = sn.rhs(cur, g, nu)
            if st < 2:
                cur = u0 + b[st] * dt * d
            acc = acc + a[st] * dt * d
        ref = acc
    assert rel_l2(got, ref) <= 1e-12


def test_2n_members_batched_in_an_ensemble_equal_solo_runs():
    N, nu, dt, steps = 32, 0.01, 0.005, 10
    uhs = [_iso(N, 40 + i, "f32") for i in range(3)]
    with Ensemble([N] * 3, [nu] * 3, [dt] * 3, "f32") as ens:
        for m, uh in zip(ens.members, uhs):
            m.set_option("integrator", 4)
            m.set_state_spectral(uh)
        ens.step(steps)
        ens.synchronize()
        got = [m.get_state_spectral() for m in ens.members]
    for g_, uh in zip(got, uhs):
        solo, _ = _run(N, nu, dt, steps, "f32", uh, "williamson3")
        np.testing.assert_array_equal(g_, solo)
