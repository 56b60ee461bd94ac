"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances. The FP64 form follows the oracle to rounding: transforms and a
single right-hand side agree to ~1e-15 relative, so the tests use 1e-12; after
100 RK4 steps at 32^3 the relative L2 error of the state must be <= 1e-12.
The FP32 form rounds every transform to ~6e-8 * log2(N): single evaluations
are held to 2e-5 (max-norm, relative to the largest coefficient) and the
100-step state to the relative L2 bound 1e-5.
"""

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import Solver, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"f64": 1e-12, "f32": 2e-5}
NP_REAL = {"f64": np.float64, "f32": np.float32}
NP_CPLX = {"f64": np.complex128, "f32": np.complex64}


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def random_physical(N, seed, dtype):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3, N, N, N)).astype(NP_REAL[dtype])


def iso_state(N, seed, dtype, k0=None):
    uh = inputs.isotropic_spectral(N, seed=seed, k0=k0 or max(2.0, N / 8.0)).numpy()
    return uh.astype(NP_CPLX[dtype])


# ---------------------------------------------------------------- transforms

@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [8, 12, 16, 24, 32, 48, 64, 96])
def test_forward_transform(N, dtype):
    u = random_physical(N, N, dtype)
    with Solver(N, 0.0, 0.01, dtype) as s:
        s.set_state(u)
        got = s.get_state_spectral()
    ref = sn.to_spectral(u.astype(np.float64))
    assert rel_max(got, ref) < TOL[dtype]
    # Nyquist modes are not part of the state
    assert np.all(got[:, N // 2] == 0) and np.all(got[:, :, N // 2] == 0) and np.all(got[..., N // 2] == 0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [8, 12, 32, 48, 128])
def test_inverse_transform_with_c2r_convention(N, dtype):
    # arbitrary (non-Hermitian) half spectrum: c2r ignores Im at kz = 0
    rng = np.random.default_rng(1000 + N)
    uh = (rng.standard_normal((3, N, N, N // 2 + 1)) + 1j * rng.standard_normal((3, N, N, N // 2 + 1))).astype(NP_CPLX[dtype])
    with Solver(N, 0.0, 0.01, dtype) as s:
        s.set_state_spectral(uh)
        got = s.get_state()
    ref = sn.inverse(sn.zero_nyquist(uh.astype(np.complex128)))
    assert rel_max(got, ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_spectral_round_trip_is_exact(dtype):
    N = 32
    uh = iso_state(N, 3, dtype)
    with Solver(N, 0.0, 0.01, dtype) as s:
        s.set_state_spectral(uh)
        got = s.get_state_spectral()
    assert np.array_equal(got, uh)  # a pure layout transpose


# ---------------------------------------------------------------- one right-hand side

@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N,variant", [(8, 0), (12, 0), (16, 1), (24, 0), (32, 0), (32, 1), (48, 0), (64, 1), (96, 0)])
def test_rhs_matches_oracle(N, variant, dtype):
    uh = iso_state(N, 7 + N, dtype, k0=N / 5.0)
    nu = 0.013
    with Solver(N, nu, 0.01, dtype, dealias_variant=variant) as s:
        s.set_state_spectral(uh)
        got = s.rhs()
        still = s.get_state_spectral()
    ref = sn.rhs(uh.astype(np.complex128), sn.Grid(N, variant), nu)
    assert rel_max(got, ref) < TOL[dtype]
    assert np.array_equal(still, uh)  # rhs() leaves the state alone


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rhs_of_full_state_outside_the_mask(dtype):
    # modes outside the 2/3 box present in the state: they enter the product
    N = 32
    u = random_physical(N, 99, dtype) * 0.1
    with Solver(N, 0.02, 0.01, dtype) as s:
        s.set_state(u)
        uh = s.get_state_spectral()
        got = s.rhs()
    ref = sn.rhs(uh.astype(np.complex128), sn.Grid(N), 0.02)
    assert rel_max(got, ref) < TOL[dtype]


# ---------------------------------------------------------------- RK4 trajectories

def _run_gpu(N, nu, dt, steps, dtype, uh=None, u=None, variant=0, graph=1):
    with Solver(N, nu, dt, dtype, dealias_variant=variant) as s:
        s.set_option("use_graph", graph)
        if uh is not None:
            s.set_state_spectral(uh)
        else:
            s.set_state(u)
        s.step(steps)
        return s.get_state_spectral(), s.diagnostics()


@pytest.mark.parametrize("dtype,bound", [("f64", 1e-12), ("f32", 1e-5)])
def test_taylor_green_32_100_steps(dtype, bound):
    # the small Taylor-Green case: 32^3, nu = 0.01, dt = 0.01, 100 steps, N/3 mask
    N, nu, dt, steps = 32, 0.01, 0.01, 100
    u = inputs.taylor_green(N).astype(NP_REAL[dtype])
    got, diag = _run_gpu(N, nu, dt, steps, dtype, u=u)
    ref = sn.run(sn.to_spectral(u.astype(np.float64)), N, nu, dt, steps)
    err = rel_l2(got, ref)
    assert err <= bound, err
    assert abs(diag["t"] - 1.0) < 1e-12
    d = sn.diagnostics(ref, nu)
    assert abs(diag["energy"] - d["energy"]) < 10 * bound * d["energy"]
    assert abs(diag["dissipation"] - d["dissipation"]) < 10 * bound * d["dissipation"]


@pytest.mark.parametrize("dtype,bound", [("f64", 1e-12), ("f32", 1e-5)])
def test_isotropic_32_100_steps(dtype, bound):
    N, nu, dt, steps = 32, 0.01, 0.01, 100
    uh = iso_state(N, 11, dtype, k0=4.0)
    got, _ = _run_gpu(N, nu, dt, steps, dtype, uh=uh)
    ref = sn.run(uh.astype(np.complex128), N, nu, dt, steps)
    assert rel_l2(got, ref) <= bound


@pytest.mark.parametrize("N", [48, 96])
def test_radix3_grids_20_steps(N):
    uh = iso_state(N, 5, "f64", k0=3.0)
    got, _ = _run_gpu(N, 0.005, 0.004, 20, "f64", uh=uh)
    ref = sn.run(uh.astype(np.complex128), N, 0.005, 0.004, 20)
    assert rel_l2(got, ref) <= 1e-12


def test_graph_and_eager_launches_agree_bitwise():
    N = 32
    uh = iso_state(N, 21, "f32")
    a, _ = _run_gpu(N, 0.01, 0.01, 5, "f32", uh=uh, graph=1)
    b, _ = _run_gpu(N, 0.01, 0.01, 5, "f32", uh=uh, graph=0)
    assert np.array_equal(a, b)


def test_split_steps_equal_one_call():
    N = 16
    uh = iso_state(N, 4, "f64")
    with Solver(N, 0.02, 0.01, "f64") as s:
        s.set_state_spectral(uh)
        s.step(3)
        s.step(0)
        s.step(4)
        a = s.get_state_spectral()
        t = s.diagnostics()["t"]
    b, _ = _run_gpu(N, 0.02, 0.01, 7, "f64", uh=uh)
    assert np.array_equal(a, b)
    assert abs(t - 0.07) < 1e-15


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_checkpoint_and_resume_equal_an_uninterrupted_run(dtype):
    # checkpoint = the spectral state and the time; a new handle resumes from it
    N, nu, dt = 24, 0.01, 0.005
    uh = iso_state(N, 33, dtype)
    with Solver(N, nu, dt, dtype) as s:
        s.set_state_spectral(uh)
        s.step(4)
        ck, t = s.get_state_spectral(), s.diagnostics()["t"]
    with Solver(N, nu, dt, dtype) as r:
        r.set_state_spectral(ck)
        r.set_option("time", t)
        r.step(3)
        resumed, tr = r.get_state_spectral(), r.diagnostics()["t"]
    ref, d = _run_gpu(N, nu, dt, 7, dtype, uh=uh)
    assert np.array_equal(resumed, ref)
    assert tr == d["t"]


def test_abc_flow_decays_by_rk4_polynomial_on_gpu():
    N, nu, dt, n = 16, 0.2, 0.1, 7
    u = inputs.abc_flow(N)
    got, _ = _run_gpu(N, nu, dt, n, "f64", u=u)
    uh0 = sn.to_spectral(u)
    z = -nu * dt
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    assert np.abs(got - uh0 * R ** n).max() < 1e-12 * np.abs(uh0).max()


@pytest.mark.parametrize("variant", [0, 1])
def test_worked_example_energy_on_gpu(variant):
    # Appendix: N = 128, nu = 0.000625, dt = 0.01, 10 RK4 steps, FP64
    u = inputs.taylor_green(128)
    _, diag = _run_gpu(128, 0.000625, 0.01, 10, "f64", u=u, variant=variant)
    assert abs(diag["energy"] - 0.124953117517) < 1e-12


# ---------------------------------------------------------------- diagnostics

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_diagnostics_match_oracle(dtype):
    N, nu = 32, 0.017
    uh = iso_state(N, 8, dtype)
    with Solver(N, nu, 0.01, dtype) as s:
        s.set_state_spectral(uh)
        d = s.diagnostics()
    ref = sn.diagnostics(uh.astype(np.complex128), nu)
    tol = 1e-12 if dtype == "f64" else 1e-6
    for key in ("energy", "dissipation", "helicity", "enstrophy"):
        assert abs(d[key] - ref[key]) <= tol * max(abs(ref[key]), 1e-3), key
    assert d["max_div"] < (1e-12 if dtype == "f64" else 1e-4)


def test_divergence_diagnostic_sees_a_divergent_field():
    N = 16
    X = sn.mesh(N)
    u = np.zeros((3, N, N, N))
    u[0] = np.sin(X[0])  # div u = cos x, max 1
    with Solver(N, 0.0, 0.01, "f64") as s:
        s.set_state(u)
        d = s.diagnostics()
    assert abs(d["max_div"] - 1.0) < 1e-13


def test_nonfinite_state_is_reported():
    N = 16
    u = inputs.taylor_green(N)
    u[1, 3, 4, 5] = np.nan
    from paper_1602_03638_gb300 import _lib

    with Solver(N, 0.01, 0.01, "f64") as s:
        s.set_state(u)
        with pytest.raises(_lib.DnsError) as ei:
            s.diagnostics()
        assert ei.value.code == _lib.DNS_ERR_NONFINITE


# ---------------------------------------------------------------- memory and pointers

def test_device_and_host_buffers_agree():
    N = 32
    u = inputs.taylor_green(N).astype(np.float32)
    with Solver(N, 0.01, 0.01, "f32") as s:
        s.set_state(torch.from_numpy(u).cuda())
        s.step(2)
        dev = torch.empty((3, N, N, N), dtype=torch.float32, device="cuda")
        s.get_state(dev)
        host = s.get_state()
        dsp = torch.empty((3, N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
        s.get_state_spectral(dsp)
        hsp = s.get_state_spectral()
    assert np.array_equal(dev.cpu().numpy(), host)
    assert np.array_equal(dsp.cpu().numpy(), hsp)


def test_user_stream_is_used():
    N = 16
    u = inputs.taylor_green(N)
    st = torch.cuda.Stream()
    with Solver(N, 0.01, 0.01, "f64") as s:
        s.set_stream(st)
        s.set_state(torch.from_numpy(u).cuda())
        s.step(3)
        a = s.get_state_spectral()
    b, _ = _run_gpu(N, 0.01, 0.01, 3, "f64", u=u)
    assert np.array_equal(a, b)


def test_allocation_failure_is_reported_and_recoverable():
    from paper_1602_03638_gb300 import _lib

    L = _lib.lib()
    for k in range(1, 8):
        assert L.dns_debug_fail_alloc_after(k) == 0
        with pytest.raises(_lib.DnsError) as ei:
            Solver(32, 0.01, 0.01, "f32")
        assert ei.value.code == _lib.DNS_ERR_OOM
    L.dns_debug_fail_alloc_after(0)
    with Solver(32, 0.01, 0.01, "f32") as s:
        assert s.device_bytes() > 0


def test_option_validation_on_device():
    from paper_1602_03638_gb300 import _lib

    with Solver(16, 0.01, 0.01, "f32") as s:
        with pytest.raises(_lib.DnsError):
            s.set_option("no_such_key", 1.0)
        with pytest.raises(_lib.DnsError):
            s.set_option("dealias_variant", 2)
        with pytest.raises(_lib.DnsError):
            s.step(-1)
        s.set_option("time", 5.0)
        assert s.diagnostics()["t"] == 5.0


# ---------------------------------------------------------------- full sizes, sampled

def _tg_low_k_reference(Nref, nu, dt, steps):
    return sn.run(sn.to_spectral(inputs.taylor_green(Nref)), Nref, nu, dt, steps)


def _low_block(uh, n):
    """Modes |kx|,|ky| <= n, 0 <= kz <= n of a (3,N,N,N/2+1) array (paper order)."""
    idx = list(range(0, n + 1)) + list(range(-n, 0))
    return uh[:, idx][:, :, idx][:, :, :, : n + 1]


@pytest.mark.parametrize("N,dtype", [(256, "f64"), (512, "f32"), (1024, "f32")])
def test_full_size_taylor_green_steps_match_low_resolution_oracle(N, dtype):
    # Taylor-Green at the bench sizes (nu = 1/1600, dt = 1e-3): for 10 steps
    # all energy stays at |k| < 16, so the state equals the oracle's 64^3 run
    # mode by mode (coefficients scale with N^3).
    nu, dt, steps, Nref = 1.0 / 1600, 1e-3, 10, 64
    ref = _tg_low_k_reference(Nref, nu, dt, steps) * (N / Nref) ** 3
    with Solver(N, nu, dt, dtype) as s:
        s.set_state(inputs.taylor_green_torch(N, device="cuda", dtype=torch.float64 if dtype == "f64" else torch.float32))
        s.step(steps)
        out = torch.empty((3, N, N, N // 2 + 1), dtype=torch.complex128 if dtype == "f64" else torch.complex64, device="cuda")
        s.get_state_spectral(out)
        d = s.diagnostics()
    n = 12
    idx = torch.tensor(list(range(0, n + 1)) + list(range(-n, 0)), device="cuda") % N
    low = out[:, idx][:, :, idx][:, :, :, : n + 1].cpu().numpy()
    refl = _low_block(ref, n)
    scale = np.abs(refl).max()
    assert np.abs(low - refl).max() < (1e-11 if dtype == "f64" else 2e-5) * scale
    # everything outside the low block is (numerically) empty
    mask = torch.ones((N,), dtype=torch.bool, device="cuda")
    mask[idx] = False
    rest = max(float(out[:, mask].abs().max()), float(out[:, :, mask].abs().max()), float(out[:, :, :, n + 1:].abs().max()))
    assert rest < (1e-11 if dtype == "f64" else 2e-5) * scale
    e_ref = sn.energy(ref / (N / Nref) ** 3)
    assert abs(d["energy"] - e_ref) < (1e-12 if dtype == "f64" else 1e-6)
    assert d["max_div"] < (1e-10 if dtype == "f64" else 1e-4)
