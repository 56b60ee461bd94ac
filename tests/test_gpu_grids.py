"""GPU tests on grids with a different number of points per direction (dns_create3;
Sec. 2 footnote: other point counts per direction).

Each compiled small grid (32 x 16 x 24 and 24 x 48 x 16, in both precisions) is
checked against the FP64 oracle on the same counts: state transfer, the two 3D
transforms, the right-hand side of a full-spectrum random field, 40 RK4 steps (both
dealias rules), a 2N scheme, box lengths, the diagnostics. Parity bounds as on the
cubic grids: FP64 1e-12, FP32 1e-5 relative L2 (FP32 transforms 1e-6).

The 1024 x 512 x 256 grid (the measured one) is checked at full size by (a) a dense
field band-limited to |k| <= (42, 42, 21) (the 2/3 box of 128 x 128 x 64), whose
right-hand side the oracle computes on a 256 x 256 x 128 grid (the product, |k| <=
(84, 84, 42), stays alias-free and inside both grids' 2/3 boxes, so the two
right-hand sides are the same Fourier coefficients up to the normalisation
Nx Ny Nz); (b) invariants of a white-noise field (every mode occupied) that hold at
any size: outside each direction's 2/3 box the right-hand side is -nu |k|^2 u_hat,
and inside it its nonlinear part (the right-hand side plus nu |k|^2 u_hat) is
divergence-free; (c) an RK4 run that keeps the state
divergence-free and follows the energy budget dE/dt = -eps.
"""

import numpy as np
import pytest

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import Solver, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CPLX = {"f32": np.complex64, "f64": np.complex128}
REAL = {"f32": np.float32, "f64": np.float64}
SMALL = [(32, 16, 24), (24, 48, 16)]
BIG = (1024, 512, 256)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _field(shape, seed, dtype, k0=3.0):
    return inputs.isotropic_spectral(shape, seed=seed, k0=k0).numpy().astype(CPLX[dtype])


def _full_spectrum(shape, seed, dtype):
    """State of a random physical field: every mode but the Nyquist ones occupied."""
    rng = np.random.default_rng(seed)
    return sn.to_spectral(rng.standard_normal((3,) + shape)).astype(CPLX[dtype])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", SMALL)
def test_state_round_trip_and_transforms(shape, dtype):
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal((3,) + shape).astype(REAL[dtype])
    tol = 1e-13 if dtype == "f64" else 1e-6
    with Solver(shape, 0.01, 1e-3, dtype) as s:
        assert (s.get_option("Nx"), s.get_option("Ny"), s.get_option("Nz")) == shape
        s.set_state(u)
        uh = s.get_state_spectral()
        ref = sn.to_spectral(u.astype(np.float64))
        assert rel_l2(uh, ref) <= tol
        back = s.get_state()
        assert rel_l2(back, sn.inverse(ref)) <= tol
        # spectral in, spectral out: the stored state is the input with Nyquist modes zeroed
        v = _full_spectrum(shape, 3, dtype)
        v[:, 1, 2, 3] += 1.0  # a non-Nyquist entry that set_state_spectral must keep
        s.set_state_spectral(v)
        assert np.array_equal(s.get_state_spectral(), sn.zero_nyquist(v))


@pytest.mark.parametrize("dtype,bound", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("shape", SMALL)
def test_rhs_of_a_full_spectrum_field_matches_oracle(shape, variant, dtype, bound):
    nu = 0.01
    uh = _full_spectrum(shape, 11, dtype)
    with Solver(shape, nu, 1e-3, dtype, dealias_variant=variant) as s:
        s.set_state_spectral(uh)
        got = s.rhs()
    ref = sn.rhs(uh.astype(np.complex128), sn.Grid(shape, variant), nu)
    assert rel_l2(got, ref) <= bound


@pytest.mark.parametrize("dtype,bound", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("shape", SMALL)
def test_40_rk4_steps_match_oracle(shape, variant, dtype, bound):
    nu, dt, steps = 0.01, 0.005, 40
    uh = _field(shape, 21, dtype)
    with Solver(shape, nu, dt, dtype, dealias_variant=variant) as s:
        s.set_state_spectral(uh)
        s.step(steps)
        got = s.get_state_spectral()
        d = s.diagnostics()
    ref = sn.run(uh.astype(np.complex128), shape, nu, dt, steps, variant=variant)
    assert rel_l2(got, ref) <= bound
    o = sn.diagnostics(ref, nu)
    # each quantity against its own scale (helicity against 2 sqrt(E Z), its Cauchy-Schwarz bound)
    scale = {"energy": o["energy"], "dissipation": o["dissipation"], "enstrophy": o["enstrophy"],
             "helicity": 2.0 * np.sqrt(o["energy"] * o["enstrophy"])}
    for key, sc in scale.items():
        assert abs(d[key] - o[key]) <= (1e-12 if dtype == "f64" else 5e-5) * sc
    assert d["max_div"] < (1e-12 if dtype == "f64" else 1e-4)


@pytest.mark.parametrize("dtype,bound", [("f64", 1e-12), ("f32", 1e-5)])
def test_2n_scheme_and_box_lengths_on_other_counts(dtype, bound):
    shape, nu, dt, steps, box = (32, 16, 24), 0.01, 0.004, 30, (2 * np.pi, np.pi, 3 * np.pi)
    uh = _field(shape, 5, dtype)
    with Solver(shape, nu, dt, dtype, integrator="williamson3", lengths=box) as s:
        s.set_state_spectral(uh)
        s.step(steps)
        got = s.get_state_spectral()
    ref = sn.run(uh.astype(np.complex128), shape, nu, dt, steps, scheme="williamson3", lengths=box)
    assert rel_l2(got, ref) <= bound


def test_abc_flow_decays_by_the_rk4_polynomial():
    # nu |k|^2 dt <= 1.75 for every mode of the grid (|k|^2 <= 11^2 + 23^2 + 7^2), inside
    # RK4's stability interval, so the round-off of the initial transform stays round-off
    shape, nu, dt, n = (24, 48, 16), 0.05, 0.05, 7
    u = inputs.abc_flow(shape)
    with Solver(shape, nu, dt, "f64") as s:
        s.set_state(u)
        s.step(n)
        got = s.get_state_spectral()
    uh0 = sn.to_spectral(u)
    R = 1 - nu * dt + (nu * dt) ** 2 / 2 - (nu * dt) ** 3 / 6 + (nu * dt) ** 4 / 24
    assert np.abs(got - uh0 * R ** n).max() < 1e-12 * np.abs(uh0).max()


def test_graph_and_eager_steps_agree_bitwise():
    uh = _field((24, 48, 16), 9, "f32")
    out = []
    for graph in (1, 0):
        with Solver((24, 48, 16), 0.01, 0.005, "f32") as s:
            s.set_option("use_graph", graph)
            s.set_state_spectral(uh)
            s.step(5)
            out.append(s.get_state_spectral())
    assert np.array_equal(out[0], out[1])


def test_unsupported_counts_and_cubic_only_features_are_refused():
    with pytest.raises(RuntimeError):
        Solver((32, 16, 48), 0.01, 1e-3, "f32")
    with Solver((32, 16, 24), 0.01, 1e-3, "f32") as s:
        with pytest.raises(RuntimeError):
            s.set_option("fft_plan", 1)
        with pytest.raises(RuntimeError):
            s.set_option("y_tile_inverse", 8)
    # equal counts give the cubic solver
    with Solver((32, 32, 32), 0.01, 1e-3, "f32") as s:
        assert s.N == 32 and s.get_option("Nz") == 32


# ----------------------------------------------------------------------------- full size

def _embed_box(src, shape, dtype, dev):
    """Half spectrum of src (3, nx, ny, nz/2+1) placed into a larger grid `shape` (same modes)."""
    _, nx, ny, h = src.shape
    NX, NY, NZ = shape
    out = torch.zeros((3, NX, NY, NZ // 2 + 1), dtype=dtype, device=dev)
    s = src.to(dev).to(dtype)
    hx, hy = nx // 2, ny // 2
    for xs, xd in ((slice(0, hx), slice(0, hx)), (slice(nx - hx, nx), slice(NX - hx, NX))):
        for ys, yd in ((slice(0, hy), slice(0, hy)), (slice(ny - hy, ny), slice(NY - hy, NY))):
            out[:, xd, yd, :h] = s[:, xs, ys, :]
    return out


@pytest.fixture(scope="module")
def big_band_case():
    """A dense divergence-free field in the 2/3 box of 128 x 128 x 64 (|k| <= (42, 42, 21)),
    its state on the 256 x 256 x 128 grid and the FP64 oracle's right-hand side there
    (nu = 0.004)."""
    nu = 0.004
    u = inputs.isotropic_spectral((128, 128, 64), seed=31, k0=12.0)
    mid = (256, 256, 128)
    u_mid = _embed_box(u, mid, torch.complex128, "cpu") * 8.0  # (256 * 256 * 128) / (128 * 128 * 64)
    ref = sn.rhs(u_mid.numpy(), sn.Grid(mid), nu)
    return u_mid, torch.from_numpy(ref), nu


@pytest.mark.parametrize("dtype,tol", [("f32", 3e-5), ("f64", 1e-12)])
def test_rhs_of_band_limited_field_on_1024x512x256_matches_oracle(big_band_case, dtype, tol):
    u_mid, ref, nu = big_band_case
    dev = "cuda"
    scale = (BIG[0] * BIG[1] * BIG[2]) / (256 * 256 * 128)  # 16
    cdt = torch.complex64 if dtype == "f32" else torch.complex128
    uh = _embed_box(u_mid, BIG, cdt, dev) * scale
    with Solver(BIG, nu, 1e-3, dtype) as s:
        s.set_state_spectral(uh)
        out = torch.empty_like(uh)
        s.rhs(out)
    expect = _embed_box(ref, BIG, torch.complex128, dev) * scale
    err = (out.to(torch.complex128) - expect).abs().max().item()
    assert err <= tol * expect.abs().max().item()


def test_rhs_invariants_of_a_full_spectrum_field_on_1024x512x256():
    nu, dev = 0.003, "cuda"
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    u = torch.randn((3,) + BIG, generator=gen, device=dev, dtype=torch.float32)
    with Solver(BIG, nu, 1e-3, "f32") as s:
        s.set_state(u)
        del u
        uh = s.get_state_spectral(torch.empty((3, BIG[0], BIG[1], BIG[2] // 2 + 1), dtype=torch.complex64, device=dev))
        out = torch.empty_like(uh)
        s.rhs(out)
    kx = torch.fft.fftfreq(BIG[0], 1.0 / BIG[0], device=dev).double()
    ky = torch.fft.fftfreq(BIG[1], 1.0 / BIG[1], device=dev).double()
    kz = torch.arange(BIG[2] // 2 + 1, device=dev).double()
    scale = float(out.abs().max())
    worst_out, worst_div, scale_nl = 0.0, 0.0, 0.0
    for x0 in range(0, BIG[0], 128):  # slabs of x keep the FP64 temporaries small
        sl = slice(x0, x0 + 128)
        KX, KY, KZ = kx[sl, None, None], ky[None, :, None], kz[None, None, :]
        inside = (3 * KX.abs() < BIG[0]) & (3 * KY.abs() < BIG[1]) & (3 * KZ < BIG[2])
        k2 = KX * KX + KY * KY + KZ * KZ
        o = out[:, sl].to(torch.complex128)
        # the projected, masked nonlinear part (white noise is not solenoidal, so the viscous
        # part is not either: the projection acts on the nonlinear term only)
        nl = o + nu * k2 * uh[:, sl].to(torch.complex128)
        worst_out = max(worst_out, (nl.abs() * (~inside)).max().item())
        scale_nl = max(scale_nl, nl.abs().max().item())
        div = KX * nl[0] + KY * nl[1] + KZ * nl[2]
        kmag = torch.sqrt(k2).clamp(min=1.0)
        worst_div = max(worst_div, (div.abs() / kmag * inside).max().item())
    assert worst_out <= 1e-6 * scale
    assert worst_div <= 1e-5 * scale_nl


def test_rk4_run_on_1024x512x256_keeps_the_energy_budget():
    dev = "cuda"
    uh = inputs.isotropic_spectral(BIG, seed=8, k0=20.0, device=dev).to(torch.complex64)
    # the field's strain time is about 1/30; samples 2 steps of 5e-4 apart keep the central
    # difference's O(dt^2) error near 1e-4 of eps
    nu, dt = 0.002, 5e-4
    with Solver(BIG, nu, dt, "f32") as s:
        s.set_state_spectral(uh)
        d = [s.diagnostics()]
        for _ in range(2):
            s.step(2)
            d.append(s.diagnostics())
    dEdt = (d[2]["energy"] - d[0]["energy"]) / (d[2]["t"] - d[0]["t"])
    assert abs(-dEdt - d[1]["dissipation"]) < 1e-3 * d[1]["dissipation"]
    assert max(x["max_div"] for x in d) < 1e-4


@pytest.mark.parametrize("dtype,bound", [("f64", 1e-12), ("f32", 1e-5)])
def test_forced_rhs_on_other_counts_matches_oracle(dtype, bound):
    from oracle import sgs_mlp

    shape, nu = (24, 48, 16), 0.01
    uh = _field(shape, 13, dtype)
    rng = np.random.default_rng(3)
    fh = sn.to_spectral(rng.standard_normal((3,) + shape)).astype(CPLX[dtype]) * 1e-3
    with Solver(shape, nu, 1e-3, dtype) as s:
        s.set_state_spectral(uh)
        s.set_forcing(fh)
        got = s.rhs()
        s.set_forcing(None)
        unforced = s.rhs()
    g = sn.Grid(shape)
    ref = sgs_mlp.rhs_forced(uh.astype(np.complex128), g, nu, fh.astype(np.complex128))
    assert rel_l2(got, ref) <= bound
    assert rel_l2(unforced, sn.rhs(uh.astype(np.complex128), g, nu)) <= bound


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_device_transforms_on_other_counts(dtype):
    shape = (32, 16, 24)
    rng = np.random.default_rng(9)
    u = rng.standard_normal((3,) + shape)
    rdt = torch.float32 if dtype == "f32" else torch.float64
    cdt = torch.complex64 if dtype == "f32" else torch.complex128
    tol = 1e-6 if dtype == "f32" else 1e-13
    with Solver(shape, 0.01, 1e-3, dtype) as s:
        ud = torch.from_numpy(u).to(rdt).cuda()
        spec = s.transform_r2c(ud, torch.empty((3, 32, 16, 13), dtype=cdt, device="cuda"))
        ref = sn.to_spectral(u)
        assert rel_l2(spec.cpu().numpy(), ref) <= tol
        back = s.transform_c2r(spec, torch.empty_like(ud))
        assert rel_l2(back.cpu().numpy(), sn.inverse(ref)) <= tol
