"""The Taylor-Green run module (the paper's verification case): series format, initial energy
and the energy budget dE/dt = -eps on a short, small run."""

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03638_gb300 import build

    build.build()


def test_short_taylor_green_run_series():
    from paper_1602_03638_gb300 import tg_run

    r = tg_run.run(N=32, T=0.2, dt=1e-3, every=20, dtype="f64")
    s = r["series"]
    assert r["steps"] == 200 and len(s) == 11
    assert abs(s[0]["E"] - 0.125) < 1e-15 and abs(s[-1]["t"] - 0.2) < 1e-12
    # early time: every Taylor-Green mode has |k|^2 = 3, so eps(0) = 3 nu * 2 E = 6 nu / 8
    assert abs(s[0]["eps"] - 0.75 / 1600.0) < 1e-15
    for a, b, c in zip(s, s[1:], s[2:]):
        dEdt = (c["E"] - a["E"]) / (c["t"] - a["t"])
        assert abs(-dEdt - b["eps"]) < 1e-4 * b["eps"]
    assert max(x["max_div"] for x in s) < 1e-12


def test_short_isotropic_run_compares_the_two_forms():
    """The isotropic run module on a small grid: both forms start from the same unit-energy
    field, lose energy at the rate eps (budget to 1e-3 with samples 10 steps apart), stay
    divergence-free, and the FP32 form stays within FP32 round-off of the FP64 form."""
    from paper_1602_03638_gb300 import iso_run

    r = iso_run.run(N=64, steps=40, every=10, nu=1e-2, dt=2e-3, seed=3, k0=4.0)
    for dtype in ("f64", "f32"):
        s = r["runs"][dtype]["series"]
        assert len(s) == 5 and abs(s[0]["E"] - 1.0) < 1e-6
        for a, b, c in zip(s, s[1:], s[2:]):
            dEdt = (c["E"] - a["E"]) / (c["t"] - a["t"])
            assert abs(-dEdt - b["eps"]) < 1e-3 * b["eps"]
        assert max(x["max_div"] for x in s) < (1e-4 if dtype == "f32" else 1e-12)
    assert 1e-9 < r["rel_l2_f32_vs_f64"] < 1e-5
