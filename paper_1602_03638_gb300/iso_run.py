"""Decaying isotropic turbulence: a seeded random divergence-free field with energy
spectrum E(k) ~ k^4 exp(-2 (k/k0)^2) and random phases, normalised to unit energy (the
isotropic initial condition of paper_1602_03638_gb300.inputs), advanced by RK4 steps of
Eq. NSfinal in FP32 and in FP64 from the same FP64 initial field, with the FP64
diagnostics every `every` steps and, at the end, the relative L2 distance between the two
final spectral states (the error of the FP32 form against the FP64 form).

    python -m paper_1602_03638_gb300.iso_run --N 1024 --steps 200 --every 20 > iso1024.json
    python -m paper_1602_03638_gb300.iso_run --shape 1024,512,256 --steps 200 > box.json

(--shape: a compiled grid with other point counts per direction, Nx,Ny,Nz.)

The two runs are sequential (the FP64 state of a 1024^3 run holds 137 GB of device memory);
the FP64 final state is kept on the device for the comparison.
"""

from __future__ import annotations

import argparse
import json
import sys
import time

import torch

from . import Solver, inputs


def _series(s, rows):
    d = s.diagnostics()
    rows.append({"t": d["t"], "E": d["energy"], "eps": d["dissipation"], "enstrophy": d["enstrophy"],
                 "helicity": d["helicity"], "max_div": d["max_div"]})


def _run_one(N, nu, dt, steps, every, dtype, seed, k0):
    cdt = torch.complex64 if dtype == "f32" else torch.complex128
    rows = []
    # the field is generated (in FP64, on the device) before the solver allocates its state
    uh = inputs.isotropic_spectral(N, seed=seed, k0=k0, energy=1.0, device="cuda").to(cdt)
    torch.cuda.empty_cache()
    with Solver(N, nu, dt, dtype) as s:
        st = torch.cuda.current_stream()
        s.set_stream(st)
        s.set_state_spectral(uh)
        del uh
        torch.cuda.empty_cache()
        _series(s, rows)
        done, gpu_ms = 0, 0.0
        t0 = time.perf_counter()
        while done < steps:
            n = min(every, steps - done)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            s.step(n)
            e1.record(st)
            e1.synchronize()
            gpu_ms += e0.elapsed_time(e1)
            done += n
            _series(s, rows)
        wall = time.perf_counter() - t0
        final = torch.empty(s.spec_shape, dtype=cdt, device="cuda")
        s.get_state_spectral(final)
    return {"dtype": dtype, "ms_per_step": gpu_ms / steps, "wall_s": wall, "series": rows}, final


def rel_l2(a: torch.Tensor, b: torch.Tensor, slab: int = 64) -> float:
    """||a - b|| / ||b|| over complex spectral arrays (3, Nx, Ny, Nz/2+1), in FP64, by slabs of kx."""
    num = den = 0.0
    for c in range(a.shape[0]):
        for i in range(0, a.shape[1], slab):
            x = a[c, i:i + slab].to(torch.complex128)
            y = b[c, i:i + slab].to(torch.complex128)
            num += float(((x - y).abs() ** 2).sum())
            den += float((y.abs() ** 2).sum())
    return (num / den) ** 0.5


def run(N=1024, steps: int = 200, every: int = 20, nu: float = 1e-3, dt: float = 5e-4, seed: int = 0,
        k0: float = 4.0, forms=("f64", "f32")) -> dict:
    """N: one point count or (Nx, Ny, Nz)."""
    out = {"N": N if isinstance(N, int) else list(N), "nu": nu, "dt": dt, "steps": steps, "seed": seed, "k0": k0,
           "runs": {}}
    finals = {}
    for dtype in forms:
        r, final = _run_one(N, nu, dt, steps, every, dtype, seed, k0)
        out["runs"][dtype] = r
        finals[dtype] = final
        torch.cuda.empty_cache()
    if "f32" in finals and "f64" in finals:
        out["rel_l2_f32_vs_f64"] = rel_l2(finals["f32"], finals["f64"])
        e32 = out["runs"]["f32"]["series"]
        e64 = out["runs"]["f64"]["series"]
        out["max_rel_diff_E"] = max(abs(a["E"] - b["E"]) / b["E"] for a, b in zip(e32, e64))
        out["max_rel_diff_eps"] = max(abs(a["eps"] - b["eps"]) / b["eps"] for a, b in zip(e32, e64))
        out["fp64_over_fp32_time"] = out["runs"]["f64"]["ms_per_step"] / out["runs"]["f32"]["ms_per_step"]
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--shape", default=None, help="Nx,Ny,Nz of a compiled grid with other counts per direction")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--nu", type=float, default=1e-3)
    ap.add_argument("--dt", type=float, default=5e-4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--k0", type=float, default=4.0)
    ap.add_argument("--forms", default="f64,f32")
    a = ap.parse_args(argv)
    N = tuple(int(v) for v in a.shape.split(",")) if a.shape else a.N
    json.dump(run(N, a.steps, a.every, a.nu, a.dt, a.seed, a.k0, tuple(a.forms.split(","))), sys.stdout)
    print()
    return 0


if __name__ == "__main__":
    sys.exit(main())
