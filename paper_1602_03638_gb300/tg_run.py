"""Taylor-Green vortex at Re = 1600 (nu = 1/1600, dt = 1e-3) from t = 0 to T: the series of
kinetic energy E, dissipation eps = nu <|omega|^2>, enstrophy and max |div u| from the solver's
FP64 diagnostics every `every` steps (the paper's verification case, Sec. 4, with the initial
condition of the Appendix).

    python -m paper_1602_03638_gb300.tg_run --N 512 --T 20 --every 250 > tg512.json
"""

from __future__ import annotations

import argparse
import json
import sys
import time

import torch

from . import Solver, inputs


def run(N: int = 512, T: float = 20.0, dt: float = 1e-3, every: int = 250, dtype: str = "f32") -> dict:
    steps = int(round(T / dt))
    rows = []

    def record(s):
        d = s.diagnostics()
        rows.append({"t": d["t"], "E": d["energy"], "eps": d["dissipation"], "enstrophy": d["enstrophy"],
                     "max_div": d["max_div"]})

    with Solver(N, 1.0 / 1600.0, dt, dtype) as s:
        td = torch.float32 if dtype == "f32" else torch.float64
        s.set_state(inputs.taylor_green_torch(N, device="cuda", dtype=td))
        record(s)
        done = 0
        t0 = time.perf_counter()
        while done < steps:
            n = min(every, steps - done)
            s.step(n)
            done += n
            record(s)
        wall = time.perf_counter() - t0
    return {"N": N, "dtype": dtype, "nu": 1.0 / 1600.0, "dt": dt, "steps": steps, "wall_s": wall, "series": rows}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--T", type=float, default=20.0)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--every", type=int, default=250)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    a = ap.parse_args(argv)
    json.dump(run(a.N, a.T, a.dt, a.every, a.dtype), sys.stdout)
    print()
    return 0


if __name__ == "__main__":
    sys.exit(main())
