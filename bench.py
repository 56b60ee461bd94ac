#!/usr/bin/env python
"""Throughput of the GB300 pseudo-spectral Navier-Stokes RK4 solver.

Metric: grid points x RK4 steps per second (higher is better), on the
Taylor-Green vortex at 512^3 in FP32 (nu = 1/1600, dt = 1e-3): the larger
Taylor-Green configuration that fits one GPU. One bench step is one full RK4
step (four right-hand-side evaluations with their transforms, projection,
viscous term and stage updates) of the whole 512^3 state, resident in HBM.

Printed on rank 0 as one JSON line, with
  value         device-timed throughput (CUDA events on the solver's stream),
                summed over all ranks (independent replicas, weak scaling)
  e2e           the same metric through the C ABI with pinned host buffers:
                state upload, K steps with a diagnostics read-back each, and
                the state download, all inside the wall-clock region
  roofline      the dominant kernel's achieved HBM bandwidth (its algorithmic
                bytes per launch over its mean CUDA-event duration) against
                the measured copy bandwidth
  step_roofline the whole step against the 132-component-volume minimum
  forms         FP64 at 512^3, FP32 and FP64 at 1024^3, both at 256^3, and the error of each
                precision against the FP64 CPU oracle at 128^3
  ensemble      128 members of mixed sizes: one graph launch per step versus
                sequential per-member launches
  cufft_comparison  the same step composed from torch.fft (cuFFT) and torch
                elementwise calls (a library comparison, not the product path)
  closure       learned subgrid closure (512^3 DNS -> 64^3): training cost,
                coarse-step cost and spectrum/dissipation error with and without it
  cpu_baseline  the FP64 CPU oracle timed on this host's cores
  clocks        nvidia-smi samples taken during the timed region

--impl reference times the CPU oracle instead (the reference arm).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid-points x RK4 steps/s (Taylor-Green 512^3 FP32; FP64 and 1024^3 in 'forms'; % HBM roofline in 'step_roofline')"
UNIT = "points*steps/s"
N_MAIN, NU, DT = 512, 1.0 / 1600.0, 1e-3
SPEC_HBM_GBS = 8000.0
# STEP_CV: the fused two-pass model of one RK4 step (x and y transforms in one sweep, 24 cv
# per stage plus 36 cv of RK4 state), in component-volumes cv = N^2 (N/2+1) complex values.
STEP_CV = 132.0
CPU_N, CPU_STEPS = 128, 8
PAPER_TG512_PTS_STEPS_PER_S = 6.2e7  # Sec. 4 verification run, 2048 Shaheen cores (context)


def pass_bytes(N, real_bytes, stages=4, rows=False, box=False):
    """Algorithmic bytes per launch of each kernel class (mean over the RK4 stages).
    N: one point count, or (Nx, Ny, Nz) for a grid with other counts per direction (then
    FV = Nx Ny (Nz/2), kc = (Nz+2)//3 planes and the rows |ky| < Ny/3 of Ny).
    rows: the state vanishes on every row (kz, ky) outside the 2/3 box (the solver's row
    flag), so the passes skip those rows (below); box: it also vanishes at |kx| >= N/3, so
    the x-stage reads and writes the RK state at the kept columns (a fraction yk) only.

    Counted from the 2/3 mask: a field-volume FV = N^2 (N/2) complex values (the stored half
    spectrum; the kz = N/2 plane is identically zero); kc = (N+2)//3 planes kz < N/3 and
    2 kc - 1 rows |ky| < N/3 carry the nonlinear term, nothing else of it is read or written.
      y_inverse  R 6 FV + W 6 FV (u and omega, every mode)
      z_pass     R 6 FV + W 3 (kc/M) FV (products kz < N/3)
      y_forward  R 3 (kc/M) FV + W 3 (kc/M)(2kc-1)/N FV (rows |ky| < N/3)
      x_stage    R 3 (kc/M)(2kc-1)/N FV (N_hat rows) + RK state + W 6 FV (u, omega)
    RK state per stage: stage 0 reads u (3) and writes u1, us (6); a middle stage reads us,
    u1, u (9) and writes u1, us (6); the last reads us, u1 (6) and writes u (3).
    With rows (a fraction zk yk of the rows kept):
      y_inverse  R 6 zk yk FV (kept rows of the planes kz < N/3) + W 6 zk FV (those planes)
      z_pass     R 6 zk FV + W 3 zk FV
      y_forward  as above
      x_stage    (R 3 + RK state + W 6) zk yk FV (kept rows only; with box the RK state x yk)
    """
    nx, ny, nz = (N,) * 3 if isinstance(N, int) else tuple(N)
    M = nz // 2
    fv = nx * ny * M * 2 * real_bytes
    kc = (nz + 2) // 3
    zk = kc / M
    yk = (2 * ((ny + 2) // 3) - 1) / ny
    rk = []
    for s_ in range(stages):
        if stages == 1:
            r, w = 3, 3
        elif s_ == 0:
            r, w = 3, 6
        elif s_ < stages - 1:
            r, w = 9, 6
        else:
            r, w = 6, 3
        rk.append(r + w)
    rk_mean = sum(rk) / len(rk)
    if rows:
        xk = (2 * ((nx + 2) // 3) - 1) / nx if box else 1.0
        return {"y_inverse": 6.0 * zk * (yk + 1.0) * fv, "z_pass": 9.0 * zk * fv,
                "y_forward": (3.0 * zk + 3.0 * zk * yk) * fv, "x_stage": (3.0 + rk_mean * xk + 6.0) * zk * yk * fv}
    return {"y_inverse": 12.0 * fv, "z_pass": (6.0 + 3.0 * zk) * fv, "y_forward": (3.0 * zk + 3.0 * zk * yk) * fv,
            "x_stage": (3.0 * zk * yk + rk_mean + 6.0) * fv}


def truncated_step_cv(N):
    """The 2-pass step model (STEP_CV) for a state that vanishes outside the 2/3 box, in cv:
    per stage the xy inverse reads the state's box modes (3 b3) and writes the planes kz < N/3
    (6 zk), the z-pass reads those (6 zk) and writes the products there (3 zk), the xy forward
    reads them (3 zk), the viscous term reads the box modes (3 b3); the RK traffic (36 cv) only
    touches the box modes (b3 = the box's share of the half spectrum)."""
    M = N // 2
    kc = (N + 2) // 3
    zk = kc / (M + 1)
    yk = (2 * kc - 1) / N
    b3 = zk * yk * yk
    return 4.0 * (6.0 * b3 + 18.0 * zk) + 36.0 * b3


def cv_bytes(N, real_bytes):
    nx, ny, nz = (N,) * 3 if isinstance(N, int) else tuple(N)
    return nx * ny * (nz // 2 + 1) * 2 * real_bytes


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons of one GPU, sampled every 200 ms."""

    FIELDS = ["index", "uuid", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid: str, index: int):
        self.uuid, self.index = uuid, index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [[p.strip() for p in line.split(",")] for line in out.strip().splitlines()]
        rows = [r for r in rows if len(r) == len(self.FIELDS)]
        mine = [r for r in rows if self.uuid and self.uuid in r[1]] or [r for r in rows if r[0] == str(self.index)]
        sm, mx, reasons = [], [], set()
        for r in mine:
            try:
                sm.append(float(r[2]))
                mx.append(float(r[3]))
            except ValueError:
                continue
            for name, v in zip(self.REASONS, r[5:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(torch, dev):
    try:
        return str(torch.cuda.get_device_properties(dev).uuid).replace("GPU-", "")
    except Exception:
        return ""


def ncu_traffic(kernel, N, dtype):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current sources."""
    from paper_1602_03638_gb300 import build

    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = build.kernel_digest()
    with open(path) as f:
        for line in f:
            tok = line.split()
            if len(tok) >= 6 and tok[0] == "traffic":
                _, k, n, dt, b, dig = tok[:6]
                if k == kernel and int(n) == N and dt == dtype and dig == digest:
                    return float(b)
    return None


def oracle_sample(N, steps, nu, dt):
    """Times `steps` RK4 steps of the FP64 oracle on Taylor-Green at N^3; returns (seconds, state, cores)."""
    from oracle import spectral_ns as sn
    from paper_1602_03638_gb300 import inputs

    uh = inputs.taylor_green_spectral(N).numpy()
    g = sn.Grid(N)
    t0 = time.perf_counter()
    for _ in range(steps):
        uh = sn.rk4_step(uh, g, nu, dt)
    return time.perf_counter() - t0, uh, sn.WORKERS


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import spectral_ns as sn
    from paper_1602_03638_gb300 import inputs

    N = CPU_N
    uh = inputs.taylor_green_spectral(N).numpy()
    g = sn.Grid(N)
    for _ in range(args.warmup):
        uh = sn.rk4_step(uh, g, NU, DT)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        uh = sn.rk4_step(uh, g, NU, DT)
    secs = time.perf_counter() - t0
    value = N ** 3 * args.steps / secs
    sample = (f"bounded sample of the Taylor-Green workload: one RK4 step of the FP64 oracle at {N}^3 per bench "
              f"step (nu=1/1600, dt=1e-3; a 512^3 oracle step takes about a minute), scipy.fft workers={sn.WORKERS}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (Taylor-Green initial condition)",
        "config": reference_config(world, N),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": sn.WORKERS, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main_config(world, N=N_MAIN):
    return {"workload": f"taylor_green_{N}_f32", "model": "pseudo-spectral NS, RK4, 2/3 dealiasing", "N": N,
            "nu": NU, "dt": DT, "global_batch": world, "seq_len": None, "parallelism": f"replicas{world}",
            "l2": "no flush needed: every pass moves 1.8-5 GB, > 129 MB L2"}


def reference_config(world, N):
    """The reference arm's own workload: Taylor-Green at N^3 in FP64 (the GPU arm's 512^3 FP32
    case is too large for the CPU oracle within a bench run); named as such."""
    return {"workload": f"taylor_green_{N}_f64", "model": "pseudo-spectral NS, RK4, 2/3 dealiasing (CPU oracle)",
            "N": N, "nu": NU, "dt": DT, "global_batch": 1, "seq_len": None, "parallelism": "cpu",
            "sample_of": f"taylor_green_{N_MAIN}_f32"}


def time_steps(torch, s, st, steps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        s.step(1)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_form(torch, Solver, inputs, N, dtype, warm, steps):
    cdt = torch.complex64 if dtype == "f32" else torch.complex128
    with Solver(N, NU, DT, dtype) as s:
        st = torch.cuda.current_stream()
        s.set_stream(st)
        s.set_state_spectral(inputs.taylor_green_spectral(N, device="cuda", dtype=cdt))
        pruned = s.get_option("rows_vanish") == 1.0 and s.get_option("prune_rows") == 1.0
        for _ in range(warm):
            s.step(1)
        torch.cuda.synchronize()
        ms = time_steps(torch, s, st, steps) / steps
    rb = 4 if dtype == "f32" else 8
    model_ms = STEP_CV * cv_bytes(N, rb) / (measured_peaks()[0] * 1e9) * 1e3
    out = {"N": N, "dtype": dtype, "ms_per_step": ms, "value": N ** 3 / (ms * 1e-3), "steps": steps, "rows_pruned": pruned,
           "hbm_roofline_frac_of_measured": model_ms / ms,
           "truncated_state_roofline_frac_of_measured": model_ms * truncated_step_cv(N) / STEP_CV / ms}
    if dtype == "f64":
        # FP64 arithmetic bound: ~270 N^3 log2 N flops per RK4 step (36 scalar 3D transforms,
        # radix-2 count, a third per direction) against the FP64 FMA rate measured on this GPU
        # (dns_measure_fp64_peak). Where the state vanishes outside the 2/3 box the passes
        # transform only the lines that are not identically zero: per stage the 6 inverse and
        # 3 forward transforms keep all z-lines, the y-lines of the planes kz < N/3 (zk) and
        # the x-lines of the rows inside the box (zk yk): a factor (1 + zk + zk yk) / 3.
        flops_full = 270.0 * N ** 3 * math.log2(N)
        kc = (N + 2) // 3
        zk, yk = kc / (N // 2), (2 * kc - 1) / N
        flops = flops_full * ((1.0 + zk + zk * yk) / 3.0 if pruned else 1.0)
        peak = fp64_peak_tflops() * 1e12
        out["roofline"] = {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": peak / 1e12,
                           "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / peak, "flops_per_step": flops,
                           "flops_per_step_full_transforms": flops_full, "rows_pruned": pruned,
                           "peak_kind": "measured (dependent-FMA probe, CUDA events)"}
    return out


_FP64_PEAK = None


def fp64_peak_tflops():
    global _FP64_PEAK
    if _FP64_PEAK is None:
        import ctypes

        from paper_1602_03638_gb300 import _lib

        v = ctypes.c_double()
        _lib.check(_lib.lib().dns_measure_fp64_peak(ctypes.byref(v)), "dns_measure_fp64_peak")
        _FP64_PEAK = float(v.value)
    return _FP64_PEAK


def run_grids(torch, Solver, inputs, shape=(1024, 512, 256), warm=3, steps=10):
    """A grid with other point counts per direction (1024 x 512 x 256, as many points as
    512^3; generic passes): step time in both precisions, and the FP32 kernel classes
    against their algorithmic bytes (pass_bytes) at the measured HBM peak."""
    out = {"shape": list(shape), "steps": steps, "forms": []}
    peak, kind = measured_peaks()
    for dtype in ("f32", "f64"):
        cdt = torch.complex64 if dtype == "f32" else torch.complex128
        rb = 4 if dtype == "f32" else 8
        with Solver(shape, NU, DT, dtype) as s:
            st = torch.cuda.current_stream()
            s.set_stream(st)
            uh = inputs.isotropic_spectral(shape, seed=1, k0=8.0, device="cuda").to(cdt)
            s.set_state_spectral(uh)
            del uh
            for _ in range(warm):
                s.step(1)
            torch.cuda.synchronize()
            n = steps if dtype == "f32" else max(2, steps // 5)
            ms = time_steps(torch, s, st, n) / n
            form = {"dtype": dtype, "ms_per_step": ms, "value": shape[0] * shape[1] * shape[2] / (ms * 1e-3),
                    "hbm_roofline_frac_of_measured": STEP_CV * cv_bytes(shape, rb) / (peak * 1e9) / (ms * 1e-3)}
            if dtype == "f32":
                prof = s.profile_steps(n)
                kb = pass_bytes(shape, rb, rows=s.get_option("rows_vanish") == 1.0,
                                box=s.get_option("box_vanish") == 1.0)
                form["kernels"] = {k: {"ms_per_launch": t / c, "launches": c,
                                       "achieved_gbs": kb[k] / (t / c * 1e-3) / 1e9,
                                       "frac_of_peak": kb[k] / (t / c * 1e-3) / 1e9 / peak}
                                   for k, (t, c) in prof.items()}
            out["forms"].append(form)
    out["peak_gbs"], out["peak_kind"] = peak, kind
    return out


def run_integrators(torch, Solver, inputs, N=512, warm=3, steps=10):
    """Taylor-Green N^3 FP32 step time of each explicit RK scheme of the integrator option;
    a stage costs the same four passes in every scheme, so ms per stage is the comparison."""
    stages = {"euler": 1, "heun": 2, "midpoint": 2, "rk4": 4}
    out = {}
    for scheme, ns in stages.items():
        with Solver(N, NU, DT, "f32", integrator=scheme) as s:
            st = torch.cuda.current_stream()
            s.set_stream(st)
            s.set_state_spectral(inputs.taylor_green_spectral(N, device="cuda", dtype=torch.complex64))
            for _ in range(warm):
                s.step(1)
            torch.cuda.synchronize()
            ms = time_steps(torch, s, st, steps) / steps
        out[scheme] = {"stages": ns, "ms_per_step": ms, "ms_per_stage": ms / ns}
    return {"N": N, "dtype": "f32", "steps": steps, "schemes": out}


def run_ensemble(torch, np, steps=10):
    """128 independent members (32 each of 32^3, 48^3, 64^3, 96^3), FP32, isotropic initial
    fields with k0 drawn from U[2, 6] per member: one graph launch per ensemble step (schedule
    chosen by dns_ensemble_tune: equal-size members batched into shared launches, or per-member
    launches on parallel branches) versus one dns_step per member (sequential launches)."""
    from paper_1602_03638_gb300 import Ensemble, inputs

    sizes = [32, 48, 64, 96]
    Ns = [sizes[i % 4] for i in range(128)]
    rng = np.random.default_rng(2024)
    k0s = rng.uniform(2.0, 6.0, size=len(Ns))
    nu, dt = 5e-3, 2e-3
    with Ensemble(Ns, [nu] * len(Ns), [dt] * len(Ns), "f32") as ens:
        for i, (m, N) in enumerate(zip(ens.members, Ns)):
            uh = inputs.isotropic_spectral(N, seed=i + 1, k0=float(k0s[i]), device="cuda").to(torch.complex64)
            m.set_state_spectral(uh)
        best = ens.tune()
        ens.step(2)
        ens.synchronize()
        graph = ens.time_steps(steps) * 1e-3 / steps
        for m in ens.members:  # warm the per-member graphs
            m.step(1)
        ens.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            for m in ens.members:
                m.step(1)
        ens.synchronize()
        sequential = (time.perf_counter() - t0) / steps
        pts = sum(N ** 3 for N in Ns)
    model = sum(STEP_CV * cv_bytes(N, 4) for N in Ns)
    peak, kind = measured_peaks()
    return {"members": len(Ns), "sizes": {str(n): Ns.count(n) for n in sizes}, "dtype": "f32", "nu": nu, "dt": dt,
            "schedule": best, "graph_ms_per_step": 1e3 * graph, "sequential_ms_per_step": 1e3 * sequential,
            "speedup": sequential / graph, "points_steps_per_s": pts / graph,
            "roofline": {"model_bytes_per_step": model, "achieved_GBps": model / graph / 1e9, "peak": peak,
                         "frac": model / graph / 1e9 / peak, "peak_kind": kind,
                         "what": "132-cv step model summed over the members / device-timed step"},
            "timing": "graph: CUDA events on the ensemble stream around K graph launches; sequential: host "
                      "wall clock around K rounds of per-member dns_step calls + synchronize"}


def run_cufft_comparison(torch, N=N_MAIN, steps=3, warm=2):
    """Library comparison (not the product path): the same RK4 step of the Taylor-Green case
    written with torch.fft (cuFFT) transforms and torch elementwise operations in FP32 on the
    GPU, the way the paper's NumPy code composes library calls; CUDA-event time per step."""
    dev = "cuda"
    k = torch.fft.fftfreq(N, 1.0 / N, device=dev)
    kx, ky, kz = k[:, None, None], k[None, :, None], torch.arange(N // 2 + 1, device=dev, dtype=k.dtype)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2inv = torch.where(k2 == 0, torch.zeros_like(k2), 1.0 / k2)
    mask = ((3 * kx.abs() < N) & (3 * ky.abs() < N) & (3 * kz.abs() < N)).to(torch.float32)

    def rhs(uh):
        u = torch.fft.irfftn(uh, s=(N, N, N), dim=(1, 2, 3))
        wh = torch.stack([1j * (ky * uh[2] - kz * uh[1]), 1j * (kz * uh[0] - kx * uh[2]), 1j * (kx * uh[1] - ky * uh[0])])
        w = torch.fft.irfftn(wh, s=(N, N, N), dim=(1, 2, 3))
        del wh
        c = torch.stack([u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]])
        del u, w
        nh = torch.fft.rfftn(c, dim=(1, 2, 3)) * mask
        del c
        p = (kx * nh[0] + ky * nh[1] + kz * nh[2]) * k2inv
        nh[0] -= kx * p
        nh[1] -= ky * p
        nh[2] -= kz * p
        return nh - NU * k2 * uh

    a, b = (1 / 6, 1 / 3, 1 / 3, 1 / 6), (0.5, 0.5, 1.0)

    def step(uh):
        u0, u1 = uh, uh.clone()
        for s in range(4):
            d = rhs(uh)
            if s < 3:
                uh = u0 + (b[s] * DT) * d
            u1 += (a[s] * DT) * d
        return u1

    from paper_1602_03638_gb300 import inputs

    uh = torch.fft.rfftn(inputs.taylor_green_torch(N, device=dev, dtype=torch.float32), dim=(1, 2, 3))
    for _ in range(warm):
        uh = step(uh)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        uh = step(uh)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    energy = float(0.5 * (torch.fft.irfftn(uh, s=(N, N, N), dim=(1, 2, 3)) ** 2).sum(0).mean())
    out = {"what": "torch.fft (cuFFT) + torch elementwise RK4 step, FP32, same workload", "N": N,
           "ms_per_step": ms, "value": N ** 3 / (ms * 1e-3), "steps": steps, "energy_after": energy,
           "steps_taken": warm + steps}
    del uh
    torch.cuda.empty_cache()
    return out


def run_closure_share(torch, N=64, steps=50):
    """Device time of the coarse 64^3 FP32 step with the closure inside the step graph, against
    the same step without it, and of the network forward alone on the N^3 features (CUDA
    events): the kernel-time share of the network (tcgen05 inference) in the modelled step."""
    import numpy as np

    from paper_1602_03638_gb300 import Solver, inputs, sgs

    st = torch.cuda.current_stream()

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(n):
            fn()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / n

    net = sgs.MLP(seed=0)
    X = torch.randn(10, N ** 3, device="cuda", dtype=torch.float32)
    T = torch.randn(6, N ** 3, device="cuda", dtype=torch.float32) * 0.01
    net.set_normalisation(X, T)
    out = {"N": N}
    with Solver(N, 2e-3, 4e-3, "f32") as s:
        s.set_stream(st)
        s.set_state_spectral(inputs.isotropic_spectral(N, seed=5, k0=4.0, device="cuda").to(torch.complex64))
        s.step(3)
        out["step_ms_no_model"] = timed(lambda: s.step(1), steps)
        s.set_closure(net)
        s.step(3)
        out["step_ms_model"] = timed(lambda: s.step(1), steps)
        s.set_closure(None)
    out["mlp_forward_ms"] = timed(lambda: net.forward(X), steps)
    out["mlp_share_of_model_step"] = out["mlp_forward_ms"] / out["step_ms_model"]
    out["closure_overhead_ratio"] = out["step_ms_model"] / out["step_ms_no_model"]
    net.close()
    return out


def run_closure():
    """Learned subgrid closure: 512^3 FP32 DNS (this solver) -> box filter width 2 pi/64 -> 64^3,
    BF16 network trained on the GPU, coarse runs with and without it against the filtered DNS over
    two large-eddy turnover times."""
    from paper_1602_03638_gb300 import sgs

    r = sgs.closure_experiment(Nf=512, Nc=64, nu=2e-3, dt_f=1e-3, dt_c=4e-3, k0=4.0, t_dev=0.3, t_run=None,
                               iters=600, batch=65536)
    keep = ("Nf", "Nc", "nu", "dt_fine", "dt_coarse", "t_dev", "t_run", "eddy", "training_points", "train_s",
            "coarse_ms_per_step_no_model",
            "coarse_ms_per_step_model", "dns_ms_per_step", "checkpoints")
    out = {k: r[k] for k in keep}
    out["final_train_loss"] = r["train_loss"][-1][1]
    return out


def combine_replicas(ms_local, steps, points, dist=None, device="cpu"):
    """Replicas only: every rank steps its own independent copy of the workload. Returns the
    maximum over ranks of the timed-region duration and the whole-job throughput (all ranks'
    grid points x steps over that maximum)."""
    import torch

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms_max = float(t.item())
    return ms_max, world * points * steps / (ms_max * 1e-3)


def step_traffic(N, dtype, classes):
    """DRAM bytes per RK4 step from the per-launch ncu traffic of the schedule's kernel classes
    (each launched once per stage, 4 stages), or None."""
    parts = [ncu_traffic(k, N, dtype) for k in classes]
    return None if any(p is None for p in parts) else 4.0 * sum(parts)


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    from paper_1602_03638_gb300 import Solver, build, inputs

    build.build()
    dev = local if torch.cuda.device_count() > local else 0
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))

    def barrier():
        if dist is not None:
            dist.barrier()

    N, dtype = args.N, "f32"
    peak, peak_kind = measured_peaks()
    s = Solver(N, NU, DT, dtype)
    st = torch.cuda.current_stream()
    s.set_stream(st)
    # the Taylor-Green vortex from its exact Fourier coefficients: the state vanishes outside
    # the 2/3 box, so the passes skip those rows (set from FP32 mesh values, the forward
    # transform would leave rounding residue there and the full transforms would run)
    s.set_state_spectral(inputs.taylor_green_spectral(N, device="cuda", dtype=torch.complex64))
    rows = s.get_option("rows_vanish") == 1.0 and s.get_option("prune_rows") == 1.0
    box = rows and s.get_option("box_vanish") == 1.0
    for _ in range(args.warmup):
        s.step(1)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_uuid(torch, dev), dev)
    ms = time_steps(torch, s, st, args.steps)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier()
    ms_max, value = combine_replicas(ms, args.steps, N ** 3, dist, "cuda")
    ms_step = ms_max / args.steps

    # per-kernel CUDA-event timing of the same workload (eager launches)
    prof = s.profile_steps(args.steps)
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    cvb = cv_bytes(N, 4)
    kb = pass_bytes(N, 4, rows=rows, box=box)
    achieved = kb[dom] / (dom_ms * 1e-3) / 1e9
    kernels = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": v[0] / sum(x[0] for x in prof.values()),
                   "algorithmic_bytes_per_launch": kb[k],
                   "algorithmic_GBps": kb[k] / (v[0] / v[1] * 1e-3) / 1e9} for k, v in prof.items()}
    full = None
    if rows and not args.no_extras:
        # the same workload with the full transforms (option prune_rows = 0): same results
        s.set_option("prune_rows", 0)
        s.step(2)
        torch.cuda.synchronize()
        fms = time_steps(torch, s, st, args.steps) / args.steps
        fprof = s.profile_steps(max(1, args.steps // 2))
        fkb = pass_bytes(N, 4)
        full = {"ms_per_step": fms, "value": N ** 3 / (fms * 1e-3),
                "step_roofline_frac_of_measured": STEP_CV * cvb / (fms * 1e-3) / 1e9 / peak,
                "kernels": {k: {"ms_per_launch": v[0] / v[1], "algorithmic_bytes_per_launch": fkb[k],
                                "algorithmic_GBps": fkb[k] / (v[0] / v[1] * 1e-3) / 1e9} for k, v in fprof.items()}}
    s.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    step_bytes = STEP_CV * cvb
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_TG512_PTS_STEPS_PER_S, "dtype": "f32",
        "data": "synthetic (Taylor-Green initial condition from its exact Fourier coefficients, on device)",
        "config": main_config(world, N),
        "gpu_launches": 4 * len(prof) * args.steps,  # kernels per RK4 stage x 4 stages x steps
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": ncu_traffic(dom, N, dtype),
                     "algorithmic_bytes_per_launch": kb[dom]},
        "step_roofline": {"model_bytes_per_step": step_bytes, "achieved_GBps": step_bytes / (ms_step * 1e-3) / 1e9,
                          "frac_of_measured": step_bytes / (ms_step * 1e-3) / 1e9 / peak,
                          "frac_of_spec_8TBps": step_bytes / (ms_step * 1e-3) / 1e9 / SPEC_HBM_GBS,
                          # the 3-pass model (x, y and z transforms each a separate HBM sweep, 204 cv
                          # per step): what the plane blocking of the 132-cv model would buy (like the
                          # 132-cv model it counts the full transforms, which a pruned step skips)
                          "frac_of_measured_3pass_model":
                              None if rows else 204.0 * cvb / (ms_step * 1e-3) / 1e9 / peak,
                          "models": "model_bytes_per_step (132 cv) and the 3-pass model count the full "
                                    "transforms; with rows_pruned the passes skip the lines a truncated state "
                                    "leaves zero, whose own 2-pass minimum is the truncated-state model",
                          # the same 2-pass model for a state that vanishes outside the 2/3 box
                          # (the one this workload has): the minimum the pruned passes could reach
                          "truncated_state_model_bytes_per_step": truncated_step_cv(N) * cvb,
                          "frac_of_measured_truncated_state_model":
                              truncated_step_cv(N) * cvb / (ms_step * 1e-3) / 1e9 / peak,
                          "rows_pruned": rows,
                          # DRAM bytes the schedule's passes move per step (ncu, profiles/)
                          "dram_bytes_per_step_measured": step_traffic(N, dtype, list(prof))},
        "kernels": kernels,
        "clocks": clocks,
    }
    if full is not None:
        line["full_transforms"] = full

    if not args.no_extras:
        # end to end through the public API with pinned host buffers
        with Solver(N, NU, DT, dtype) as s2:
            host_uh = inputs.taylor_green_spectral(N, dtype=torch.complex64).pin_memory()
            out_u = torch.empty((3, N, N, N), dtype=torch.float32).pin_memory()
            s2.set_state_spectral(host_uh)
            s2.step(1)
            s2.diagnostics()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2.set_state_spectral(host_uh)
            for _ in range(args.steps):
                s2.step(1)
                d = s2.diagnostics()
            s2.get_state(out_u)
            e2e_s = time.perf_counter() - t0
            sh, ph = host_uh.numel() * 8, 3 * N ** 3 * 4
            line["e2e"] = {"value": N ** 3 * args.steps / e2e_s, "unit": UNIT,
                           "h2d_bytes_per_step": sh / args.steps,
                           "d2h_bytes_per_step": (ph + args.steps * 5 * 8) / args.steps,
                           "final_energy": d["energy"],
                           "what": "upload of the spectral state (pinned), K steps with a diagnostics read-back "
                                   "each, download of the physical state (pinned)"}
        # precision forms
        forms = [run_form(torch, Solver, inputs, 512, "f64", 2, 3), run_form(torch, Solver, inputs, 1024, "f32", 2, 3),
                 run_form(torch, Solver, inputs, 1024, "f64", 1, 2),
                 run_form(torch, Solver, inputs, 256, "f32", 3, 20), run_form(torch, Solver, inputs, 256, "f64", 2, 5)]
        # CPU oracle baseline and error of each GPU precision against it
        secs, ref, cores = oracle_sample(CPU_N, CPU_STEPS, NU, DT)
        errs = {}
        for dt_ in ("f32", "f64"):
            with Solver(CPU_N, NU, DT, dt_) as s3:
                s3.set_state_spectral(inputs.taylor_green_spectral(CPU_N).numpy().astype(
                    np.complex64 if dt_ == "f32" else np.complex128))
                s3.step(CPU_STEPS)
                got = s3.get_state_spectral()
            errs[dt_] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        line["forms"] = forms
        line["integrators"] = run_integrators(torch, Solver, inputs)
        line["grids"] = run_grids(torch, Solver, inputs)
        line["ensemble"] = run_ensemble(torch, np)
        line["cufft_comparison"] = run_cufft_comparison(torch)
        line["closure"] = run_closure()
        line["closure"]["in_graph"] = run_closure_share(torch)
        line["error_vs_oracle"] = {"case": f"Taylor-Green {CPU_N}^3, {CPU_STEPS} RK4 steps, nu=1/1600, dt=1e-3",
                                   "rel_l2_f32": errs["f32"], "rel_l2_f64": errs["f64"]}
        line["cpu_baseline"] = {"value": CPU_N ** 3 * CPU_STEPS / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"Taylor-Green {CPU_N}^3 FP64, {CPU_STEPS} RK4 steps (bounded sample of the "
                                          f"Taylor-Green workload), scipy.fft workers={cores}"}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, forms and the CPU baseline")
    ap.add_argument("--N", type=int, default=N_MAIN, help="grid size of the timed workload (profiling runs only)")
    ap.add_argument("--closure-only", action="store_true",
                    help="print only the in-graph closure timing at 64^3 (run_closure_share) and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.closure_only:
        import torch

        from paper_1602_03638_gb300 import build

        build.build()
        print(json.dumps(run_closure_share(torch)), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
