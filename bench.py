"""Benchmark of the GB300 fractional-step Navier-Stokes step (FSEI fluid hot
path, arXiv 2103.15187 Sec. 2.1 / Sec. 3.1).

Workload: 256^3 wall-bounded channel (periodic x, y of lengths 2 pi, pi;
no-slip walls at z = +-1, tanh-stretched z with factor 2), Poiseuille profile
plus a seeded solenoidal perturbation (RMS 0.1, horizontal wavenumbers 1-8),
Re = 2000, CFL 0.5, uniform drive f_x = 2/Re.  The headline is the mixed
precision step (FP32 fields; FP64 near-zero Poisson modes and reductions) in
Mcell-updates/s; the FP64 step, the mixed-vs-FP64 error after 100 steps, the
per-kernel HBM roofline, an end-to-end number with host buffers and the CPU
oracle are reported beside it.

One JSON line on stdout (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica (the step has no sharding); value = all cells advanced by
all ranks / max-over-ranks time.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(nx=256, ny=256, nz=256, lx=2 * np.pi, ly=np.pi, stretch=2.0,
                re=2000.0, cfl=0.5, kmin=1.0, kmax=8.0, rms=0.1, seed=2)
FIELDS = ("u", "v", "w", "p", "hu", "hv", "hw")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------- roofline ----
def algorithmic_words(nx, ny, nz, with_force):
    """Words per cell each kernel must move (read + write once), with the
    spectrum counted at its true size (nx/2+1) x ny x nz complex."""
    spec = 2.0 * (nx // 2 + 1) / nx
    return {
        "rhs_x (RHS + x sweep)": 7 + (3 if with_force else 0) + 6,
        "sweep_y": 6,
        "sweep_z (+ u*)": 9,
        "rfft_x (div + x R2C)": 3 + spec,
        "fft_y (forward)": 2 * spec,
        "poisson_z (+ exact modes)": 2 * spec,
        "fft_y (inverse)": 2 * spec,
        "irfft_x (x C2R)": spec + 1,
        "project (+ p update, stats)": 9,
    }


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
# of the dominant kernel, from an ncu --set full capture of the 256^3
# channel workload; reported only for that workload and that kernel build
MEASURED_TRAFFIC = {
    "rhs_x (RHS + x sweep)": {"bytes": 826.5e6, "cells": 256 ** 3,
                              "kernel": "k_rhs_x_row<float, 4, 64>"},
}

# FP64 instructions of one FP64 step per cell (DFMA + DADD + DMUL thread
# instructions, the CFL pre-pass excluded), from one ncu capture of the FP64
# step on a 128^3 channel (the count per cell does not depend on the size).
# The FP64 step is bound by the FP64 pipe: its peak is 2 FP64 thread
# instructions per clock per SM (1.25 TFLOP/s of DFMA nominal), times 152
# SMs at the 2070 MHz maximum clock.
FP64_INSTR_PER_CELL = 342.6
FP64_PEAK_GINST = 2 * 152 * 2.070


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi samples (every 50 ms) during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # wait for nvidia-smi's first sample, then keep only samples taken
            # from here on (the timed region starts right after)
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.02)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- GPU arm -----
def make_case():
    from paper_2103_15187_gb300 import inputs
    w = WORKLOAD
    return inputs.case_channel(w["nx"], w["ny"], w["nz"], w["lx"], w["ly"], w["stretch"],
                               w["re"], w["cfl"], 100, w["kmin"], w["kmax"], 0.0, w["rms"],
                               w["seed"])


def device_state(case, dtype):
    import torch
    z = np.zeros_like(case.u)
    src = {"u": case.u, "v": case.v, "w": case.w, "p": case.p, "hu": z, "hv": z, "hw": z}
    st = {k: torch.tensor(src[k], dtype=dtype, device="cuda") for k in FIELDS}
    st["have_prev_h"] = 0
    return st


def run_gpu_arm(args, rank, world):
    import torch
    from paper_2103_15187_gb300 import fsei
    import __graft_entry__
    __graft_entry__.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    case = make_case()
    prm = dict(re=case.re, dt=case.dt, cfl=case.cfl, fconst=case.fconst)
    cells = case.cells
    K, W = args.steps, args.warmup
    dist = None
    if world > 1:
        import torch.distributed as dist

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    results = {}
    for prec_name, prec, dtype in (("mixed", fsei.FSEI_MIXED, torch.float32),
                                   ("fp64", fsei.FSEI_FP64, torch.float64)):
        if prec_name == "fp64" and args.no_fp64:
            continue
        grid = fsei.Grid(case.nx, case.ny, case.nz, case.lx, case.ly, zbc=case.zbc,
                         lz=case.lz, stretch=case.stretch, prec=prec)
        if args.schedule and prec_name == "mixed":
            grid.set_schedule(json.loads(args.schedule))
            sched = grid.schedule
        else:
            sched = grid.autotune() if not args.no_autotune else grid.schedule
        st = device_state(case, dtype)
        stream = torch.cuda.current_stream()
        if W > 0:
            fsei.step(grid, st, None, nsteps=W, stats=False, **prm)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            e0.record(stream)
            fsei.step(grid, st, None, nsteps=K, stats=False, **prm)
            e1.record(stream)
            barrier()
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(ms)
        stats = fsei.step(grid, st, None, nsteps=0, **prm)
        res = {"ms_total": ms, "ms_per_step": ms / K, "cells": cells,
               "mcups": cells * K * world / (ms * 1e-3) / 1e6, "clocks": clk.summary(),
               "last_stats": stats}
        # per-kernel device time over K more steps (event pairs on the stream)
        fsei.set_kernel_timing(grid, True)
        fsei.step(grid, st, None, nsteps=K, stats=False, **prm)
        kt = fsei.kernel_times(grid)
        fsei.set_kernel_timing(grid, False)
        res["kernels"] = kt
        res["schedule"] = sched
        results[prec_name] = (res, grid, st)
        log("%s: %.3f ms/step, %.1f Mcell/s" % (prec_name, res["ms_per_step"], res["mcups"]))

    # mixed vs FP64 error after 100 steps from the same initial state
    err = None
    if not args.no_fp64 and args.error_steps > 0:
        outs = {}
        for prec_name, prec, dtype in (("mixed", fsei.FSEI_MIXED, torch.float32),
                                       ("fp64", fsei.FSEI_FP64, torch.float64)):
            grid = results[prec_name][1]
            st = device_state(case, dtype)
            fsei.step(grid, st, None, nsteps=args.error_steps, stats=False, **prm)
            torch.cuda.synchronize()
            outs[prec_name] = {k: st[k].double() for k in ("u", "v", "w")}
        num = sum(float(torch.linalg.vector_norm(outs["mixed"][k] - outs["fp64"][k]) ** 2)
                  for k in "uvw")
        den = sum(float(torch.linalg.vector_norm(outs["fp64"][k]) ** 2) for k in "uvw")
        err = (num / den) ** 0.5
        log("mixed vs fp64 velocity rel L2 after %d steps: %.3e" % (args.error_steps, err))

    # end to end through the public API with host buffers: per step the
    # state goes host -> device, one step runs, the new state comes back
    mixed_res, mgrid, _ = results["mixed"]
    e2e = None
    if args.e2e_steps > 0:
        host = {k: torch.empty((case.nz, case.ny, case.nx), dtype=torch.float32).pin_memory()
                for k in FIELDS}
        dst = device_state(case, torch.float32)
        for k in FIELDS:
            host[k].copy_(dst[k].cpu())
        stream = torch.cuda.current_stream()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        have = 0
        for _ in range(args.e2e_steps):
            for k in FIELDS:
                dst[k].copy_(host[k], non_blocking=True)
            dst["have_prev_h"] = have
            fsei.step(mgrid, dst, None, nsteps=1, stats=False, **prm)
            have = 1
            for k in FIELDS:
                host[k].copy_(dst[k], non_blocking=True)
        e1.record(stream)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        nbytes = sum(host[k].numel() * 4 for k in FIELDS)
        e2e = {"value": cells * args.e2e_steps * world / (ms * 1e-3) / 1e6,
               "unit": "Mcell-updates/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps}
    return case, results, err, e2e


def run_ensemble(args):
    """64 independent boxes of uneven sizes (32^3, 64^3, 96x96x128, 128x128x192),
    FP32 fields, one batched call per K steps (CUDA graph replayed per step),
    against the same boxes advanced one after another with fsei_step."""
    import torch
    from paper_2103_15187_gb300 import fsei, inputs
    cases = inputs.case_ensemble(args.ensemble_boxes, steps=args.steps)
    boxes = [dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                  stretch=c.stretch, prec=fsei.FSEI_MIXED) for c in cases]
    batch = fsei.Batch(boxes)
    if not args.no_autotune:
        batch.autotune()
    states = [device_state(c, torch.float32) for c in cases]
    params = [dict(re=c.re, dt=c.dt, cfl=c.cfl, fconst=c.fconst) for c in cases]
    cells = sum(c.cells for c in cases)
    K = args.ensemble_steps
    # two warm-up calls: the first captures the graphs of a fresh state, the
    # second those of a state with history; the timed call reuses the latter
    fsei.batch_step(batch, states, None, params, nsteps=2, stats=False)
    fsei.batch_step(batch, states, None, params, nsteps=2, stats=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fsei.batch_step(batch, states, None, params, nsteps=K, stats=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = fsei.batch_step(batch, states, None, params, nsteps=0, stats=True)
    # the same boxes one after another (no graph, no overlap)
    grids = [fsei.Grid(**b) for b in boxes]
    solo = [device_state(c, torch.float32) for c in cases]
    for g, s, p in zip(grids, solo, params):
        fsei.step(g, s, None, nsteps=2, stats=False, **p)
    torch.cuda.synchronize()
    e0.record(stream)
    for g, s, p in zip(grids, solo, params):
        fsei.step(g, s, None, nsteps=K, stats=False, **p)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    return {"value": round(cells * K / (ms * 1e-3) / 1e6, 2), "unit": "Mcell-updates/s",
            "boxes": len(cases), "cells": cells, "steps": K, "ms_per_step": round(ms / K, 4),
            "precision": "mixed", "max_div": max(x["max_div"] for x in st),
            "sequential_fsei_step": {"value": round(cells * K / (ms_seq * 1e-3) / 1e6, 2),
                                     "ms_per_step": round(ms_seq / K, 4)},
            "sizes": "64 boxes from {32^3, 64^3, 96x96x128, 128x128x192}, seed 5"}


def run_heart_scale(args, peak):
    """512x512x768 heart-scale box (stretched walls, k^-5/3 field, 20 force
    blobs), mixed precision, 50 steps in one call."""
    import torch
    from paper_2103_15187_gb300 import fsei, inputs
    case = inputs.case_heart_scale(steps=args.heart_steps)
    grid = fsei.Grid(case.nx, case.ny, case.nz, case.lx, case.ly, zbc=case.zbc, lz=case.lz,
                     stretch=case.stretch, prec=fsei.FSEI_MIXED)
    if not args.no_autotune:
        grid.autotune()
    st = device_state(case, torch.float32)
    f = tuple(torch.tensor(a, dtype=torch.float32, device="cuda") for a in case.f)
    prm = dict(re=case.re, dt=case.dt, cfl=case.cfl, fconst=case.fconst)
    fsei.step(grid, st, f, nsteps=3, stats=False, **prm)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fsei.step(grid, st, f, nsteps=args.heart_steps, stats=False, **prm)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stats = fsei.step(grid, st, f, nsteps=0, **prm)
    words = sum(algorithmic_words(case.nx, case.ny, case.nz, True).values())
    mcups = case.cells * args.heart_steps / (ms * 1e-3) / 1e6
    gbs = words * 4 * mcups * 1e6 / 1e9
    return {"value": round(mcups, 2), "unit": "Mcell-updates/s", "cells": case.cells,
            "steps": args.heart_steps, "ms_per_step": round(ms / args.heart_steps, 4),
            "precision": "mixed", "step_hbm_frac": round(gbs / peak, 4),
            "alg_words_per_cell": round(words, 3), "max_div": stats["max_div"],
            "workload": "512x512x768, Lx=Ly=2*96/156, tanh walls 2.0, Re 3000, CFL 0.5, "
                        "k^-5/3 field (|k|<=32, unit RMS) + 20 Gaussian force blobs"}


def roofline_of(res, nx, ny, nz, bytes_per_word, peak_gbs, peak_kind):
    words = algorithmic_words(nx, ny, nz, False)
    table = {}
    best = None
    for name, (tot_ms, n) in res["kernels"].items():
        if n == 0:
            continue
        avg = tot_ms / n
        entry = {"avg_ms": avg, "launches": n}
        if name in words:
            b = words[name] * bytes_per_word * nx * ny * nz
            entry["alg_bytes"] = b
            entry["gbs"] = b / (avg * 1e-3) / 1e9
            entry["frac"] = entry["gbs"] / peak_gbs
        table[name] = entry
        if name in words and (best is None or tot_ms > res["kernels"][best][0]):
            best = name
    e = table[best]
    tr = MEASURED_TRAFFIC.get(best)
    traffic = tr["bytes"] if (tr and tr["cells"] == nx * ny * nz and bytes_per_word == 4) else None
    roof = {"bound": "hbm", "kernel": best, "achieved": round(e["gbs"], 1),
            "peak": peak_gbs, "unit": "GB/s", "frac": round(e["frac"], 4),
            "traffic": traffic, "alg_bytes": e["alg_bytes"],
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
            if peak_kind == "measured" else peak_kind}
    if traffic is not None:
        roof["traffic_kernel"] = tr["kernel"]
    step_words = sum(words.values())
    return roof, table, step_words


def cpu_oracle_sample(case, steps=2):
    """The oracle (numpy, FP64) advancing the full workload by `steps` steps
    on the host: the first (Euler start) and then Adams-Bashforth steps."""
    from oracle.grid import Grid as OGrid
    from oracle.step import oracle_step
    g = OGrid(case.nx, case.ny, case.nz, case.lx, case.ly, case.zbc, lz=case.lz,
              stretch=case.stretch)
    z = np.zeros_like(case.u)
    s = {"u": case.u, "v": case.v, "w": case.w, "p": case.p, "hu": z, "hv": z, "hw": z,
         "have_prev_h": 0}
    t0 = time.perf_counter()
    for _ in range(steps):
        s, _ = oracle_step(g, s, None, re=case.re, dt=case.dt, cfl=case.cfl,
                           fconst=case.fconst)
    dt = time.perf_counter() - t0
    return {"value": case.cells * steps / dt / 1e6, "unit": "Mcell-updates/s", "cores": 1,
            "kind": "oracle",
            "sample": "%d steps of the full %dx%dx%d workload, numpy FP64, single thread "
                      "(%.1f s)" % (steps, case.nx, case.ny, case.nz, dt)}


# ------------------------------------------------------- reference arm -----
def run_reference_arm(args, rank, world):
    """The oracle as the reference implementation, on the host cores: each
    step advances the 128^3 version of the channel workload (same physics,
    1/8 of the cells), so a --steps K --warmup W run stays within minutes."""
    if rank != 0:
        return 0
    from paper_2103_15187_gb300 import inputs
    from oracle.grid import Grid as OGrid
    from oracle.step import oracle_step
    w = WORKLOAD
    n = 128
    case = inputs.case_channel(n, n, n, w["lx"], w["ly"], w["stretch"], w["re"], w["cfl"],
                               100, w["kmin"], w["kmax"], 0.0, w["rms"], w["seed"])
    g = OGrid(n, n, n, case.lx, case.ly, case.zbc, lz=case.lz, stretch=case.stretch)
    z = np.zeros_like(case.u)
    s = {"u": case.u, "v": case.v, "w": case.w, "p": case.p, "hu": z, "hv": z, "hw": z,
         "have_prev_h": 0}
    prm = dict(re=case.re, dt=case.dt, cfl=case.cfl, fconst=case.fconst)
    for _ in range(args.warmup):
        s, _ = oracle_step(g, s, None, **prm)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s, _ = oracle_step(g, s, None, **prm)
    el = time.perf_counter() - t0
    v = case.cells * args.steps / el / 1e6
    sample = ("oracle steps of the 128^3 version of the 256^3 channel workload (same "
              "Re, CFL, stretching and spectrum; 1/8 of the cells per step), numpy FP64, "
              "single thread")
    line = {"impl": "reference", "metric": "fractional-step Mcell-updates/s", "value": v,
            "unit": "Mcell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "channel 256x256x256 (reference sample 128^3)",
                       "precision": "fp64 oracle"},
            "cpu_baseline": {"value": v, "unit": "Mcell-updates/s", "cores": 1,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fsei", choices=["fsei", "reference"])
    ap.add_argument("--error-steps", type=int, default=100)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ensemble-boxes", type=int, default=64)
    ap.add_argument("--ensemble-steps", type=int, default=100)
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--heart-steps", type=int, default=50)
    ap.add_argument("--no-heart", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="run the default launch schedule instead of a measured one")
    ap.add_argument("--schedule", default=None,
                    help="JSON dict of fsei_schedule fields for the mixed-precision grid "
                         "(e.g. one a previous run printed), applied instead of autotuning")
    ap.add_argument("--nx", type=int, default=None, help="profiling override of the extents")
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--nz", type=int, default=None)
    args = ap.parse_args()
    for key in ("nx", "ny", "nz"):
        if getattr(args, key):
            WORKLOAD[key] = getattr(args, key)
    args.warmup = max(args.warmup, 3) if args.impl == "fsei" else args.warmup
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference_arm(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    case, results, err, e2e = run_gpu_arm(args, rank, world)
    if rank != 0:
        return 0
    peak, peak_kind = measured_peaks()
    nx, ny, nz = case.nx, case.ny, case.nz
    mres = results["mixed"][0]
    roof, table, step_words = roofline_of(mres, nx, ny, nz, 4, peak, peak_kind)
    step_gbs = step_words * 4 * nx * ny * nz * mres["mcups"] / max(1, args.gpus) * 1e6 / 1e9 \
        / (nx * ny * nz)
    line = {
        "metric": "fractional-step Mcell-updates/s (mixed FP32/FP64 step)",
        "value": round(mres["mcups"], 2),
        "unit": "Mcell-updates/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(mres["ms_per_step"], 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "channel %dx%dx%d, tanh-stretched walls (2.0), Re 2000, "
                               "CFL 0.5, Poiseuille + solenoidal perturbation (RMS 0.1, k 1-8)"
                               % (nx, ny, nz),
                   "cells": nx * ny * nz, "precision": "mixed (FP32 fields; FP64 near-zero "
                   "Poisson modes and reductions)", "parallelism": "replicas only",
                   "l2": "inputs larger than L2 (state 470 MB + workspace 420 MB per step)"},
        "roofline": roof,
        "step_hbm": {"alg_words_per_cell": round(step_words, 3),
                     "achieved_gbs": round(step_gbs, 1), "frac": round(step_gbs / peak, 4)},
        "clocks": mres["clocks"],
        "schedule": {"mixed": mres["schedule"],
                     "source": ("given" if args.schedule else
                                "default" if args.no_autotune else "autotuned")},
        "gpu_launches": int(sum(n for _, n in mres["kernels"].values())),
        "kernels": {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv)
                        for kk, vv in v.items()} for k, v in table.items()},
    }
    if "fp64" in results:
        fres = results["fp64"][0]
        ginst = FP64_INSTR_PER_CELL * fres["mcups"] / max(1, args.gpus) / 1e3
        line["fp64"] = {"value": round(fres["mcups"], 2), "unit": "Mcell-updates/s",
                        "ms_per_step": round(fres["ms_per_step"], 4),
                        "mixed_speedup": round(mres["mcups"] / fres["mcups"], 3),
                        "alu": {"bound": "alu", "achieved": round(ginst, 1),
                                "peak": round(FP64_PEAK_GINST, 1),
                                "unit": "G FP64 thread-instructions/s",
                                "frac": round(ginst / FP64_PEAK_GINST, 4),
                                "instr_per_cell": FP64_INSTR_PER_CELL,
                                "peak_source": "derived: 2 FP64 lanes/clk/SM x 152 SMs x "
                                               "2070 MHz"}}
    if err is not None:
        line["mixed_error"] = {"rel_l2_velocity_vs_fp64": err, "steps": args.error_steps}
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_ensemble and args.ensemble_boxes > 0:
        line["ensemble"] = run_ensemble(args)
    if not args.no_heart and args.heart_steps > 0:
        line["heart_scale"] = run_heart_scale(args, peak)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(case)
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
