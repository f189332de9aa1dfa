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

METRIC = "fractional-step Mcell-updates/s"
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


def step_words_model(with_force):
    """Words per cell one whole step must move in the pass-minimal model:
    one pass per global line dependency (x, y and z line solves; x and y
    transforms; the z Poisson lines), each word read or written once per
    pass, the spectrum counted as one word per pass and the inverse x
    transform fused with the projection.  RHS + x sweep 13 (16 with a body
    force field), y sweep 6, z sweep + u* 9, divergence + x transform 4,
    y transforms and z Poisson 2 each, inverse x transform + projection 9:
    47 words (50 with a force field)."""
    return 50.0 if with_force else 47.0


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
# of a kernel, from an ncu --set full capture of the 256^3 channel workload,
# keyed by the kernel's name as ncu prints it; reported only for that
# workload and only while the kernel is the one the schedule launches
MEASURED_TRAFFIC = {
    "k_rhs_x_march<float, 8, 32>": {"bytes": 845.5e6, "cells": 256 ** 3},
}


def rhs_kernel_name(sched, nx, elem):
    """The RHS + x sweep kernel a single-grid schedule launches (the
    row-resident or the y-marched one; cells and lanes per row)."""
    cpl = sched.get("rhs_cells_per_lane", 0)
    if not cpl:
        return None
    kind = "k_rhs_x_march" if sched.get("rhs_rows_per_strip", 0) else "k_rhs_x_row"
    return "%s<%s, %d, %d>" % (kind, elem, cpl, nx // cpl)

# FP64 instructions of one FP64 step per cell (DFMA + DADD + DMUL thread
# instructions, the CFL pre-pass excluded), from one ncu capture of the FP64
# step on a 128^3 channel (the count per cell does not depend on the size).
# The FP64 step is bound by the FP64 pipe; its peak is measured in the run
# (fsei_fp64_fma_rate: DFMA thread instructions per second with every SM
# busy), and each of DFMA, DADD and DMUL takes one slot of that pipe.
FP64_INSTR_PER_CELL = 329.8


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


class ReplicaSync:
    """Barrier and max-over-ranks of the N-replica run: one process per GPU,
    each advancing its own copy of the workload (the step has no sharding,
    so no data moves between replicas; only these timing collectives run).
    dist: torch.distributed or None (one process); device: where the
    collective's scalar lives ("cuda" with NCCL, "cpu" with gloo)."""

    def __init__(self, dist=None, device="cuda"):
        self.dist = dist
        self.device = device

    def barrier(self):
        import torch
        if self.dist is not None:
            self.dist.barrier()
        if self.device == "cuda":
            torch.cuda.synchronize()

    def max(self, x):
        import torch
        if self.dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_rate(cells, steps, world, ms):
    """Cell updates per second of all replicas together, in millions: every
    replica advanced `cells` cells `steps` times in at most `ms` ms (the
    maximum over ranks)."""
    return cells * steps * world / (ms * 1e-3) / 1e6


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
    sync = ReplicaSync(dist, "cuda")
    barrier, max_over_ranks = sync.barrier, sync.max

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
        # blocks of exactly K steps, each bracketed by a barrier and a device
        # synchronisation, repeated until at least min_timed_s of device time
        # (and 3 blocks) have run, so that the clock sampler sees the load;
        # the median block is reported
        blocks = []
        with ClockSampler(dev) as clk:
            while len(blocks) < 3 or sum(blocks) < args.min_timed_s * 1e3:
                barrier()
                e0.record(stream)
                fsei.step(grid, st, None, nsteps=K, stats=False, **prm)
                e1.record(stream)
                barrier()
                blocks.append(max_over_ranks(e0.elapsed_time(e1)))
                if len(blocks) >= args.max_blocks:
                    break
        ms = float(np.median(blocks))
        stats = fsei.step(grid, st, None, nsteps=0, **prm)
        res = {"ms_total": ms, "ms_per_step": ms / K, "cells": cells,
               "mcups": whole_job_rate(cells, K, world, ms), "clocks": clk.summary(),
               "last_stats": stats, "blocks": len(blocks),
               "block_ms": {"median": ms, "min": float(min(blocks)), "max": float(max(blocks))}}
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

    # end to end through the public API with host buffers: per step
    # fsei_step_host copies the state (7 fields) from pinned host memory into
    # device buffers, runs one step and copies the new state back (the
    # history fields under the rest of the step); step_host_join orders the
    # stream after the last copies back before the closing event
    mixed_res, mgrid, _ = results["mixed"]
    e2e = None
    if args.e2e_steps > 0:
        init = device_state(case, torch.float32)
        host = {k: init[k].cpu().pin_memory() for k in FIELDS}
        host["have_prev_h"] = 0
        dst = {k: torch.empty_like(init[k]) for k in FIELDS}
        del init
        stream = torch.cuda.current_stream()
        for _ in range(2):      # untimed: first copies and launches
            fsei.step_host(mgrid, host, dst, None, nsteps=1, stats=False, **prm)
        fsei.step_host_join(mgrid)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            fsei.step_host(mgrid, host, dst, None, nsteps=1, stats=False, **prm)
        fsei.step_host_join(mgrid)
        e1.record(stream)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        nbytes = sum(host[k].numel() * 4 for k in FIELDS)
        assert host["have_prev_h"] == 1
        e2e = {"value": whole_job_rate(cells, args.e2e_steps, world, ms),
               "unit": "Mcell-updates/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps}
    return case, results, err, e2e


def _time_batch(cases, K, autotune, max_group=None):
    """ms per step of the boxes `cases` advanced together by fsei_batch_step
    (grouped launches in a CUDA graph), and the last call's statistics."""
    import torch
    from paper_2103_15187_gb300 import fsei
    boxes = [dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                  stretch=c.stretch, prec=fsei.FSEI_MIXED) for c in cases]
    batch = fsei.Batch(boxes)
    if autotune:
        batch.autotune()
    if max_group is not None:
        batch.set_max_group(max_group)
    states = [device_state(c, torch.float32) for c in cases]
    params = [dict(re=c.re, dt=c.dt, cfl=c.cfl, fconst=c.fconst) for c in cases]
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
    st = fsei.batch_step(batch, states, None, params, nsteps=0, stats=True)
    return e0.elapsed_time(e1) / K, st, batch.launch_groups


def run_ensemble(args):
    """64 independent boxes of uneven sizes (32^3, 64^3, 96x96x128, 128x128x192),
    FP32 fields, one batched call per K steps (CUDA graph replayed per step,
    one launch per pass for the boxes of each size), against the same boxes
    advanced one after another with fsei_step; and each size's boxes batched
    on their own."""
    import torch
    from paper_2103_15187_gb300 import fsei, inputs
    cases = inputs.case_ensemble(args.ensemble_boxes, steps=args.steps)
    if args.ensemble_sizes:
        keep = {tuple(int(v) for v in t.split("x")) for t in args.ensemble_sizes.split(",")}
        cases = [c for c in cases if (c.nx, c.ny, c.nz) in keep]
    cells = sum(c.cells for c in cases)
    K = args.ensemble_steps
    ms, st, ng = _time_batch(cases, K, not args.no_autotune)
    out = {"value": round(cells / (ms * 1e-3) / 1e6, 2), "unit": "Mcell-updates/s",
           "boxes": len(cases), "cells": cells, "steps": K, "ms_per_step": round(ms, 4),
           "precision": "mixed", "max_div": max(x["max_div"] for x in st),
           "launch_groups": ng,
           "sizes": "%d boxes from {32^3, 64^3, 96x96x128, 128x128x192}, seed 5" % len(cases)}
    # boxes per launch group (0: every box of a description in one launch)
    by_group = {}
    for mg in (1, 2, 8, 0):
        ms_g, _, ng_g = _time_batch(cases, K, not args.no_autotune, max_group=mg)
        by_group[str(mg)] = {"launch_groups": ng_g, "ms_per_step": round(ms_g, 4),
                             "value": round(cells / (ms_g * 1e-3) / 1e6, 2)}
    out["by_max_group"] = by_group
    by_size = {}
    for size in sorted({(c.nx, c.ny, c.nz) for c in cases}):
        sub = [c for c in cases if (c.nx, c.ny, c.nz) == size]
        ms_s, _, _ = _time_batch(sub, K, not args.no_autotune, max_group=0)
        csub = sum(c.cells for c in sub)
        by_size["%dx%dx%d" % size] = {"boxes": len(sub), "ms_per_step": round(ms_s, 4),
                                      "value": round(csub / (ms_s * 1e-3) / 1e6, 2)}
    out["by_size"] = by_size
    if not args.no_ensemble_seq:
        # the same boxes one after another (no graph, no overlap)
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        grids = [fsei.Grid(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                           stretch=c.stretch, prec=fsei.FSEI_MIXED) for c in cases]
        solo = [device_state(c, torch.float32) for c in cases]
        params = [dict(re=c.re, dt=c.dt, cfl=c.cfl, fconst=c.fconst) for c in cases]
        for g, s, p in zip(grids, solo, params):
            fsei.step(g, s, None, nsteps=2, stats=False, **p)
        torch.cuda.synchronize()
        e0.record(stream)
        for g, s, p in zip(grids, solo, params):
            fsei.step(g, s, None, nsteps=K, stats=False, **p)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_seq = e0.elapsed_time(e1)
        out["sequential_fsei_step"] = {"value": round(cells * K / (ms_seq * 1e-3) / 1e6, 2),
                                       "ms_per_step": round(ms_seq / K, 4)}
    return out


def run_variants(args, case, peak):
    """The other rows of the path on the 256^3 channel in mixed precision:
    the RK3 scheme (three fractional sub-steps per step), the Carreau-Yasuda
    law (its explicit remainder beside the step), and the immersed-boundary
    operators for a triangulated sphere of 20 480 faces (level-5 icosphere,
    radius 0.4, rotating): forcing of its markers and the loads on its
    faces."""
    import torch
    from paper_2103_15187_gb300 import fsei, inputs
    grid = fsei.Grid(case.nx, case.ny, case.nz, case.lx, case.ly, zbc=case.zbc, lz=case.lz,
                     stretch=case.stretch, prec=fsei.FSEI_MIXED)
    if not args.no_autotune:
        grid.autotune()
    prm = dict(re=case.re, dt=case.dt, cfl=case.cfl, fconst=case.fconst)
    K = max(args.steps, 10)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = {}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    cy = dict(lam=1.5, n=0.5, a=2.0, eta_inf=0.3)
    for name, kw in (("rk3", dict(scheme=fsei.FSEI_RK3_CN)), ("carreau_yasuda", dict(rheology=cy))):
        st = device_state(case, torch.float32)
        ms = timed(lambda: fsei.step(grid, st, None, nsteps=K, stats=False, **kw, **prm), 1) / K
        out[name] = {"ms_per_step": round(ms, 4), "value": round(case.cells / (ms * 1e-3) / 1e6, 2),
                     "unit": "Mcell-updates/s"}
    out["rk3"]["note"] = "three fractional sub-steps per time step (same CFL 0.5 rule)"
    out["carreau_yasuda"]["law"] = cy
    surf = inputs.ib_surface((0.5 * case.lx + 0.013, 0.5 * case.ly - 0.011, 0.017), 0.4, 5,
                             omega=(0.0, 0.0, 2.0))
    dev = lambda a, t=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=t, device="cuda")  # noqa: E731
    dx = case.lx / case.nx
    mk = {"xb": dev(surf["xf"]), "ub": dev(surf["ub"]), "dvb": dev(surf["af"] * dx)}
    st = device_state(case, torch.float32)
    f = [torch.zeros_like(st["u"]) for _ in range(3)]
    vel = (st["u"], st["v"], st["w"])
    lib = fsei.load()
    nm = len(surf["xf"])
    ms_f = timed(lambda: lib.fsei_ib_forcing(
        grid.handle, fsei._ptr(vel[0]), fsei._ptr(vel[1]), fsei._ptr(vel[2]), fsei._ptr(mk["xb"]),
        fsei._ptr(mk["ub"]), fsei._ptr(mk["dvb"]), nm, 1e-3, fsei._ptr(f[0]), fsei._ptr(f[1]),
        fsei._ptr(f[2]), None, fsei._stream_handle(None), None), 20)
    surf_d = {"xf": dev(surf["xf"]), "nf": dev(surf["nf"]), "af": dev(surf["af"]),
              "tris": dev(surf["tris"].astype(np.int32), torch.int32), "nnodes": len(surf["verts"])}
    ff = torch.empty((nm, 3), dtype=torch.float64, device="cuda")
    nodal = torch.zeros((len(surf["verts"]), 3), dtype=torch.float64, device="cuda")
    ms_l = timed(lambda: lib.fsei_ib_loads(
        grid.handle, fsei._ptr(st["p"]), fsei._ptr(vel[0]), fsei._ptr(vel[1]), fsei._ptr(vel[2]),
        fsei._ptr(surf_d["xf"]), fsei._ptr(surf_d["nf"]), fsei._ptr(surf_d["af"]), None,
        fsei._ptr(surf_d["tris"]), nm, surf_d["nnodes"], 1.5 * dx, case.re, fsei._ptr(ff),
        fsei._ptr(nodal), fsei._stream_handle(None), None), 20)
    out["ib"] = {"markers": nm, "forcing_ms": round(ms_f, 4), "loads_ms": round(ms_l, 4),
                 "surface": "level-5 icosphere (20 480 triangles) of radius 0.4 in the "
                            "256^3 channel, rotating; forcing of every marker's three "
                            "components, loads on every face with nodal thirds"}
    return out


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
    # per-kernel device time over 3 more steps (event pairs on the stream)
    fsei.set_kernel_timing(grid, True)
    fsei.step(grid, st, f, nsteps=3, stats=False, **prm)
    kt = fsei.kernel_times(grid)
    fsei.set_kernel_timing(grid, False)
    kwords = algorithmic_words(case.nx, case.ny, case.nz, True)
    table = {}
    for name, (tot_ms, n) in kt.items():
        if n == 0:
            continue
        entry = {"avg_ms": round(tot_ms / n, 5), "launches": n}
        if name in kwords:
            b = kwords[name] * 4 * case.cells
            entry["alg_bytes"] = b
            entry["gbs"] = round(b / (tot_ms / n * 1e-3) / 1e9, 1)
            entry["frac"] = round(entry["gbs"] / peak, 4)
        table[name] = entry
    words = step_words_model(True)
    mcups = case.cells * args.heart_steps / (ms * 1e-3) / 1e6
    gbs = words * 4 * mcups * 1e6 / 1e9
    return {"value": round(mcups, 2), "unit": "Mcell-updates/s", "cells": case.cells,
            "steps": args.heart_steps, "ms_per_step": round(ms / args.heart_steps, 4),
            "precision": "mixed", "step_hbm_frac": round(gbs / peak, 4),
            "alg_words_per_cell": round(words, 3), "max_div": stats["max_div"],
            "schedule": grid.schedule, "kernels": table,
            "workload": "512x512x768, Lx=Ly=2*96/156, tanh walls 2.0, Re 3000, CFL 0.5, "
                        "k^-5/3 field (|k|<=32, unit RMS) + 20 Gaussian force blobs"}


def adjoint_words(nx, with_fbar=True):
    """Words per cell each launch group of the adjoint step must move (read
    + write once; spectrum at its true size)."""
    spec = 2.0 * (nx // 2 + 1) / nx
    return {
        "adj_phibar": 4 + 1,                       # u,v,w,p cotangents -> x
        "adj_poisson (5 launches)": 2 + 8 * spec,   # as the forward Poisson chain
        "adj_ustar": 4 + 6,                        # cotangents, psi -> cotangents, q
        "adj_sweep_z": 6,
        "adj_sweep_y": 6,
        "adj_sweep_x": 6,
        "adj_hist": 12 + (6 if with_fbar else 0),  # q, H-bar -> H-bar, Hb (+ f-bar +=)
        "adj_gather": 13 + 4,                      # u, q, Hb, cotangents -> cotangents
    }


def run_adjoint(args, peak):
    """The 128x128x192 channel's gradient window (20 steps, checkpoint every
    5, dt frozen from CFL 0.5 at step 0, loss = kinetic energy of the central
    32^3 block): forward and backward device time per step in mixed precision
    and FP64, the adjoint kernels' device times and HBM fractions (mixed),
    and the mixed-vs-FP64 gradient error."""
    import torch
    from paper_2103_15187_gb300 import autograd as fad
    from paper_2103_15187_gb300 import fsei, inputs
    case = inputs.case_channel(128, 128, 192, steps=20, seed=4)
    zf = inputs.z_faces(case.nz, case.zbc, case.lz, case.stretch)
    nsteps, ck = 20, 5
    g64 = fsei.Grid(case.nx, case.ny, case.nz, case.lx, case.ly, zbc=case.zbc, lz=case.lz,
                    stretch=case.stretch, prec=fsei.FSEI_FP64)
    dt = fad.frozen_dt(g64, *[torch.tensor(a, dtype=torch.float64, device="cuda")
                              for a in (case.u, case.v, case.w)], case.cfl, case.re,
                       fconst=case.fconst)
    stream = torch.cuda.current_stream()
    out, grads = {}, {}
    for name, prec, dtype in (("mixed", fsei.FSEI_MIXED, torch.float32),
                              ("fp64", fsei.FSEI_FP64, torch.float64)):
        grid = g64 if prec == fsei.FSEI_FP64 else fsei.Grid(
            case.nx, case.ny, case.nz, case.lx, case.ly, zbc=case.zbc, lz=case.lz,
            stretch=case.stretch, prec=prec)
        if not args.no_autotune:
            grid.autotune()

        def once(timing=False):
            xs = [torch.tensor(a, dtype=dtype, device="cuda").requires_grad_(True)
                  for a in (case.u, case.v, case.w)]
            fs = [torch.zeros_like(xs[0]).requires_grad_(True) for _ in range(3)]
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize()
            e[0].record(stream)
            u, v, w = fad.window(grid, *xs, *fs, nsteps=nsteps, dt=dt, re=case.re,
                                 checkpoint_every=ck, fconst=case.fconst)
            e[1].record(stream)
            J = fad.kinetic_energy_subbox(u, v, w, zf, case.lx, case.ly)
            if timing:
                fsei.set_kernel_timing(grid, True)
            J.backward()
            e[2].record(stream)
            torch.cuda.synchronize()
            kt = None
            if timing:
                kt = fsei.kernel_times(grid)
                fsei.set_kernel_timing(grid, False)
            return (e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]),
                    [t.grad.detach().double() for t in xs + fs], kt)

        once()
        fwd_ms, bwd_ms, gr, _ = once()
        res = {"forward_ms_per_step": round(fwd_ms / nsteps, 4),
               "backward_ms_per_step": round(bwd_ms / nsteps, 4),
               "backward_note": "recompute of each checkpointed segment + adjoint steps"}
        if name == "mixed":
            _, _, _, kt = once(timing=True)
            words = adjoint_words(case.nx)
            table = {}
            for kname, (tot, n) in kt.items():
                if n == 0 or kname not in words:
                    continue
                avg = tot / n
                b = words[kname] * 4 * case.cells
                table[kname] = {"avg_ms": round(avg, 5), "launches": n,
                                "alg_bytes": int(b),
                                "gbs": round(b / (avg * 1e-3) / 1e9, 1),
                                "frac": round(b / (avg * 1e-3) / 1e9 / peak, 4)}
            res["kernels"] = table
            tot_words = sum(words.values())
            adj_ms = sum(v["avg_ms"] for v in table.values())
            res["adjoint_step"] = {"ms": round(adj_ms, 4), "alg_words_per_cell": round(tot_words, 3),
                                   "frac": round(tot_words * 4 * case.cells / (adj_ms * 1e-3)
                                                 / 1e9 / peak, 4)}
        out[name] = res
        grads[name] = gr
    num = sum(float(torch.linalg.vector_norm(a - b) ** 2)
              for a, b in zip(grads["mixed"], grads["fp64"]))
    den = sum(float(torch.linalg.vector_norm(b) ** 2) for b in grads["fp64"])
    out["mixed_vs_fp64_gradient_rel_l2"] = (num / den) ** 0.5
    out["workload"] = ("128x128x192 channel (as the 256^3 one), 20-step window, checkpoint "
                       "every 5, dt frozen from CFL 0.5, J = KE of the central 32^3 block; "
                       "gradients wrt u0, v0, w0, fx, fy, fz")
    return out


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
    kname = None
    if best == "rhs_x (RHS + x sweep)" and res.get("schedule"):
        kname = rhs_kernel_name(res["schedule"], nx, "float" if bytes_per_word == 4 else "double")
    tr = MEASURED_TRAFFIC.get(kname)
    traffic = tr["bytes"] if (tr and tr["cells"] == nx * ny * nz) else None
    roof = {"bound": "hbm", "kernel": best, "achieved": round(e["gbs"], 1),
            "peak": peak_gbs, "unit": "GB/s", "frac": round(e["frac"], 4),
            "traffic": traffic, "alg_bytes": e["alg_bytes"],
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
            if peak_kind == "measured" else peak_kind}
    if kname:
        roof["kernel_launched"] = kname
    step_words = sum(words.values())
    return roof, table, step_words


def host_cpu():
    """Logical CPU count and the model name lscpu reports."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return os.cpu_count() or 1, model


def _mem_available_bytes():
    try:
        with open("/proc/meminfo") as fh:
            for ln in fh:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except Exception:
        pass
    return None


def _oracle_state(case):
    z = np.zeros_like(case.u)
    return {"u": case.u, "v": case.v, "w": case.w, "p": case.p, "hu": z, "hv": z, "hw": z,
            "have_prev_h": 0}


def _oracle_steps(case, steps):
    """Seconds the oracle (numpy, FP64, one thread) takes for `steps` steps
    of `case` from its initial state."""
    from oracle.grid import Grid as OGrid
    from oracle.step import oracle_step
    g = OGrid(case.nx, case.ny, case.nz, case.lx, case.ly, case.zbc, lz=case.lz,
              stretch=case.stretch)
    s = _oracle_state(case)
    t0 = time.perf_counter()
    for _ in range(steps):
        s, _ = oracle_step(g, s, None, re=case.re, dt=case.dt, cfl=case.cfl,
                           fconst=case.fconst)
    return time.perf_counter() - t0


def _oracle_worker(q, start, steps, workload):
    """One process of the all-cores leg: builds the workload, waits for the
    common start, times its steps."""
    os.environ["OMP_NUM_THREADS"] = "1"
    WORKLOAD.update(workload)
    case = make_case()
    q.put(("ready", None))
    start.wait()
    q.put(("done", _oracle_steps(case, steps)))


def cpu_oracle_sample(case, steps=2, all_cores=True):
    """The oracle advancing the full workload on the host, as it stands (it
    is single-threaded numpy): once in this process, and as one independent
    copy per core run at the same time (as many copies as the free host
    memory holds at about 6.5 GB each), whose aggregate is the all-cores
    figure.  The processes are spawned (the parent already holds a CUDA
    context)."""
    ncpu, model = host_cpu()
    dt1 = _oracle_steps(case, steps)
    one = case.cells * steps / dt1 / 1e6
    out = {"value": round(one, 3), "unit": "Mcell-updates/s", "cores": 1, "kind": "oracle",
           "sample": "%d steps of the full %dx%dx%d workload, numpy FP64, one thread "
                     "(%.1f s)" % (steps, case.nx, case.ny, case.nz, dt1),
           "host": {"nproc": ncpu, "model": model}}
    if not all_cores or ncpu < 2:
        return out
    avail = _mem_available_bytes()
    nproc = ncpu if avail is None else max(1, min(ncpu, int(0.6 * avail // 6.5e9)))
    if nproc < 2:
        return out
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    start = ctx.Event()
    procs = [ctx.Process(target=_oracle_worker, args=(q, start, 1, dict(WORKLOAD)), daemon=True)
             for _ in range(nproc)]
    for p in procs:
        p.start()
    try:
        ready = 0
        while ready < nproc:
            kind, _ = q.get(timeout=600)
            ready += kind == "ready"
        start.set()
        times = [q.get(timeout=1200)[1] for _ in range(nproc)]
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
    agg = case.cells * nproc / max(times) / 1e6
    out["all_cores"] = {"value": round(agg, 3), "unit": "Mcell-updates/s", "cores": nproc,
                        "sample": "%d concurrent copies of the oracle, one per core, each "
                                  "advancing its own copy of the full workload by one step "
                                  "(slowest %.1f s)" % (nproc, max(times))}
    return out


# ------------------------------------------------------- reference arm -----
def run_reference_arm(args, rank, world):
    """The oracle as the reference implementation, on the host cores: each
    step advances the full 256^3 channel workload (numpy, FP64, one thread;
    about 6 s per step on a Grace core, so a --steps 20 --warmup 5 run takes
    a few minutes)."""
    if rank != 0:
        return 0
    from oracle.grid import Grid as OGrid
    from oracle.step import oracle_step
    case = make_case()
    g = OGrid(case.nx, case.ny, case.nz, case.lx, case.ly, case.zbc, lz=case.lz,
              stretch=case.stretch)
    s = _oracle_state(case)
    prm = dict(re=case.re, dt=case.dt, cfl=case.cfl, fconst=case.fconst)
    for _ in range(args.warmup):
        s, _ = oracle_step(g, s, None, **prm)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s, _ = oracle_step(g, s, None, **prm)
    el = time.perf_counter() - t0
    v = case.cells * args.steps / el / 1e6
    ncpu, model = host_cpu()
    sample = ("%d oracle steps of the full %dx%dx%d channel workload after %d untimed ones, "
              "numpy FP64, one thread (host: %d logical CPUs, %s)"
              % (args.steps, case.nx, case.ny, case.nz, args.warmup, ncpu, model))
    line = {"impl": "reference", "metric": METRIC, "value": v,
            "unit": "Mcell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(case),
            "cpu_baseline": {"value": v, "unit": "Mcell-updates/s", "cores": 1,
                             "kind": "oracle", "sample": sample,
                             "host": {"nproc": ncpu, "model": model}},
            "e2e": {"value": v, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(case):
    return {"workload": "channel %dx%dx%d, tanh-stretched walls (2.0), Re 2000, CFL 0.5, "
                        "Poiseuille + solenoidal perturbation (RMS 0.1, k 1-8)"
                        % (case.nx, case.ny, case.nz),
            "cells": case.cells, "parallelism": "replicas only",
            "l2": "inputs larger than L2 (state 470 MB + workspace 420 MB per step)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fsei", choices=["fsei", "reference"])
    ap.add_argument("--error-steps", type=int, default=100)
    ap.add_argument("--min-timed-s", type=float, default=1.0,
                    help="repeat the K-step timed block until this much device time has run")
    ap.add_argument("--max-blocks", type=int, default=1000)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ensemble-boxes", type=int, default=64)
    ap.add_argument("--ensemble-steps", type=int, default=100)
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--ensemble-sizes", default=None,
                    help="comma-separated NXxNYxNZ sizes of the ensemble to keep")
    ap.add_argument("--no-ensemble-seq", action="store_true")
    ap.add_argument("--ensemble-only", action="store_true",
                    help="print only the ensemble object (profiling runs)")
    ap.add_argument("--heart-steps", type=int, default=50)
    ap.add_argument("--no-heart", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the RK3, Carreau-Yasuda and immersed-boundary timings")
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
    if args.ensemble_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"ensemble": run_ensemble(args)}), flush=True)
        return 0
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
    roof, table, kernel_words = roofline_of(mres, nx, ny, nz, 4, peak, peak_kind)
    step_words = step_words_model(False)
    per_gpu_cells_s = mres["mcups"] / max(1, args.gpus) * 1e6
    step_gbs = step_words * 4 * per_gpu_cells_s / 1e9
    line = {
        "metric": METRIC,
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
        "config": dict(workload_config(case),
                       precision="mixed (FP32 fields; FP64 near-zero Poisson modes and "
                                 "reductions)"),
        "roofline": roof,
        "step_hbm": {"alg_words_per_cell": step_words,
                     "model": "pass-minimal: one pass per global line dependency, spectrum "
                              "1 word per pass, inverse x transform fused with the projection",
                     "achieved_gbs": round(step_gbs, 1), "frac": round(step_gbs / peak, 4),
                     "kernel_words_per_cell": round(kernel_words, 3),
                     "kernel_gbs": round(kernel_words * 4 * per_gpu_cells_s / 1e9, 1)},
        "clocks": mres["clocks"],
        "schedule": {"mixed": mres["schedule"],
                     "source": ("given" if args.schedule else
                                "default" if args.no_autotune else "autotuned")},
        "gpu_launches": int(sum(n for _, n in mres["kernels"].values())),
        "kernels": {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv)
                        for kk, vv in v.items()} for k, v in table.items()},
    }
    if "fp64" in results:
        import torch
        from paper_2103_15187_gb300 import fsei
        fres = results["fp64"][0]
        ginst = FP64_INSTR_PER_CELL * fres["mcups"] / max(1, args.gpus) / 1e3
        fpeak = fsei.fp64_fma_rate()
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        line["fp64"] = {"value": round(fres["mcups"], 2), "unit": "Mcell-updates/s",
                        "ms_per_step": round(fres["ms_per_step"], 4),
                        "mixed_speedup": round(mres["mcups"] / fres["mcups"], 3),
                        "clocks": fres["clocks"],
                        "alu": {"bound": "alu", "achieved": round(ginst, 1),
                                "peak": round(fpeak, 1),
                                "unit": "G FP64 thread-instructions/s",
                                "frac": round(ginst / fpeak, 4),
                                "instr_per_cell": FP64_INSTR_PER_CELL,
                                "peak_source": "measured in this run: fsei_fp64_fma_rate "
                                               "(independent DFMA chains on all %d SMs)"
                                               % props.multi_processor_count}}
    if err is not None:
        line["mixed_error"] = {"rel_l2_velocity_vs_fp64": err, "steps": args.error_steps}
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_ensemble and args.ensemble_boxes > 0:
        line["ensemble"] = run_ensemble(args)
    if not args.no_heart and args.heart_steps > 0:
        line["heart_scale"] = run_heart_scale(args, peak)
    if not args.no_adjoint:
        line["adjoint"] = run_adjoint(args, peak)
    if not args.no_variants:
        line.update(run_variants(args, case, peak))
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(case)
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
