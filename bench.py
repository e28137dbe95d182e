#!/usr/bin/env python3
"""RKETD-FDTD throughput on one GB300: the long inhomogeneous 1D plasma slab.

Workload (synthetic, seeded): Nz = 2^24 cells, dz = 1 um, Courant 0.5, 40000 leapfrog
steps, Epstein density ramp wp0 = 2pi*50 GHz, L = 2 mm, with a 5% Gaussian ripple, nu
uniform in [1e9, 5e10] 1/s, 32-cell CPML at both ends, Eq. 15 source, running DFT at two
probes x 512 frequencies. One bench step = one whole run of that workload: the per-cell
RKETD coefficient precompute from (wp2, nu), 40000 steps of Eqs. 14/13/11 with the
source, CPML ends and DFT folds, and the spectra. Fields are FP32 (coefficients from
FP64, compensated DFT); an FP64 run of the same workload is reported beside it.

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle (OpenMP, all
host cores) on a bounded prefix of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import math
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RKETD-FDTD Gcell-updates/s, % HBM roofline; adjoint/forward time ratio"
UNIT = "Gcell-updates/s"
WORKLOAD = ("1D long inhomogeneous Drude slab: Nz=2^24, dz=1um, Courant 0.5, 40000 steps, Epstein wp^2 ramp "
            "(wp0=2pi*50GHz, L=2mm, 5% seeded ripple), nu~U[1e9,5e10], CPML 32+32, 2 probes x 512 DFT freqs")
B_ALG = {"f32": 32.0, "f64": 64.0}  # algorithmic bytes per cell-update: E,H,J read+write + wp2,nu read
# Arithmetic per cell-update with the folded current G = cj J~ - da E: Eq. 14 sub + fma; Eq. 13
# sub + fma + sub; the G recursion (Eq. 11) mul + 2 fma + add (small terms summed before G is
# added). Nine pipe operations in either precision (13 flops, fma = 2).
OPS_PER_CELL_UPDATE = {"f32": 9.0, "f64": 9.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nz", type=int, default=1 << 24)
    ap.add_argument("--run-steps", type=int, default=40000)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=0, help="oracle steps per CPU sample (0 = auto)")
    ap.add_argument("--options", default="", help="library options, e.g. cells_per_lane=16,tb_steps=32")
    ap.add_argument("--no-batch", action="store_true", help="skip the ragged-batch measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--adj-profiles", type=int, default=64)
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D sphere measurement")
    ap.add_argument("--no-c1", action="store_true", help="skip the paper-slab (config 1) measurement")
    ap.add_argument("--no-2d", action="store_true", help="skip the 2D TMz/TEz measurement")
    ap.add_argument("--steps2d", type=int, default=1000)
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the Eq. 9 / Eq. 10 / split-PML measurement on the long slab")
    ap.add_argument("--variant-steps", type=int, default=4096)
    ap.add_argument("--c1-reps", type=int, default=9)
    ap.add_argument("--profile", choices=PROFILE_CASES, default=None,
                    help="run one short workload for an ncu capture and exit (no timing)")
    ap.add_argument("--profile-steps", type=int, default=96)
    ap.add_argument("--only-3d", action="store_true", help="run only the 3D sphere measurement (profiling)")
    ap.add_argument("--n3d", type=int, default=512)
    ap.add_argument("--kc3d", type=int, default=0, help="planes per 3D work item (0 = the library default)")
    ap.add_argument("--box3d", type=int, default=None,
                    help="TF/SF box this many cells in from every face (profile case c5-sphere; default: the recipe)")
    ap.add_argument("--steps3d", type=int, default=4000)
    ap.add_argument("--batch-slabs", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=20000)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured", p
    except Exception:
        return 6800.0, "fallback", {}


def fp32_pipe_peak_tops(clock_mhz: float) -> float:
    """FP32 pipe operations per second from unit counts: 152 SMs x 128 FP32 lanes x clock."""
    return 152 * 128 * clock_mhz * 1e6 / 1e12


def fp64_pipe_peak_tops() -> float:
    """FP64 pipe operations per second measured on this machine's GB300 with an FMA-chain
    microbenchmark: 0.60 T DFMA/s (2 per clock per SM); DADD occupies the same pipe."""
    return 0.60


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.index is not None:
            cmd += ["-i", str(self.index)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except ValueError:
                continue
            for n, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        load = [x for x in sm if x > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def tile_kernel_sha(prec):
    """sha256 over the sources of the interior tiled kernel of a precision (its launch file and the
    tile bodies and helpers it includes)."""
    csrc = os.path.join(ROOT, "paper_1709_00821_gb300", "csrc")
    names = ["step_tb2.cu" if prec == "f32" else "step_tb.cu", "tile_bodies.cuh", "tile_common.cuh"]
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(csrc, n), "rb").read())
    return h.hexdigest()


def traffic_record(prec):
    """Per-cell-update DRAM bytes of the interior tiled kernel from the committed ncu summary
    (profiles/tb_kernel_traffic.json), valid only while that kernel's sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "tb_kernel_traffic.json")
    key = "step_tb2_sha256" if prec == "f32" else "step_tb_sha256"
    try:
        rec = json.load(open(path))
        sha = tile_kernel_sha(prec)
        if rec.get(key) == sha and prec in rec:
            return rec[prec]["dram_bytes_per_cell_update"], rec
    except Exception:
        pass
    return None, None


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist

    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local, dist


def max_over_ranks(x: float, dist) -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def cpu_baseline(slab, steps_per_sample: int, samples: int, warm: int = 0):
    """Times the FP64 oracle (OpenMP build, all host cores) on prefixes of the workload."""
    import oracle

    oracle.build(omp=True)
    cores = oracle.threads(omp=True)
    times = []
    for i in range(warm + samples):
        t0 = time.perf_counter()
        oracle.run1d(slab, steps=steps_per_sample, omp=True)
        dt = time.perf_counter() - t0
        if i >= warm:
            times.append(dt)
    cu = slab.nz * steps_per_sample * samples
    return cu / sum(times) / 1e9, cores, times


def run_reference(args):
    rank, ws, local, dist = dist_init()
    if rank != 0:
        return
    from paper_1709_00821_gb300 import workloads as wl

    slab = wl.c2_epstein(nz=args.nz, steps=args.run_steps)
    steps_per = args.cpu_steps or 60
    val, cores, times = cpu_baseline(slab, steps_per, args.steps, warm=args.warmup)
    sample = (f"{steps_per}-step prefix of the run (per bench step, incl. the oracle's per-call coefficient "
              f"setup) on all {args.nz} cells, {args.steps} timed after {args.warmup} warm-up")
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "nz": args.nz, "steps_per_run": args.run_steps},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def parse_options(s):
    out = {}
    for kv in filter(None, s.split(",")):
        k, v = kv.split("=")
        out[k.strip()] = int(v)
    return out


def gpu_run(args, prec, steps, warmup, slab, wp2_d, nu_d, timing=True, opts=None):
    """Timed whole runs with device-resident inputs; returns dict of measurements."""
    import torch

    from paper_1709_00821_gb300 import rketd as rk

    ctx = rk.Context(slab, prec, options=opts or None)
    stream = torch.cuda.current_stream()
    P = ctx.n_slabs * ctx.n_probes * len(ctx.freq)
    xr = torch.empty(P, dtype=torch.float64, device="cuda")
    xi = torch.empty(P, dtype=torch.float64, device="cuda")

    def one_run():
        ctx.set_medium(wp2_d, nu_d)
        ctx.reset()
        ctx.step(slab.steps)
        ctx.spectra_device(xr.data_ptr(), xi.data_ptr())

    for _ in range(warmup):
        one_run()
    ctx.sync()
    torch.cuda.synchronize()
    return ctx, one_run, (xr, xi)


# The paper's Table 2 (1000 steps, GTX 1080): Yee cells -> GPU ms, quoted as context beside our sweep.
PAPER_TABLE2_GPU_MS = {1024: 33, 5120: 33, 10240: 33, 20480: 34, 30720: 46, 40960: 53, 51200: 61, 61440: 64}


def _time_runs(slabs, prec, steps, reps, warm=2, opts=None):
    """Median CUDA-event time (ms) of reset + steps + spectra into device buffers; also the variant used
    and the launches per run."""
    import torch

    from paper_1709_00821_gb300 import rketd as rk

    with rk.Context(slabs, prec, options=opts) as ctx:
        P = ctx.n_slabs * ctx.n_probes * len(ctx.freq)
        xr = torch.empty(max(P, 1), dtype=torch.float64, device="cuda")
        xi = torch.empty_like(xr)

        def run():
            ctx.reset()
            ctx.step(steps)
            if P:
                ctx.spectra_device(xr.data_ptr(), xi.data_ptr())

        for _ in range(warm):
            run()
        torch.cuda.synchronize()
        ts = []
        l0 = ctx.launches
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), ctx.options(), (ctx.launches - l0) / reps


def _time_pair(s1, s2, prec, steps, reps, warm=2):
    """Median CUDA-event time (ms) of two independent runs (reset + steps + spectra into device
    buffers) issued on two streams at once: the plasma run and its vacuum reference, each in its
    own context."""
    import torch

    from paper_1709_00821_gb300 import rketd as rk

    main = torch.cuda.current_stream()
    other = torch.cuda.Stream()
    with rk.Context(s1, prec) as ca, rk.Context(s2, prec, stream=other.cuda_stream) as cb:
        bufs = []
        for ctx in (ca, cb):
            P = ctx.n_slabs * ctx.n_probes * len(ctx.freq)
            bufs.append((P, torch.empty(max(P, 1), dtype=torch.float64, device="cuda"),
                         torch.empty(max(P, 1), dtype=torch.float64, device="cuda")))

        def run():
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event()
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(main)
            other.wait_event(e0)
            for ctx, (P, xr, xi) in zip((ca, cb), bufs):
                ctx.reset()
                ctx.step(steps)
                if P:
                    ctx.spectra_device(xr.data_ptr(), xi.data_ptr())
            e1.record(other)
            main.wait_event(e1)
            e2.record(main)
            return e0, e2

        for _ in range(warm):
            run()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e2 = run()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e2))
        return statistics.median(ts), ca.options()["variant"], cb.options()["variant"]


def measure_c1(args):
    """Config 1 (the paper's slab: 2000 cells, 8000 steps, Mur ends, 2 probes x 200 frequencies), FP64
    as the config states and FP32 beside it. A run is latency-bound (the state is 48 KB): the library
    picks the resident variant (one thread-block cluster holds the slab for a whole DFT block of
    steps). Plus the paper's Table 2 sweep (1000 steps, slab in the middle 29%) as context."""
    import oracle
    from paper_1709_00821_gb300 import workloads as wl

    s = wl.c1_plain_slab()
    cells = s.nz * s.steps
    out = {"workload": "2000-cell Drude slab (cells 800-919), Mur ends, 8000 steps, 2 probes x 200 freqs",
           "unit": UNIT}
    for prec in ("f64", "f32"):
        ms, opt, nl = _time_runs(s, prec, s.steps, reps=args.c1_reps)
        ms_rt, va, vb = _time_pair(s, s.vacuum(), prec, s.steps, reps=args.c1_reps)
        names = {3: "resident", 2: "tiled", 1: "plain"}
        out[prec] = {"ms_per_run": ms, "value": cells / (ms / 1e3) / 1e9, "gpu_launches_per_run": nl,
                     "variant": names[opt["variant"]],
                     "ms_plasma_and_vacuum_reference": ms_rt,
                     "note_reference": "R/T need the vacuum run too: the plasma and vacuum runs in two contexts "
                                       f"({names[va]}, {names[vb]}) on two streams at once"}
    oracle.build()
    t0 = time.perf_counter()
    oracle.run1d(s)
    t = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": cells / t / 1e9, "unit": UNIT, "ms_per_run": 1e3 * t, "cores": 1,
                           "kind": "oracle", "sample": "the whole run (plasma slab), serial FP64 oracle"}
    sweep = []
    for nz, paper_ms in PAPER_TABLE2_GPU_MS.items():
        t = wl.c1_plain_slab(nz=nz, steps=1000)
        lo = int(round(nz * (0.5 - 0.145)))
        hi = int(round(nz * (0.5 + 0.145)))
        t.wp2[:] = 0.0
        t.nu[:] = 0.0
        t.wp2[lo:hi] = (2 * math.pi * 28.7e9) ** 2
        t.nu[lo:hi] = 2e10
        row = {"cells": nz, "paper_gpu_ms": paper_ms}
        for prec in ("f64", "f32"):
            ms, opt, _ = _time_runs(t, prec, 1000, reps=5)
            row[f"{prec}_ms"] = ms
            row[f"{prec}_variant"] = {3: "resident", 2: "tiled", 1: "plain"}[opt["variant"]]
        sweep.append(row)
    out["table2_sweep"] = {"rows": sweep, "steps": 1000,
                           "note": "paper: GTX 1080, precision not stated, middle 1200/4096 of the domain is "
                                   "plasma; here the middle 29% (our reading), same plasma, Mur ends, the same "
                                   "2 probes x 200 frequencies DFT included"}
    return out


def measure_batch(args):
    """Ragged batch: 4096 independent slabs (nz log-uniform in [1024, 65536]) for 20000 steps in
    one context, FP32 fields, replayed as one CUDA graph per run. Compared with the paper's
    structure (one H and one E+J launch per step): slab by slab on one stream, and all slabs per
    launch; both plain forms are timed on a prefix and scaled to the full run."""
    import torch

    from paper_1709_00821_gb300 import rketd as rk
    from paper_1709_00821_gb300 import workloads as wl

    b = wl.c3_batch(n_slabs=args.batch_slabs, steps=args.batch_steps)
    cells = b.total_cells
    cu = cells * b.steps
    ctx = rk.Context(b.slabs, "f32")
    # tile shape (cells per lane, steps per pass, warps per block) picked by the library's
    # autotuner on this batch (state saved and restored around the trials)
    t_tune = time.perf_counter()
    ctx.autotune(4)
    t_tune = time.perf_counter() - t_tune
    P = ctx.n_slabs * ctx.n_probes * len(ctx.freq)
    xr = torch.empty(P, dtype=torch.float64, device="cuda")
    xi = torch.empty(P, dtype=torch.float64, device="cuda")

    def run():
        ctx.reset()
        ctx.step(b.steps)
        ctx.spectra_device(xr.data_ptr(), xi.data_ptr())

    run()  # captures the graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launches
    e0.record()
    run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = ctx.launches - l0
    opts = ctx.options()
    ctx.close()
    del ctx
    # the persistent variant with the same tile shape: every pass of a DFT block in one launch
    with rk.Context(b.slabs, "f32", options={"variant": 4, "cells_per_lane": opts["cells_per_lane"],
                                             "tb_steps": opts["tb_steps"]}) as cq:
        def run_p():
            cq.reset()
            cq.step(b.steps)
            cq.spectra_device(xr.data_ptr(), xi.data_ptr())

        run_p()  # captures the graph
        torch.cuda.synchronize()
        lp0 = cq.launches
        e0.record()
        run_p()
        e1.record()
        torch.cuda.synchronize()
        ms_p = e0.elapsed_time(e1)
        persistent = {"value": cu / (ms_p / 1e3) / 1e9, "ms_per_run": ms_p, "gpu_launches_per_run": cq.launches - lp0,
                      "variant": f"persistent (options.variant 4), K={opts['cells_per_lane']}, "
                                 f"{opts['tb_steps']} steps/pass: one launch per DFT block of "
                                 f"{cq.options()['dft_block']} steps"}
    # plain form, all slabs per launch (one H + one E/J launch per step over every cell)
    pre = 100
    with rk.Context(b.slabs, "f32", options={"variant": 1}) as cp:
        cp.step(5)
        cp.sync()
        e0.record()
        cp.step(pre)
        e1.record()
        torch.cuda.synchronize()
        ms_all = e0.elapsed_time(e1) * b.steps / pre
    # plain form, one slab per launch: a sample of slabs, scaled by cell count share
    rng = np.random.default_rng(5)
    pick = sorted(rng.choice(len(b.slabs), size=min(16, len(b.slabs)), replace=False).tolist())
    t_sample = 0.0
    for i in pick:
        with rk.Context(b.slabs[i], "f32", options={"variant": 1}) as cs:
            cs.step(5)
            cs.sync()
            e0.record()
            cs.step(pre)
            e1.record()
            torch.cuda.synchronize()
            t_sample += e0.elapsed_time(e1) * b.steps / pre
    ms_slab = t_sample * len(b.slabs) / len(pick)
    return {"workload": f"{len(b.slabs)} slabs, {cells} cells, {b.steps} steps, FP32, Mur, 2 probes x 200 freqs",
            "value": cu / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_run": ms, "gpu_launches_per_run": launches,
            "graph": "one CUDA graph per run (captured on the first run)",
            "variant": f"tiled K={opts['cells_per_lane']}, {opts['tb_steps']} steps/pass, "
                       f"{opts['warps_per_block']} warps/CTA (rketd_autotune, {t_tune:.1f} s)",
            "plain_all_slabs_per_launch": {"value": cu / (ms_all / 1e3) / 1e9, "ms_per_run": ms_all,
                                           "measured": f"{pre}-step prefix, scaled to {b.steps}"},
            "plain_slab_by_slab": {"value": cu / (ms_slab / 1e3) / 1e9, "ms_per_run": ms_slab,
                                   "measured": f"{len(pick)} sampled slabs x {pre} steps, scaled by slab count "
                                               f"and steps"},
            "speedup_vs_slab_by_slab": ms_slab / ms, "speedup_vs_all_slabs_plain": ms_all / ms,
            "persistent": persistent}


def measure_adjoint(args):
    """Adjoint workload: 64 profiles of 65536 cells, 30000 FP32 steps, trainable cells
    [2048, 6144), loss = sum_f (|R(f)| - |R_t(f)|)^2 over 256 frequencies against the target
    spectrum the FP64 oracle wrote to tests/golden/c4_target.txt. Times the checkpointed forward
    (every 512 steps) and the adjoint (segment recompute + transposed sweep + gradients)."""
    import torch

    from paper_1709_00821_gb300 import rketd as rk
    from paper_1709_00821_gb300 import workloads as wl

    tgt = np.loadtxt(os.path.join(ROOT, "tests", "golden", "c4_target.txt"))[:, 1]
    profs = [wl.c4_profile(i) for i in range(args.adj_profiles)]
    steps, every, win = profs[0].steps, 512, (2048, 6144)
    # incident spectrum: the same line without plasma (every profile shares source and probe)
    with rk.Context(profs[0].vacuum(), "f32") as cv:
        cv.step(steps)
        Xi = cv.spectra()[0, 0]
    ctx = rk.Context(profs, "f32")
    n = sum(p.nz for p in profs)
    gw = torch.empty(n, dtype=torch.float64, device="cuda")
    gn = torch.empty(n, dtype=torch.float64, device="cuda")
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def once(timed):
        e[0].record()
        ctx.forward_ckpt(steps, every)
        e[1].record()
        X = ctx.spectra()[:, 0]
        d = X - Xi[None]
        absr = np.abs(d) / np.abs(Xi)[None]
        loss = float(np.sum((absr - tgt[None]) ** 2))
        coef = 2 * (absr - tgt[None]) / (np.abs(Xi)[None] * np.abs(d))
        gX = np.zeros((len(profs), ctx.n_probes, len(ctx.freq)), complex)
        gX[:, 0] = coef * d.real + 1j * coef * d.imag
        gre = torch.from_numpy(np.ascontiguousarray(gX.real)).cuda()
        gim = torch.from_numpy(np.ascontiguousarray(gX.imag)).cuda()
        torch.cuda.synchronize()
        e[2].record()
        ctx.adjoint(gre, gim, win[0], win[1], gw, gn)
        e[3].record()
        torch.cuda.synchronize()
        return loss, e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])

    once(False)
    runs = [once(True) for _ in range(3)]
    loss = runs[-1][0]
    t_fwd = float(np.median([r[1] for r in runs]))
    t_adj = float(np.median([r[2] for r in runs]))
    cu = n * steps
    ctx.close()
    return {"workload": f"{len(profs)} profiles x 65536 cells, {steps} steps, FP32, checkpoint every {every}, "
                        f"window [{win[0]}, {win[1]}), 256 frequencies",
            "forward_ms": t_fwd, "adjoint_ms": t_adj, "ratio": t_adj / t_fwd,
            "runs": [{"forward_ms": r[1], "adjoint_ms": r[2]} for r in runs],
            "timing": "median of 3 runs after one warm-up run",
            "forward_gcells": cu / (t_fwd / 1e3) / 1e9, "loss": loss,
            "adjoint_includes": "segment recompute with window recording, seeds, transposed sweep, gradient sums, "
                                "chain rule"}


# Algorithmic DRAM bytes per 2D cell-update (FP32; twice that in FP64): the H kernel reads the E
# component(s) it differences and reads and writes H; the E+J kernel reads H, reads and writes E
# and the carried current, and reads the material byte.
B_ALG_2D = {"tm": {"f32": 20 + 25, "f64": 40 + 49}, "te": {"f32": 16 + 37, "f64": 32 + 73}}


def measure_2d(args, hbm_peak):
    """2D TMz/TEz step (the paper's stated generalisation): a plasma layer across a periodic-x grid
    of 4096 x 16384 cells, one transverse Fourier mode meeting it at oblique incidence, Mur y ends,
    2 probes x 200 frequencies; 1000 timed steps after 24 untimed ones, CUDA events on the context's
    stream. Plus the serial 2D oracle on a 512 x 512 sample of the same recipe."""
    import torch

    import oracle
    from paper_1709_00821_gb300 import rketd as rk
    from paper_1709_00821_gb300 import workloads as wl

    nx, ny, steps = 4096, 16384, args.steps2d
    out = {"workload": f"{nx} x {ny} periodic-x grid, plasma layer (rows {ny // 2 - 15}..{ny // 2 + 14}), "
                       f"transverse mode 16 at oblique incidence, Mur y ends, {steps} steps, 2 probes x 200 freqs",
           "unit": UNIT}
    for pol, prec in (("tm", "f32"), ("te", "f32"), ("tm", "f64")):
        p = wl.slab_2d(nx, ny, pol, mode=16, steps=steps)
        with rk.Context2D(p, prec) as ctx:
            ctx.step(24)
            ctx.sync()
            l0 = ctx.launches
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.step(steps)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            ok = np.all(np.isfinite(ctx.spectra()))
            launches = ctx.launches - l0
        rate = nx * ny * steps / (ms / 1e3)
        b = B_ALG_2D[pol][prec]
        out[f"{pol}_{prec}"] = {"value": rate / 1e9, "ms_per_step": ms / steps, "gpu_launches": launches,
                                "spectra_finite": bool(ok),
                                "roofline": {"bound": "hbm", "achieved": b * rate / 1e9, "peak": hbm_peak,
                                             "unit": "GB/s", "frac": b * rate / 1e9 / hbm_peak,
                                             "bytes_per_cell_update": b, "kernels": f"k2_{pol}_h + k2_{pol}_e"}}
    q = wl.slab_2d(512, 512, "tm", mode=1, steps=20)
    oracle.build()
    t0 = time.perf_counter()
    oracle.run2d(q)
    t = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": 512 * 512 * 20 / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                           "sample": f"the same recipe (TMz) on a 512 x 512 grid, 20 steps, serial FP64 2D oracle, "
                                     f"{t:.2f} s"}
    return out


def measure_variants(args):
    """The paper's other current recursions and its boundary on the long slab (2^24 cells, FP32 and
    FP64, 4096 steps each): Eq. 9 (coefficients only: the tiled kernels), Eq. 10 read literally
    (carries E^{n-1}: the plain kernels), and the 5-cell split-field PML ends, beside the Eq. 11 run
    with CPML ends on the same slab."""
    import copy

    from paper_1709_00821_gb300 import workloads as wl

    steps = args.variant_steps
    base = wl.c2_epstein(nz=args.nz, steps=steps)
    names = {3: "resident", 2: "tiled", 1: "plain"}
    out = {"workload": f"long Drude slab, {base.nz} cells, {steps} steps per run", "unit": UNIT}
    for prec in ("f32", "f64"):
        for label, scheme, bc in (("eq11_cpml", wl.SCHEME_RKETD, "cpml"), ("eq9_cpml", wl.SCHEME_ETD1, "cpml"),
                                  ("eq10_cpml", wl.SCHEME_ETD2, "cpml"), ("eq11_pml5", wl.SCHEME_RKETD, "pml")):
            s = copy.deepcopy(base)
            s.scheme = scheme
            if bc == "pml":
                s.bc, s.cpml_cells = "pml", 5
                s.wp2 = s.wp2.copy()
                s.wp2[:5] = s.wp2[-5:] = 0.0  # the split-field layers are vacuum
            ms, opt, nl = _time_runs(s, prec, steps, reps=2, warm=1)
            out[f"{label}_{prec}"] = {"value": base.nz * steps / (ms / 1e3) / 1e9, "ms_per_run": ms,
                                      "variant": names[opt["variant"]], "gpu_launches_per_run": nl}
    return out


def bytes_3d(p, esz=4):
    """Algorithmic DRAM bytes per cell-update of the 3D step: E and H read once and written
    once (6 components), the material byte, the carried current read and written where the
    component is plasma, and each CPML memory read and written where its grading is active
    (2 npml positions per axis)."""
    n = p.nx * p.ny * p.nz
    m = np.asarray(p.mat)
    plasma = int(np.count_nonzero(m & 3) + np.count_nonzero((m >> 2) & 3) + np.count_nonzero((m >> 4) & 3))
    per_axis = {0: p.ny * p.nz, 1: p.nx * p.nz, 2: p.nx * p.ny}
    axes = [1, 2, 2, 0, 0, 1] * 2  # derivative axis of the 12 memories (E side, then H side)
    psi = sum(2 * p.npml * per_axis[ax] for ax in axes if not (p.periodic_xy and ax < 2))
    total = 12 * esz * n + n + 2 * esz * plasma + 2 * esz * psi
    return total / n, {"fields": 12 * esz, "material": 1, "current": 2 * esz * plasma / n, "cpml": 2 * esz * psi / n}


def traffic_record_3d(n):
    """DRAM bytes per step of the 3D staged form from the committed ncu summary
    (profiles/k3_staged_traffic.json), valid while fdtd3d.cu is unchanged: per work kind, the bytes
    per tile-plane of small captures (one kind per capture, a smaller grid of the same recipe),
    scaled to an n^3 grid by that grid's tile-planes of each kind."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "k3_staged_traffic.json")))
        sha = hashlib.sha256(open(os.path.join(ROOT, "paper_1709_00821_gb300", "csrc", "fdtd3d.cu"), "rb")
                             .read()).hexdigest()
        if rec.get("fdtd3d_sha256") == sha and str(n) in rec.get("scaled", {}):
            out = dict(rec["scaled"][str(n)])
            out["captured_n"] = rec["captured"]["n"]
            return out
    except Exception:
        pass
    return None


def measure_3d(args, hbm_peak):
    """3D scale-up: 512^3 Yee grid, Drude sphere of radius 120 cells, TF/SF plane wave, 16-cell
    CPML on every face, 4000 FP32 steps, 2 probes x 200 frequencies; one run = reset, all steps
    and the spectra read back, timed with CUDA events on the context's stream."""
    import torch

    from paper_1709_00821_gb300 import rketd as rk
    from paper_1709_00821_gb300 import workloads as wl

    p = wl.sphere_problem(n=args.n3d, steps=args.steps3d)
    cells = p.nx * p.ny * p.nz
    bpc, parts = bytes_3d(p)
    with rk.Context3D(p, "f32", k_chunk=args.kc3d or None) as ctx:
        ctx.step(20)
        ctx.sync()
        ctx.reset()
        torch.cuda.synchronize()
        l0 = ctx.launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.step(p.steps)
        e1.record()
        X = ctx.spectra()
        ms = e0.elapsed_time(e1)
        launches = ctx.launches - l0
    rate = cells * p.steps / (ms / 1e3)
    ach = bpc * rate / 1e9
    trec = traffic_record_3d(args.n3d)
    cpu = None
    if not args.no_cpu:
        # the 3D oracle (serial C, FP64) on a bounded sample: the same recipe on a 256^3 grid
        import oracle

        q = wl.sphere_problem(n=256, steps=3)
        t0 = time.perf_counter()
        oracle.run3d(q)
        dt_cpu = time.perf_counter() - t0
        cpu = {"value": q.nx * q.ny * q.nz * q.steps / dt_cpu / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the same sphere recipe on a 256^3 grid, 3 steps (serial FP64 3D oracle, allocation "
                         f"included), {dt_cpu:.1f} s"}
    return {"workload": f"{p.nx}^3 Yee grid, sphere r={args.n3d * 120 // 512} cells (wp=2pi*40 GHz, nu=2e10), "
                        f"TF/SF plane wave, {p.npml}-cell CPML all faces, {p.steps} steps, FP32, "
                        f"{len(p.probes)} probes x {len(p.freq_hz)} freqs",
            "value": rate / 1e9, "unit": UNIT, "ms_per_step": ms / p.steps, "gpu_launches_per_run": launches,
            "variant": "staged (TMA-fed fused H+E/J step; interior and boundary tile kernels)",
            "spectra_finite": bool(np.all(np.isfinite(X))), "cpu_baseline": cpu,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                         "bytes_per_cell_update": bpc, "bytes_parts": parts,
                         "traffic": trec["dram_bytes_per_step"] if trec else None,
                         "traffic_per_cell_update": trec["dram_bytes_per_cell_update"] if trec else None,
                         "traffic_source": ("ncu dram bytes per tile-plane of each staged kind, captured one kind "
                                            f"at a time on the {trec['captured_n']}^3 grid and scaled to this grid "
                                            "by its tile-planes of each kind (profiles/k3_staged_traffic.json)")
                                           if trec else None,
                         "note": "the unit is one step: two tile kernels run concurrently on two streams"}}


def run_ours(args):
    import torch

    from paper_1709_00821_gb300 import rketd as rk
    from paper_1709_00821_gb300 import workloads as wl

    rank, ws, local, dist = dist_init()
    torch.cuda.set_device(local)
    dev_index = None
    try:
        props = torch.cuda.get_device_properties(local)
        dev_index = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
    except Exception:
        dev_index = None
    hbm_peak, peak_kind, peak_rec = peaks()
    slab = wl.c2_epstein(nz=args.nz, steps=args.run_steps)
    cells = slab.nz * slab.steps  # cell-updates per bench step
    wp2_d = torch.from_numpy(slab.wp2).cuda()
    nu_d = torch.from_numpy(slab.nu).cuda()
    opts = parse_options(args.options)

    # ---- FP32 headline: device-resident inputs ----
    ctx, one_run, spec = gpu_run(args, "f32", args.steps, args.warmup, slab, wp2_d, nu_d, opts=opts)
    barrier(dist)
    torch.cuda.synchronize()
    launches0 = ctx.launches
    ctx.kernel_timing(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev_index) as clk:
        ev0.record()
        for _ in range(args.steps):
            one_run()
        ev1.record()
        torch.cuda.synchronize()
    barrier(dist)
    ms = ev0.elapsed_time(ev1)
    k_ms, k_launches, k_cells = ctx.get_kernel_timing()
    ctx.kernel_timing(False)
    launches = ctx.launches - launches0
    ms_max = max_over_ranks(ms, dist)
    value = ws * cells * args.steps / (ms_max / 1e3) / 1e9
    opt_used = ctx.options()
    clocks = clk.summary()

    # roofline of the dominant kernel (interior tiled step)
    avg_launch_s = k_ms / 1e3 / max(k_launches, 1)
    cu_per_launch = k_cells / max(k_launches, 1)
    kern_rate = cu_per_launch / avg_launch_s  # cell-updates/s inside the kernel
    clock_for_peak = 2070.0
    alu_peak = fp32_pipe_peak_tops(clock_for_peak)
    alu_ach = OPS_PER_CELL_UPDATE["f32"] * kern_rate / 1e12
    bpc, trec = traffic_record("f32")
    roofline = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "Tops/s (FP32 lane-ops)",
                "frac": alu_ach / alu_peak,
                "traffic": (bpc * cu_per_launch if bpc is not None else None),
                "kernel": (f"k_tb2<K={opt_used['cells_per_lane']}> (FP32x2 pairs, interior tiles, "
                           f"{opt_used['tb_steps']} steps/launch)" if opt_used.get("fp32_pairs", 0) != 2 else
                           f"k_tb<float,K={opt_used['cells_per_lane']},interior> ({opt_used['tb_steps']} steps/launch)"),
                "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz (unit counts x max clock)",
                "ops_per_cell_update": OPS_PER_CELL_UPDATE["f32"],
                "traffic_source": "ncu dram bytes per exact cell-update (profiles/tb_kernel_traffic.json) x launch",
                "cell_updates_per_launch": cu_per_launch, "avg_launch_ms": avg_launch_s * 1e3}
    hbm_eff = {"bound": "hbm", "achieved": B_ALG["f32"] * kern_rate / 1e9, "peak": hbm_peak, "unit": "GB/s",
               "frac": B_ALG["f32"] * kern_rate / 1e9 / hbm_peak, "peak_kind": peak_kind,
               "bytes_per_cell_update": B_ALG["f32"],
               "whole_step_frac": B_ALG["f32"] * value / ws / hbm_peak,
               "note": "algorithmic bytes x rate; temporal blocking moves fewer DRAM bytes than this"}
    if bpc is not None:
        hbm_eff["dram_bytes_per_cell_update"] = bpc
        hbm_eff["dram_gbs"] = bpc * kern_rate / 1e9

    # ---- e2e through the C ABI with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        hw = torch.from_numpy(slab.wp2).pin_memory()
        hn = torch.from_numpy(slab.nu).pin_memory()
        nP = ctx.n_slabs * ctx.n_probes * len(ctx.freq)

        def e2e_run():
            ctx.set_medium_host_ptr(hw.data_ptr(), hn.data_ptr())
            ctx.reset()
            ctx.step(slab.steps)
            return ctx.spectra()  # device->host, synchronises

        e2e_run()
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_run()
        t = time.perf_counter() - t0
        t = max_over_ranks(t, dist)
        e2e = {"value": ws * cells * args.steps / t / 1e9, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * slab.nz,
               "d2h_bytes_per_step": 2 * 8 * nP}
    ctx.close()
    del ctx

    # ---- FP64 beside it ----
    fp64 = None
    if not args.no_fp64:
        ctx64, run64, _ = gpu_run(args, "f64", 1, 1, slab, wp2_d, nu_d)
        barrier(dist)
        ctx64.kernel_timing(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        run64()
        e1.record()
        torch.cuda.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1), dist)
        k64 = ctx64.get_kernel_timing()
        o64 = ctx64.options()
        ctx64.close()
        v64 = ws * cells / (ms64 / 1e3) / 1e9
        krate64 = (k64[2] / max(k64[1], 1)) / (k64[0] / 1e3 / max(k64[1], 1))
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64, "steps": 1, "warmup": 1, "dtype": "f64",
                "roofline": {"bound": "alu", "achieved": OPS_PER_CELL_UPDATE["f64"] * krate64 / 1e12,
                             "peak": fp64_pipe_peak_tops(), "unit": "Tops/s (FP64 pipe ops)",
                             "frac": OPS_PER_CELL_UPDATE["f64"] * krate64 / 1e12 / fp64_pipe_peak_tops(),
                             "kernel": f"k_tb<double,K={o64['cells_per_lane']},interior>",
                             "peak_source": "measured FP64 FMA-chain throughput (0.60 T DFMA/s)"},
                "hbm_effective": {"achieved": B_ALG["f64"] * krate64 / 1e9, "peak": hbm_peak,
                                  "frac": B_ALG["f64"] * krate64 / 1e9 / hbm_peak, "unit": "GB/s"}}

    # ---- adjoint: 64 trainable profiles of 65536 cells ----
    adjoint = None
    if not args.no_adjoint:
        adjoint = measure_adjoint(args)

    # ---- 3D scale-up: 512^3 plasma sphere ----
    cfg3d = None
    if not args.no_3d:
        cfg3d = measure_3d(args, hbm_peak)

    # ---- the paper's slab (config 1) and the Table 2 sweep ----
    c1 = None
    if not args.no_c1 and rank == 0:
        c1 = measure_c1(args)

    # ---- ragged batch: 4096 slabs ----
    batch = None
    if not args.no_batch:
        batch = measure_batch(args)

    # ---- 2D TMz/TEz ----
    two_d = None
    if not args.no_2d and rank == 0:
        two_d = measure_2d(args, hbm_peak)

    # ---- Eq. 9, Eq. 10 and the split-field PML on the long slab ----
    variants = None
    if not args.no_variants and rank == 0:
        variants = measure_variants(args)

    # ---- CPU oracle baseline (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        steps_per = args.cpu_steps or 60
        v, cores, times = cpu_baseline(slab, steps_per, 2, warm=0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"2 x {steps_per}-step prefixes of the same workload on all {slab.nz} cells (FP64, "
                         f"OpenMP build, per-call coefficient setup included), {sum(times):.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "nz": slab.nz, "steps_per_run": slab.steps,
                           "cell_updates_per_step": cells, "parallelism": f"replicas x{ws}",
                           "l2": "inputs larger than L2 (fields 2x192 MiB + coefficients 384 MiB FP32)",
                           "variant": f"temporally blocked warp tiles, K={opt_used['cells_per_lane']}, "
                                      f"{opt_used['tb_steps']} steps/pass, {opt_used['warps_per_block']} warps/CTA",
                           "precision": "FP32 fields, FP64-derived delta coefficients, Kahan-FP32 DFT blocks into FP64"},
                "roofline": roofline, "hbm_roofline_effective": hbm_eff, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "fp64": fp64, "paper_slab_c1": c1, "batched": batch, "adjoint": adjoint,
                "sphere_3d": cfg3d, "two_d": two_d, "variants": variants,
                "cpu_baseline": cpu,
                "adjoint_forward_ratio": adjoint["ratio"] if adjoint else None}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


PROFILE_CASES = ("c2-tiled-f32", "c2-tiled-f64", "c2-plain-f32", "c2-plain-f64", "c2-eq10-f32", "c2-eq10-f64",
                 "c1-resident-f64",
                 "c1-resident-f32", "c3-batch", "c3-batch-persist", "c4-adjoint", "c4-adjoint-full", "c5-sphere", "2d-tm-f32",
                 "2d-te-f32", "2d-tm-f64")


def run_profile_case(args):
    """One short run of a workload for an ncu capture (no timing, no JSON): the commands under
    profiles/ run these. c2-*: the long slab (--nz cells), --profile-steps steps after one
    warm-up pass; c1-*: the paper's slab, one whole run; c3-batch: the ragged batch with its tuned
    tile shape (K = 12, 32 steps per pass), 64 + 128 steps; c4-adjoint: 8 profiles of the adjoint
    workload, 4096 steps, checkpoint every 512, forward and adjoint (c4-adjoint-full: the whole
    workload, 64 profiles and 30000 steps); c5-sphere: the sphere on an
    --n3d grid for --steps3d steps; 2d-*: the 2D bench grid (4096 x 16384) for --profile-steps
    steps."""
    import torch

    from paper_1709_00821_gb300 import rketd as rk
    from paper_1709_00821_gb300 import workloads as wl

    torch.cuda.set_device(0)
    case = args.profile
    if case.startswith("c2-"):
        _, variant, prec = case.split("-")
        slab = wl.c2_epstein(nz=args.nz, steps=args.run_steps)
        if variant == "eq10":  # Eq. 10 read literally: the plain kernels
            slab.scheme = wl.SCHEME_ETD2
        opts = {"variant": 2 if variant == "tiled" else 1, "use_graphs": 2}
        opts.update(parse_options(args.options))
        with rk.Context(slab, prec, options=opts) as ctx:
            warm = ctx.options()["tb_steps"] if variant == "tiled" else 1
            ctx.step(warm)
            ctx.step(args.profile_steps)
            ctx.sync()
    elif case.startswith("c1-"):
        prec = case.split("-")[2]
        s = wl.c1_plain_slab()
        with rk.Context(s, prec) as ctx:
            ctx.step(s.steps)
            ctx.spectra()
    elif case == "c3-batch":
        b = wl.c3_batch()
        with rk.Context(b.slabs, "f32", options={"cells_per_lane": 12, "tb_steps": 32, "warps_per_block": 2,
                                                 "use_graphs": 2}) as ctx:
            ctx.step(64)
            ctx.step(128)
            ctx.sync()
    elif case == "c3-batch-persist":
        # the persistent variant on the batch: one launch of 16 passes after a one-pass warm-up
        b = wl.c3_batch()
        with rk.Context(b.slabs, "f32", options={"variant": 4, "cells_per_lane": 16, "tb_steps": 32,
                                                 "use_graphs": 2}) as ctx:
            ctx.step(32)
            ctx.step(512 - 32)
            ctx.sync()
    elif case in ("c4-adjoint", "c4-adjoint-full"):
        full = case == "c4-adjoint-full"
        n_prof, steps = (64, 30000) if full else (8, 4096)
        profs = [wl.c4_profile(i, steps=steps) for i in range(n_prof)]
        with rk.Context(profs, "f32") as ctx:
            ctx.forward_ckpt(steps, 512)
            X = ctx.spectra()
            gX = np.zeros_like(X)
            gX[:, 0] = np.conj(X[:, 0]) / np.abs(X[:, 0]).max()
            n = sum(p.nz for p in profs)
            gw = torch.empty(n, dtype=torch.float64, device="cuda")
            gn = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.adjoint(np.ascontiguousarray(gX.real), np.ascontiguousarray(gX.imag), 2048, 6144, gw, gn)
            ctx.sync()
    elif case.startswith("2d-"):
        _, pol, prec = case.split("-")
        p = wl.slab_2d(4096, 16384, pol, mode=16, steps=args.profile_steps)
        with rk.Context2D(p, prec) as ctx:
            ctx.step(args.profile_steps)
            ctx.sync()
    elif case == "c5-sphere":
        p = wl.sphere_problem(n=args.n3d, steps=args.steps3d, box_in=args.box3d)
        with rk.Context3D(p, "f32", k_chunk=args.kc3d or None) as ctx:
            print(json.dumps({"n3d": args.n3d, "tile_planes_per_step": ctx.work()}), flush=True)
            ctx.step(args.steps3d)
            ctx.sync()
    print(f"profile case {case} done", flush=True)


def main():
    args = parse()
    if args.profile:
        run_profile_case(args)
        return
    if args.only_3d:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps(measure_3d(args, peaks()[0])), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
