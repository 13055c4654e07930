#!/usr/bin/env python
"""Throughput of the RR stream-and-collide step on GB300 (one JSON line on stdout).

Workload: the doubly periodic shear layer of Sec. III.B at Re = 3e4, Ma = 0.1,
on 1024^2 grids, one grid per lattice: D2Q9 (2nd-order equilibrium), D2V17
(3rd order) and D2V37 (4th order), RR collision, FP32 compute and FP32
storage.  One bench step advances all three grids by one time step, as one
batch (lbm_batch_step: a single kernel launch per step, graph-replayed).
`value` is the aggregate GLUPS (cells updated per second, all lattices, all
ranks); per-lattice GLUPS (each grid stepped by its own context), HBM
roofline fractions and the low-precision
(shifted FP16 / BF16) and FP64 variants are reported alongside, with further
sections (4096^2 grids, finite-difference a1, accuracy, batched sweep, learned
closure, stability map, and the 3D lattices of Tab. II on a 256^3 Taylor-Green
vortex) after the timed headline steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the method written plainly in C)
on the host cores for the same workload, on a bounded band of rows.
Under torchrun each rank runs the full workload on its own GPU (weak scaling,
no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import signal
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1704_04413_gb300 import workloads as wl  # noqa: E402

GRID = 1024
RE, MACH = 3e4, 0.1
LATTICES = (("D2Q9", 2), ("D2V17", 3), ("D2V37", 4))
# Launch order of the timed headline steps: the dominant D2V37 kernel follows the lattice that writes the
# fewest bytes (D2Q9, 38 MB), so it starts with the fewest of another grid's dirty lines in L2 to write back.
HEADLINE_ORDER = ("D2V17", "D2Q9", "D2V37")
BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "i16": 2}
METRIC = "RR stream-collide GLUPS & HBM-roofline fraction per lattice; low-prec vs FP32"
REF_BAND = 128  # rows of the oracle's sample band
PROFILE = os.path.join(ROOT, "profiles", "batch_rr_f32_3x1024.txt")
PROFILE_SOURCES = ("lattice.cuh", "collide.cuh", "step.cuh", "vec2.cuh", "batch.cu")


def kernel_source_hash(files=PROFILE_SOURCES) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1704_04413_gb300", "csrc")
    for fn in files:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(path=PROFILE):
    """dram bytes per launch of the timed kernel (the batched three-lattice step) from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.path = "/tmp/lbm_clocks_%d_%d.csv" % (os.getpid(), index)
        self.proc = None
        self.index = index
        self.window = None

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __enter__(self):
        q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.send_signal(signal.SIGTERM)
            self.proc.wait()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        if self.window:  # keep the samples taken inside the timed region (host wall clock, 0.1 s slack)
            import datetime
            def ts(r):
                try:
                    return datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    return None
            inside = [r for r in rows if ts(r) is not None and self.window[0] - 0.1 <= ts(r) <= self.window[1] + 0.1]
            rows = inside or rows[-1:]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def shear_fields(name, L):
    from paper_1704_04413_gb300 import lbm
    V, cx, cy, w, cs2 = lbm.lbm_lattice_info(name)
    u0, nu, _ = wl.shear_layer_params(L, np.sqrt(cs2), MACH, RE)
    return V, cs2, nu, wl.double_shear_layer(L, u0)


def make_contexts(storage, stream, grid=GRID, a1_source=0, only=None):
    from paper_1704_04413_gb300 import lbm
    ctxs = []
    for name, neq in LATTICES:
        if only and name != only:
            continue
        V, cs2, nu, fl = shear_fields(name, grid)
        p = lbm.make_params(name, grid, grid, nu=nu, collision="rr", hermite_order=neq, storage=storage,
                            stream=stream, a1_source=a1_source)
        ctx = lbm.lbm_create(p)
        lbm.lbm_init(ctx, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
        ctxs.append((name, V, ctx, fl if grid == GRID else None))
    return ctxs


def make_batch(storage, stream, grid=GRID, launch=None):
    """The three lattices' shear layers as one batch (lbm_batch_*): one kernel launch per step; the
    launch shape from the library's autotuner (run before the initial state is set), or `launch` =
    (threads, rows per item, blocks per SM) when given."""
    from paper_1704_04413_gb300 import lbm
    ps, fields = [], []
    for name, neq in LATTICES:
        V, cs2, nu, fl = shear_fields(name, grid)
        ps.append(lbm.make_params(name, grid, grid, nu=nu, collision="rr", hermite_order=neq, storage=storage,
                                  stream=stream))
        fields.append(fl)
    b = lbm.lbm_batch_create(ps)
    if launch:
        lbm.lbm_batch_set_launch(b, *launch)
    else:
        lbm.lbm_batch_autotune(b, 3)
    ctxs = [lbm.lbm_batch_context(b, i) for i in range(len(ps))]
    for c, fl in zip(ctxs, fields):
        lbm.lbm_init(c, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
    return b, ctxs


def timed_batch_steps(b, steps, warmup, stream_t):
    """Whole-region ms of `steps` batched steps (graph replays of the one-launch step) after `warmup`."""
    import torch
    from paper_1704_04413_gb300 import lbm
    lbm.lbm_batch_step(b, warmup + (warmup % 2))
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    w0 = time.time()
    t0.record(stream_t)
    lbm.lbm_batch_step(b, steps)
    t1.record(stream_t)
    torch.cuda.synchronize()
    w1 = time.time()
    return t0.elapsed_time(t1), (w0, w1)


def timed_steps(ctxs, steps, warmup, stream_t):
    """Per-lattice kernel ms (events around each launch) and the whole-region ms."""
    import torch
    from paper_1704_04413_gb300 import lbm
    for _ in range(warmup):
        for _, _, ctx, _ in ctxs:
            lbm.lbm_step(ctx, 1)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
          for _ in ctxs]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    w0 = time.time()
    t0.record(stream_t)
    for k in range(steps):
        for j, (_, _, ctx, _) in enumerate(ctxs):
            ev[j][k][0].record(stream_t)
            lbm.lbm_step(ctx, 1)
            ev[j][k][1].record(stream_t)
    t1.record(stream_t)
    torch.cuda.synchronize()
    w1 = time.time()
    per = [float(np.mean([a.elapsed_time(b) for a, b in ev[j]])) for j in range(len(ctxs))]
    return per, t0.elapsed_time(t1), (w0, w1)


def e2e_bench(args, st, stream_t):
    """The headline metric end to end through the public C ABI: every step, each lattice's fields are
    copied in from pinned host memory (lbm_init with host rho, u, grad u), stepped (lbm_step) and its
    moments copied back to pinned host memory (lbm_moments).  Each lattice has its own context, stream and
    host thread, so one lattice's transfers overlap another's (ctypes releases the GIL during the calls;
    lbm_init and lbm_moments synchronize only their own stream)."""
    import threading
    import torch
    from paper_1704_04413_gb300 import lbm
    streams = [torch.cuda.Stream() for _ in LATTICES]
    ctxs = [make_contexts("f32", s.cuda_stream, only=name)[0] for s, (name, _) in zip(streams, LATTICES)]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hosts = []
    for name, V, ctx, fl in ctxs:
        hosts.append((ctx, pin(fl.rho), pin(fl.ux), pin(fl.uy), pin(fl.grad_u),
                      [torch.empty((GRID, GRID), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]))
    steps = max(3, min(args.steps, 10))

    def worker(h, n, start, errs):
        ctx, r, u, v, g, outs = h
        start.wait()
        try:
            for _ in range(n):
                lbm.lbm_init(ctx, r, u, v, None, g)
                lbm.lbm_step(ctx, 1)
                lbm.lbm_moments(ctx, outs[0], outs[1], outs[2])
        except Exception as e:  # reported below
            errs.append(e)

    def run(n):
        start, errs = threading.Barrier(len(hosts) + 1), []
        ts = [threading.Thread(target=worker, args=(h, n, start, errs)) for h in hosts]
        for t in ts:
            t.start()
        torch.cuda.synchronize()
        start.wait()
        t0 = time.perf_counter()
        for t in ts:
            t.join()
        torch.cuda.synchronize()
        if errs:
            raise errs[0]
        return time.perf_counter() - t0

    run(1)  # warm-up (first host transfers, work areas)
    e2e_s = run(steps)
    h2d = sum(r.nbytes + u.nbytes + v.nbytes + g.nbytes for _, r, u, v, g, _ in hosts)
    d2h = sum(sum(o.nbytes for o in outs) for *_, outs in hosts)
    for _, _, ctx, _ in ctxs:
        lbm.lbm_destroy(ctx)
    ncell = GRID * GRID
    return {"value": round(len(hosts) * ncell * steps / max(e2e_s, 1e-9) / 1e9, 4), "unit": "GLUPS",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "path": "per lattice, own stream and host thread: lbm_init(pinned host rho,u,grad_u) + lbm_step(1) + "
                    "lbm_moments(pinned host) every step"}


def job_time_ms(total_ms, world, device="cuda"):
    """Time of the whole job's timed region: the maximum over ranks (each rank timed its own region between
    barriers); one rank: its own time."""
    if world == 1:
        return total_ms
    import torch
    torch.distributed.barrier()
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_glups(cells_per_step, steps, world, total_ms):
    """Whole-job throughput: the cells every rank updated over the job's time (replicas: each rank the same)."""
    return cells_per_step * steps * world / (total_ms * 1e-3) / 1e9


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1704_04413_gb300 import lbm
    lbm.load()
    torch.cuda.set_device(local_rank)
    stream_t = torch.cuda.Stream()
    torch.cuda.set_stream(stream_t)
    st = stream_t.cuda_stream
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "measured" if peaks else "fallback"
    ncell = GRID * GRID

    # ---- headline: FP32 compute + storage, RR, the three lattices' grids as one batch (one launch a step) ----
    b, bctx = make_batch("f32", st)
    if world > 1:
        torch.distributed.barrier()
    with Clocks(local_rank) as clk:
        total_ms, window = timed_batch_steps(b, args.steps, args.warmup, stream_t)
        clk.mark(*window)
    total_ms = job_time_ms(total_ms, world)
    threads, rows, bps = lbm.lbm_batch_get_launch(b)
    lbm.lbm_batch_destroy(b)
    ms_per_step = total_ms / args.steps
    value = job_glups(len(LATTICES) * ncell, args.steps, world, total_ms)
    # dominant (and only) kernel of the timed region: the batched step, one launch per step
    dom_bytes = sum(2 * V * BYTES["f32"] * ncell for V in (9, 17, 37))
    achieved = dom_bytes / (ms_per_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "traffic": profiled_traffic(),
                "kernel": "k_batch<RR,f32,with D2V37>: D2Q9 + D2V17 + D2V37 1024^2 in one launch",
                "algorithmic_bytes": dom_bytes, "launch_duration_us": round(ms_per_step * 1e3, 2),
                "launch": {"threads": threads, "rows_per_item": rows, "blocks_per_sm": bps or "one block per item"},
                "peak_source": peak_src + " hbm_gbs (copy)"}
    # ---- per lattice: each grid stepped by its own context (the single-grid kernels), interleaved ----
    ctxs = [make_contexts("f32", st, only=name)[0] for name in HEADLINE_ORDER]
    per, _, _ = timed_steps(ctxs, min(args.steps, 200), args.warmup, stream_t)
    per_lattice = {}
    for (name, V, ctx, _), ms in zip(ctxs, per):
        glups = ncell / (ms * 1e-3) / 1e9
        gbs = glups * 2 * V * BYTES["f32"]
        per_lattice[name] = {"f32": {"glups": round(glups, 3), "ms": round(ms, 5), "gbs": round(gbs, 1),
                                     "frac": round(gbs / hbm_peak, 4)}}
    sec = set(args.sections.split(","))
    # ---- e2e through the C ABI with host buffers (pinned), every step: init from host, step, moments to host ----
    e2e = e2e_bench(args, st, stream_t) if "e2e" in sec else None
    for _, _, ctx, _ in ctxs:
        lbm.lbm_destroy(ctx)

    # ---- low precision (shifted FP16 / BF16 storage) and FP64, same workload ----
    other = (("f16", args.steps), ("bf16", args.steps), ("f64", max(2, min(args.steps // 10, 50))))
    for storage, k in (other if "storages" in sec else ()):
        cs = make_contexts(storage, st)
        per_s, _, _ = timed_steps(cs, k, min(args.warmup, 2), stream_t)
        for (name, V, ctx, _), ms in zip(cs, per_s):
            glups = ncell / (ms * 1e-3) / 1e9
            gbs = glups * 2 * V * BYTES[storage]
            per_lattice[name][storage] = {"glups": round(glups, 3), "ms": round(ms, 5), "gbs": round(gbs, 1),
                                          "frac": round(gbs / hbm_peak, 4),
                                          "vs_f32": round(glups / per_lattice[name]["f32"]["glups"], 3)}
            lbm.lbm_destroy(ctx)

    # ---- RR with a1 from finite differences (a moments pass + the step per lattice per step), FP32 ----
    fd = {}
    if "fd" in sec:
        cs = make_contexts("f32", st, a1_source=1)
        per_s, _, _ = timed_steps(cs, max(10, min(args.steps, 200)), 3, stream_t)
        for (name, V, ctx, _), ms in zip(cs, per_s):
            glups = ncell / (ms * 1e-3) / 1e9
            fd[name] = {"glups": round(glups, 3), "ms": round(ms, 5),
                        "vs_projection": round(glups / per_lattice[name]["f32"]["glups"], 3)}
            lbm.lbm_destroy(ctx)
    # ---- above-L2 grids: consecutive steps of one 4096^2 grid (buffers 0.6-5 GB, far above the 129 MB L2) ----
    large = {}
    if "large" in sec:
        for storage in ("f32", "f16", "bf16"):
            for name, V, ctx, _ in make_contexts(storage, st, grid=4096):
                per_s, _, _ = timed_steps([(name, V, ctx, None)], 20, 3, stream_t)
                glups = 4096 * 4096 / (per_s[0] * 1e-3) / 1e9
                gbs = glups * 2 * V * BYTES[storage]
                large.setdefault(name, {})[storage] = {"glups": round(glups, 3), "gbs": round(gbs, 1),
                                                       "frac": round(gbs / hbm_peak, 4)}
                lbm.lbm_destroy(ctx)
        for name in large:
            for storage in ("f16", "bf16"):
                large[name][storage]["vs_f32"] = round(large[name][storage]["glups"] / large[name]["f32"]["glups"], 3)
    # compact roofline map kept in the headline object: GLUPS and fraction of the measured copy per lattice
    # and storage, at 1024^2 (the benchmark's interleaved steps) and 4096^2 (one grid, far above L2)
    roofline["per_lattice"] = {
        name: {"1024": {st_: [v["glups"], v["frac"]] for st_, v in per_lattice[name].items()},
               "4096": {st_: [v["glups"], v["frac"]] for st_, v in large.get(name, {}).items()}}
        for name in per_lattice}
    accuracy = accuracy_vs_f64(st) if "accuracy" in sec else None
    batched = batched_sweep_bench(stream_t, steps=max(10, min(args.steps, 200))) if "batched" in sec else None
    closure = closure_bench(stream_t, fine=2048, reynolds=1e6) if "closure" in sec else None
    stab = stability_bench(st) if "stability" in sec else None
    d3 = d3_bench(stream_t) if "d3" in sec else None

    line = {"metric": METRIC, "value": round(value, 3), "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "double shear layer Re=3e4 Ma=0.1 (kappa=80, delta=0.05), 1024x1024 periodic; "
                                   "one step = one batched launch (lbm_batch_step) over the D2Q9 (N=2), D2V17 "
                                   "(N=3) and D2V37 (N=4) grids, RR, FP32",
                       "grid": GRID, "lattices": [n for n, _ in LATTICES], "collision": "rr",
                       "storage": "f32", "parallelism": "replicas" if world > 1 else "single",
                       "l2": "not flushed: each step moves 528 MB (the three grids' 75/143/310 MB pairs of "
                             "buffers), above the 129 MB L2"},
            "roofline": roofline, "per_lattice": per_lattice, "e2e": e2e,
            "per_lattice_4096": large, "a1_finite_difference_f32": fd, "accuracy_vs_f64_gpu": accuracy, "batched_sweep": batched,
            "learned_closure": closure, "stability_map": stab, "lattices_3d": d3,
            "gpu_launches": args.steps, "clocks": clk.summary()}
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(min_seconds=10.0) if "cpu" in sec else None
        print(json.dumps(line), flush=True)


LATTICES3 = (("D3Q19", 2), ("D3Q27", 3), ("D3V39", 3), ("D3Q103", 4))


def d3_bench(stream_t, steps=20, n=256, storages=("f32", "f16"), only=None):
    """Fused stream + RR step of the Tab. II lattices on a periodic n^3 Taylor-Green vortex (Ma = 0.1,
    Re = 1600 on the length n / 2 pi), consecutive steps of one grid (buffers 2.5-14 GB, far above L2).
    GLUPS, HBM bytes 2 V sizeof(storage) per cell and their fraction of the measured copy bandwidth."""
    import torch
    from paper_1704_04413_gb300 import lbm
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    nx, ny, nz = (n, n, n) if isinstance(n, int) else n
    rho, u1, g1 = wl.taylor_green_3d(n, 1.0) if isinstance(n, int) else wl.taylor_green_3d_box(nx, ny, nz, 1.0)
    out = {"grid": [nx, ny, nz], "workload": "3D Taylor-Green vortex, Ma=0.1, Re=1600, periodic, RR"}
    ncell = nx * ny * nz
    for name, neq in LATTICES3:
        if only and name not in only:
            continue
        V, cx, cy, cz, w, cs2 = lbm.lbm3_lattice_info(name)
        u0 = MACH * np.sqrt(cs2)
        nu = u0 * nx / (2 * np.pi) / 1600.0
        res = {"hermite_order": neq}
        for storage in storages:
            p = lbm.make_params3(name, nx, ny, nz, nu=nu, collision="rr", hermite_order=neq, storage=storage,
                                 stream=stream_t.cuda_stream)
            ctx = lbm.lbm3_create(p)
            lbm.lbm3_init(ctx, rho, u0 * u1, u0 * g1)
            for _ in range(3):
                lbm.lbm3_step(ctx, 1)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            torch.cuda.synchronize()
            for a, b in ev:
                a.record(stream_t)
                lbm.lbm3_step(ctx, 1)
                b.record(stream_t)
            torch.cuda.synchronize()
            ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
            glups = ncell / (ms * 1e-3) / 1e9
            gbs = glups * 2 * V * BYTES[storage]
            res[storage] = {"glups": round(glups, 3), "ms": round(ms, 4), "gbs": round(gbs, 1),
                            "frac": round(gbs / hbm_peak, 4)}
            lbm.lbm3_destroy(ctx)
        if "f16" in res and "f32" in res:
            res["f16"]["vs_f32"] = round(res["f16"]["glups"] / res["f32"]["glups"], 3)
        out[name] = res
    return out


def batched_sweep_bench(stream_t, steps, n=64, storage="f16"):
    """64 shear-layer instances (sizes uniform over {128..1024}^2, Re log-uniform in [1e4, 1e6], D2Q9 / D2V17
    alternating, shifted FP16 storage): autotuned persistent graph-captured batch vs one launch per instance."""
    import torch
    from paper_1704_04413_gb300 import lbm
    st = stream_t.cuda_stream
    insts = wl.batched_sweep(n, seed=0)
    ps, fields = [], []
    for inst in insts:
        V, cx, cy, w, cs2 = lbm.lbm_lattice_info(inst.lattice)
        u0, nu, _ = wl.shear_layer_params(inst.L, np.sqrt(cs2), MACH, inst.reynolds)
        ps.append(lbm.make_params(inst.lattice, inst.L, inst.L, nu=nu, collision="rr",
                                  hermite_order=2 if inst.lattice == "D2Q9" else 3, storage=storage, stream=st))
        fields.append(wl.double_shear_layer(inst.L, u0))
    b = lbm.lbm_batch_create(ps)
    try:
        tune_ms = lbm.lbm_batch_autotune(b, 3)
        ctxs = [lbm.lbm_batch_context(b, i) for i in range(n)]
        for c, fl in zip(ctxs, fields):
            lbm.lbm_init(c, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
        cells = sum(i.L * i.L for i in insts)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        lbm.lbm_batch_step(b, 4)
        torch.cuda.synchronize()
        e[0].record(stream_t)
        lbm.lbm_batch_step(b, steps)
        e[1].record(stream_t)
        for c in ctxs:
            lbm.lbm_step(c, 2)
        torch.cuda.synchronize()
        e[2].record(stream_t)
        for _ in range(steps):
            for c in ctxs:
                lbm.lbm_step(c, 1)
        e[3].record(stream_t)
        torch.cuda.synchronize()
        t_b, t_s = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
        t, r, q = lbm.lbm_batch_get_launch(b)
        return {"instances": n, "cells": cells, "storage": storage, "collision": "rr",
                "sizes": sorted({i.L for i in insts}), "steps": steps,
                "launch": {"threads": t, "rows_per_item": r, "blocks_per_sm": q or "one block per item"},
                "autotune_best_ms_per_step": round(tune_ms, 4),
                "batched_glups": round(cells * steps / (t_b * 1e-3) / 1e9, 3),
                "per_instance_launch_glups": round(cells * steps / (t_s * 1e-3) / 1e9, 3),
                "speedup": round(t_s / t_b, 3)}
    finally:
        lbm.lbm_batch_destroy(b)


def closure_forward_bench(stream_t, n=1 << 22, reps=10):
    """Inference throughput of the closure network alone (lbm_closure_forward, tcgen05) on n rows of seeded
    random BF16 features with the seeded initial weights: the profiling case of its kernel."""
    import torch
    from paper_1704_04413_gb300 import lbm
    st = stream_t.cuda_stream
    cl = lbm.lbm_closure_create()
    try:
        lbm.lbm_closure_set_weights(cl, wl.closure_initial_weights(3, out_scale=1.0))
        g = torch.Generator(device="cuda").manual_seed(5)
        x = (0.5 * torch.randn((n, lbm.CLOSURE_IN), device="cuda", generator=g)).to(torch.bfloat16)
        y = torch.empty((n, lbm.CLOSURE_OUT), dtype=torch.float32, device="cuda")
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for _ in range(3):
            lbm.lbm_closure_forward(cl, x, n, y, st)
        e[0].record(stream_t)
        for _ in range(reps):
            lbm.lbm_closure_forward(cl, x, n, y, st)
        e[1].record(stream_t)
        torch.cuda.synchronize()
        ms = e[0].elapsed_time(e[1]) / reps
    finally:
        lbm.lbm_closure_destroy(cl)
    flops = 2 * (lbm.CLOSURE_IN * lbm.CLOSURE_HID + 2 * lbm.CLOSURE_HID ** 2 + lbm.CLOSURE_HID * lbm.CLOSURE_OUT)
    return {"closure_forward": {"rows": n, "ms": round(ms, 4), "tflops": round(flops * n / ms / 1e9, 2)}}


def closure_step_bench(stream_t, n=256, steps=200):
    """The fused closure step alone (lbm_step_closure: moments pass + tensor-core network + corrected
    collision) on an n^2 D2Q9 shear layer with the seeded initial weights: the profiling case of its kernels."""
    import torch
    from paper_1704_04413_gb300 import lbm
    st = stream_t.cuda_stream
    u0 = 0.05
    c = lbm.lbm_create(lbm.make_params("D2Q9", n, n, tau=0.51, collision="rr", hermite_order=2, storage="f32",
                                       stream=st))
    cl = lbm.lbm_closure_create()
    try:
        lbm.lbm_closure_set_weights(cl, wl.closure_initial_weights(3, out_scale=0.1))
        fl = wl.double_shear_layer(n, u0)
        lbm.lbm_init(c, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        lbm.lbm_step_closure(c, cl, u0, 3)
        e[0].record(stream_t)
        lbm.lbm_step_closure(c, cl, u0, steps)
        e[1].record(stream_t)
        torch.cuda.synchronize()
        ms = e[0].elapsed_time(e[1]) / steps
    finally:
        lbm.lbm_closure_destroy(cl)
        lbm.lbm_destroy(c)
    return {"closure_step": {"grid": n, "us_per_step": round(1000 * ms, 2), "glups": round(n * n / ms / 1e6, 3)}}


def closure_bench(stream_t, fine=1024, factor=8, reynolds=1e5, seeds=4, held_out=3, epochs=20):
    """Learned a1^(2) closure: training data from box-filtered fine D2Q9 RR shear layers, Adam training of the
    BF16 tensor-core MLP, then the coarse grid run from the filtered initial state with and without the
    closure, scored against the filtered fine run by the vorticity-spectrum error and the pointwise
    vorticity relative L2 error (lower is better), each averaged over the snapshots; reported for the first
    training seed and as mean and spread over `held_out` seeds kept out of training.  A gain is stated per
    metric, only where the closure's mean is lower."""
    import torch
    from paper_1704_04413_gb300 import closure_pipeline as cp
    from paper_1704_04413_gb300 import lbm
    st = stream_t.cuda_stream
    data = cp.generate(fine, factor, reynolds, seeds=range(seeds), stream=st,
                       held_out=range(100, 100 + held_out))
    cl, losses, train_s = cp.train(data, epochs=epochs)
    try:
        res = cp.compare(data, cl, stream=st)
        res_held = {sd: cp.compare(data, cl, stream=st, truth=t) for sd, t in data.held_out.items()}
        # inference and closure-step throughput on 4M samples / the coarse grid
        n = 1 << 22
        x = data.x[torch.arange(n, device="cuda") % data.x.shape[0]].contiguous()
        y = torch.empty((n, lbm.CLOSURE_OUT), dtype=torch.float32, device="cuda")
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for _ in range(3):
            lbm.lbm_closure_forward(cl, x, n, y, st)
        e[0].record(stream_t)
        for _ in range(10):
            lbm.lbm_closure_forward(cl, x, n, y, st)
        e[1].record(stream_t)
        torch.cuda.synchronize()
        fwd_ms = e[0].elapsed_time(e[1]) / 10
        flops = 2 * (lbm.CLOSURE_IN * lbm.CLOSURE_HID + 2 * lbm.CLOSURE_HID ** 2 + lbm.CLOSURE_HID * lbm.CLOSURE_OUT)
        nc = data.coarse
        rates = {}
        for mode in ("plain", "closure"):
            c = lbm.lbm_create(lbm.make_params("D2Q9", nc, nc, nu=data.nu_coarse, collision="rr", hermite_order=2,
                                               storage="f32", stream=st))
            try:
                fl = wl.double_shear_layer(nc, data.u0)
                lbm.lbm_init(c, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
                step = (lambda k: lbm.lbm_step(c, k)) if mode == "plain" else \
                    (lambda k: lbm.lbm_step_closure(c, cl, data.u0, k))
                step(5)
                e[0].record(stream_t)
                step(200)
                e[1].record(stream_t)
                torch.cuda.synchronize()
                rates[mode] = nc * nc * 200 / (e[0].elapsed_time(e[1]) * 1e-3) / 1e9
            finally:
                lbm.lbm_destroy(c)
    finally:
        lbm.lbm_closure_destroy(cl)
    var = float(data.y[:, :3].var(dim=0).sum().item())
    mean = lambda mode, key: round(float(np.mean([r[key] for r in res[mode]])), 4)
    held = {}
    for key in ("spectrum_err", "vorticity_rel_l2"):
        per_seed = {m: [float(np.mean([r[key] for r in rs[m]])) for rs in res_held.values()] for m in ("plain", "closure")}
        held[key] = {m: {"mean": round(float(np.mean(v)), 4), "std": round(float(np.std(v, ddof=1)), 4) if len(v) > 1
                         else 0.0, "per_seed": [round(x, 4) for x in v]} for m, v in per_seed.items()}
        held[key]["closure_lower"] = held[key]["closure"]["mean"] < held[key]["plain"]["mean"]
    return {"fine": fine, "coarse": data.coarse, "reynolds": reynolds, "seeds": seeds,
            "samples": int(data.x.shape[0]), "generate_s": round(data.seconds, 2),
            "train": {"epochs": epochs, "batch": 4096, "seconds": round(train_s, 2),
                      "samples_per_s": round(epochs * data.x.shape[0] / train_s, 0),
                      "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1], "target_variance": var},
            "forward": {"samples": n, "ms": round(fwd_ms, 4), "samples_per_s": round(n / (fwd_ms * 1e-3), 0),
                        "tflops": round(flops * n / (fwd_ms * 1e-3) / 1e12, 2)},
            "coarse_step_glups": {k: round(v, 3) for k, v in rates.items()},
            "training_seed_0": {
                "spectrum_err_mean": {"plain_rr": mean("plain", "spectrum_err"), "closure": mean("closure", "spectrum_err")},
                "vorticity_rel_l2_mean": {"plain_rr": mean("plain", "vorticity_rel_l2"),
                                          "closure": mean("closure", "vorticity_rel_l2")}},
            "held_out_seeds": held,
            "gain": {"spectrum": held["spectrum_err"]["closure_lower"],
                     "pointwise_vorticity": held["vorticity_rel_l2"]["closure_lower"]}}


def stability_bench(stream, reynolds=(1e4, 3e4, 1e5, 1e6), L=128):
    """M0^max of the double shear layer at L = 128 up to t = 2 t_c (Sec. III.B), FP32 storage, for BGK, the
    projection at every order and the recursive regularization at every order >= 3 with a1 projected
    ("rr<N>") and from finite differences ("rrfd<N>"), per lattice."""
    from paper_1704_04413_gb300 import stability as S
    t0 = time.perf_counter()
    out = S.stability_map(reynolds=reynolds, L=L, stream=stream)
    res = {"grid": L, "reynolds": list(reynolds), "criterion": "<u^2>(t) < <u^2>(0) for t <= 2 t_c, checked every 20 steps",
           "storage": "f32", "dM0": 0.01}
    for lat, d in out.items():
        res[lat] = {k: ({"%g" % re: v[0] if isinstance(v, tuple) else v for re, v in d[k].items()}
                        if isinstance(d[k], dict) else d[k]) for k in d}
    res["seconds"] = round(time.perf_counter() - t0, 1)
    return res


def vorticity(ux, uy):
    """omega = d_x u_y - d_y u_x, fourth-order centred differences, periodic (Sec. III.B)."""
    def d(g, axis):
        return (-np.roll(g, -2, axis) + 8 * np.roll(g, -1, axis) - 8 * np.roll(g, 1, axis)
                + np.roll(g, 2, axis)) / 12.0
    return d(uy, 1) - d(ux, 0)


def accuracy_vs_f64(stream, L=256, storages=("f32", "f16", "bf16", "i16"), checkpoints=8):
    """Relative L2 error of vorticity (and of rho, u) of each storage format against the FP64 GPU run of the
    same lattice, at `checkpoints` equally spaced times up to one convective time t_c = L/u0 of the shear
    layer (the curve) and at t_c.  "f64_perturbed" is the control: the FP64 run with its initial
    populations multiplied by (1 + eta), eta uniform in [-2^-24, 2^-24] (one FP32 rounding), i.e. how the
    flow itself amplifies rounding-size noise injected once."""
    from paper_1704_04413_gb300 import lbm
    out = {}
    for name, neq in LATTICES:
        V, cs2, nu, fl = shear_fields(name, L)
        u0, _, steps = wl.shear_layer_params(L, np.sqrt(cs2), MACH, RE)
        runs = {}
        for storage in ("f64",) + tuple(storages) + ("f64_perturbed",):
            st_fmt = "f64" if storage == "f64_perturbed" else storage
            p = lbm.make_params(name, L, L, nu=nu, collision="rr", hermite_order=neq, storage=st_fmt, stream=stream)
            ctx = lbm.lbm_create(p)
            lbm.lbm_init(ctx, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
            if storage == "f64_perturbed":
                f = np.empty((V, L, L))
                lbm.lbm_get_populations(ctx, f)
                f *= 1.0 + wl.population_noise(V, L, L, seed=11, eps=2.0 ** -24)
                lbm.lbm_set_populations(ctx, f)
            runs[storage] = ctx
        marks = [int(round(steps * (k + 1) / checkpoints)) for k in range(checkpoints)]
        curve = {s_: [] for s_ in runs if s_ != "f64"}
        done, final = 0, {}
        for t in marks:
            fields = {}
            for storage, ctx in runs.items():
                lbm.lbm_step(ctx, t - done)
                r, u, v = (np.empty((L, L)) for _ in range(3))
                lbm.lbm_moments(ctx, r, u, v)
                fields[storage] = (r, u, v, vorticity(u, v))
            done = t
            r0, u0_, v0, w0 = fields["f64"]
            for storage in curve:
                r, u, v, w = fields[storage]
                ok = bool(np.all(np.isfinite(w)))
                curve[storage].append(round(float(np.linalg.norm(w - w0) / np.linalg.norm(w0)), 6) if ok else None)
                if t == marks[-1]:
                    final[storage] = {
                        "vorticity_rel_l2": float(np.linalg.norm(w - w0) / np.linalg.norm(w0)) if ok else None,
                        "u_rel_l2": float(np.linalg.norm(np.hypot(u - u0_, v - v0)) / np.linalg.norm(np.hypot(u0_, v0)))
                        if ok else None,
                        "rho_rel_l2": float(np.linalg.norm(r - r0) / np.linalg.norm(r0)) if ok else None}
        for ctx in runs.values():
            lbm.lbm_destroy(ctx)
        out[name] = {"steps": steps, "grid": L, "t_over_tc": [round(m / steps, 4) for m in marks]}
        for storage in curve:
            out[name][storage] = dict(final[storage], vorticity_rel_l2_vs_t=curve[storage])
    return out


def oracle_sample_step(pairs):
    from oracle import oracle as orc
    for p, f in pairs:
        f[0] = orc.step(p, f[0])


def oracle_setup(band):
    from oracle import oracle as orc
    pairs = []
    for name, neq in LATTICES:
        L = orc.lattice(name)
        u0, nu, _ = wl.shear_layer_params(GRID, np.sqrt(L.cs2), MACH, RE)
        fl = wl.double_shear_layer(GRID, u0)
        rows = slice(GRID // 4 - band // 2, GRID // 4 + band // 2)  # band across the lower shear layer
        p = orc.params(name, GRID, band, orc.tau_from_nu(L.cs2, nu), "rr", neq)
        f = orc.init(p, fl.rho[rows].copy(), fl.ux[rows].copy(), fl.uy[rows].copy(), None,
                     fl.grad_u[:, rows].copy())
        pairs.append((p, [f]))
    return pairs


def cpu_baseline(min_seconds=10.0, max_steps=20):
    from oracle import oracle as orc
    orc.build_oracle()
    pairs = oracle_setup(REF_BAND)
    oracle_sample_step(pairs)  # warm-up
    n = 0
    t0 = time.perf_counter()
    while n < max_steps and (time.perf_counter() - t0) < min_seconds:
        oracle_sample_step(pairs)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": round(len(pairs) * GRID * REF_BAND * n / dt / 1e9, 6), "unit": "GLUPS",
            "cores": orc.num_threads(), "kind": "oracle",
            "sample": "%d steps of a %dx%d periodic band across the lower shear layer, per lattice "
                      "(D2Q9, D2V17, D2V37 RR), FP64 C oracle with OpenMP over rows" % (n, GRID, REF_BAND)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build_oracle()
    pairs = oracle_setup(REF_BAND)
    for _ in range(args.warmup):
        oracle_sample_step(pairs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample_step(pairs)
    dt = time.perf_counter() - t0
    value = len(pairs) * GRID * REF_BAND * args.steps / dt / 1e9
    sample = ("%dx%d periodic band across the lower shear layer per lattice (D2Q9 N=2, D2V17 N=3, D2V37 N=4, "
              "RR), FP64 C oracle with OpenMP over rows" % (GRID, REF_BAND))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "double shear layer Re=3e4 Ma=0.1, 1024-wide grid; one step = one step of "
                                   "each of D2Q9/D2V17/D2V37 RR (oracle on a band of rows)", "grid": GRID,
                       "band_rows": REF_BAND},
            "cpu_baseline": {"value": round(value, 6), "unit": "GLUPS", "cores": orc.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_only(args):
    """One lattice, one storage format: warm-up then timed steps; prints per-step ms (profiling case)."""
    import torch
    from paper_1704_04413_gb300 import lbm
    torch.cuda.set_device(0)
    stream_t = torch.cuda.Stream()
    neq = dict(LATTICES)[args.kernel_only]
    V, cs2, nu, fl = shear_fields(args.kernel_only, args.grid)
    p = lbm.make_params(args.kernel_only, args.grid, args.grid, nu=nu, collision="rr", hermite_order=neq,
                        storage=args.storage, stream=stream_t.cuda_stream)
    ctx = lbm.lbm_create(p)
    lbm.lbm_init(ctx, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
    per, total, _ = timed_steps([(args.kernel_only, V, ctx, fl)], args.steps, args.warmup, stream_t)
    glups = args.grid * args.grid / (per[0] * 1e-3) / 1e9
    print(json.dumps({"kernel_only": args.kernel_only, "grid": args.grid, "storage": args.storage,
                      "ms": per[0], "glups": glups, "gbs": glups * 2 * V * BYTES[args.storage]}))
    lbm.lbm_destroy(ctx)


def headline_only(args):
    """The timed headline alone (profiling case): the three-lattice batch with the launch shape of
    --batch-launch (else autotuned: 16 shapes x 4 launches), `warmup` (rounded up to even) then `steps`
    batched launches; prints ms per step."""
    import torch
    from paper_1704_04413_gb300 import lbm
    torch.cuda.set_device(0)
    stream_t = torch.cuda.Stream()
    launch = tuple(int(v) for v in args.batch_launch.split(",")) if args.batch_launch else None
    b, _ = make_batch(args.storage, stream_t.cuda_stream, launch=launch)
    total_ms, _ = timed_batch_steps(b, args.steps, args.warmup, stream_t)
    t, r, q = lbm.lbm_batch_get_launch(b)
    lbm.lbm_batch_destroy(b)
    print(json.dumps({"headline_only": True, "ms_per_step": total_ms / args.steps, "launch": [t, r, q]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--kernel-only", default=None, metavar="LATTICE",
                    help="profiling case: run only this lattice's RR step (for ncu captures)")
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--storage", default="f32")
    ap.add_argument("--batched-only", action="store_true", help="profiling case: only the batched sweep")
    ap.add_argument("--headline-only", action="store_true",
                    help="profiling case: only the timed headline batch (no other section)")
    ap.add_argument("--batch-launch", default=None, metavar="THREADS,ROWS,BLOCKS_PER_SM",
                    help="launch shape of --headline-only instead of the autotuner's")
    ap.add_argument("--closure-only", action="store_true", help="only the learned-closure section")
    ap.add_argument("--closure-forward-only", action="store_true",
                    help="profiling case: only the closure network's inference on 4M random rows")
    ap.add_argument("--closure-step-only", action="store_true",
                    help="profiling case: only the fused closure step on a 256^2 grid (--steps steps)")
    ap.add_argument("--d3-only", action="store_true",
                    help="only the 3D lattice section (--grid3, --storage as a comma list, --lattices3)")
    ap.add_argument("--grid3", default="256", help="n (an n^3 grid) or nx,ny,nz of the 3D section")
    ap.add_argument("--lattices3", default=None, help="comma list of 3D lattices for --d3-only (default all)")
    ap.add_argument("--sections", default="e2e,storages,fd,large,accuracy,batched,closure,stability,d3,cpu",
                    help="comma list of sections run after the timed headline steps (profiling runs pass "
                         "'none' to keep only the headline)")
    ap.add_argument("--closure-fine", type=int, default=2048)
    ap.add_argument("--closure-re", type=float, default=1e6)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.kernel_only:
        kernel_only(args)
        return
    if args.headline_only:
        headline_only(args)
        return
    if args.batched_only:
        import torch
        torch.cuda.set_device(0)
        stream_t = torch.cuda.Stream()
        torch.cuda.set_stream(stream_t)
        print(json.dumps(batched_sweep_bench(stream_t, steps=args.steps)))
        return
    if args.closure_only:
        import torch
        torch.cuda.set_device(0)
        stream_t = torch.cuda.Stream()
        torch.cuda.set_stream(stream_t)
        print(json.dumps(closure_bench(stream_t, fine=args.closure_fine, reynolds=args.closure_re)))
        return
    if args.closure_step_only:
        import torch
        torch.cuda.set_device(0)
        stream_t = torch.cuda.Stream()
        torch.cuda.set_stream(stream_t)
        print(json.dumps(closure_step_bench(stream_t, steps=max(1, args.steps))))
        return
    if args.closure_forward_only:
        import torch
        torch.cuda.set_device(0)
        stream_t = torch.cuda.Stream()
        torch.cuda.set_stream(stream_t)
        print(json.dumps(closure_forward_bench(stream_t, reps=max(1, args.steps))))
        return
    if args.d3_only:
        import torch
        torch.cuda.set_device(0)
        stream_t = torch.cuda.Stream()
        torch.cuda.set_stream(stream_t)
        only = args.lattices3.split(",") if args.lattices3 else None
        storages = args.storage.split(",")
        n3 = [int(v) for v in args.grid3.split(",")]
        print(json.dumps(d3_bench(stream_t, steps=args.steps, n=n3[0] if len(n3) == 1 else tuple(n3),
                                  storages=storages, only=only)))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
