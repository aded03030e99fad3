#!/usr/bin/env python
"""Throughput benchmark of the TreeRay/RadPressure hot path on GB300.

Workload: 128^3 uniform grid in a 2 pc box, lognormal turbulent density (P(k) ~ k^-4,
sigma_ln rho = 1.5, mean 1e-20 g/cm^3, seed 2), T_d ~ U[10, 40] K (seed 3), Planck-mean
opacity 0.1 (T/10 K)^2 cm^2/g, one 1e5 Lsun star at the box centre; N_pix = 48
(--npix 192 for the second ray count), 20 geometric radial segments, theta = 0.5;
gas temperature U[10, 100] K for the dust balance. Synthetic, seeded.

One step is one pass of the whole hot path through the C ABI: tree build (leaf
quantities, Morton sort, nodes, moments), ray evaluation of every cell (walk, mapping,
integration, finalization), radiation pressure, and the dust-temperature solve.
Metric: target-cell ray evaluations per second = cells x N_pix / step time.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the
launching stream; a 256 MiB buffer is written between steps to flush the 129 MB L2
(outside the events). The evaluate kernel is timed separately for the roofline.
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample.
Under torchrun every rank runs an independent replica (weak scaling, no collective
on the data path); value = cells x N_pix x ranks / max-over-ranks step time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "target-cell ray evaluations/sec (cells x N_pix)"
UNIT = "ray-evals/s"


def workload(npix: int):
    import synth
    w = synth.turbulent_cloud(128, npix=npix)
    return synth.with_gas(w, seed=7, tgas_lo=10.0, tgas_hi=100.0)


def config(npix: int, extra=None):
    c = {"workload": f"turb128_npix{npix}", "cells": 128 ** 3, "grid": "uniform 128^3, box 2 pc",
         "density": "lognormal P(k)~k^-4 sigma_lnrho=1.5 mean 1e-20 g/cm^3",
         "npix": npix, "nbins": 20, "theta": 0.5, "stars": 1,
         "l2": "flushed between steps (256 MiB write); tree rebuilt every step",
         "step": "build+evaluate+radpressure+dust_temperature"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("evaluate.cu", "internal.h"):
        with open(os.path.join(ROOT, "paper_2204_09072_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload_name: str, key: str = "bytes_per_launch"):
    """DRAM bytes (key "bytes_per_launch") or L2 bytes ("lts_bytes_per_launch") per evaluate
    launch from the committed ncu summary, if it was taken on the current kernel source;
    else None."""
    p = os.path.join(ROOT, "profiles", "evaluate_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("kernel_sha") == kernel_source_sha() and workload_name in d.get(key, {}):
            return float(d[key][workload_name])
    except Exception:
        pass
    return None


def job_times(ms_values, dist=None, device="cpu"):
    """Step times of the whole job: each value reduced with MAX over the ranks (every rank
    runs its own replica; the job is as slow as its slowest rank). Without a process group
    the values pass through."""
    if dist is None:
        return [float(x) for x in ms_values]
    import torch
    t = torch.tensor([float(x) for x in ms_values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_value(cells: int, npix: int, world: int, ms: float) -> float:
    """Whole-job ray evaluations per second: `world` replicas of `cells` cells x `npix` rays
    each, in `ms` milliseconds (the slowest rank's step)."""
    return cells * npix * world / (ms * 1e-3)


# Node-stream model of the evaluate kernel (the roofline's algorithmic bytes): every
# visited node's 16 B geometry record (centre, level, first child) and every accepted
# node's two 16 B value records (thin and thick moments, COL offset), own cell included.
NODE_BYTES_VISIT, NODE_BYTES_ACCEPT = 16, 32
# A wider count of the same launch's loads, reported beside it: the angular-kernel tables
# too (8 B offset pair per accepted node but the own cell, 4 B per entry) and per target
# 16 B own geometry, 32 B own values, 8 B map lookups, 8 B J_src and 28 B of outputs.
BYTES_VISIT, BYTES_ACCEPT, BYTES_ENTRY, BYTES_TARGET = 16, 40, 4, 92


def node_stream_bytes(visits: int, accepted: int) -> int:
    return NODE_BYTES_VISIT * visits + NODE_BYTES_ACCEPT * accepted


def time_evaluate(tr, torch, w, dev, steps: int, flush):
    """Evaluate-kernel time (ms, CUDA events on the launching stream, L2 flushed before each
    launch) of one workload, with the autotuner's team size and the walk totals."""
    import numpy as np
    st = torch.cuda.Stream(device=dev)
    ctx = tr.Context(w.params)
    n = w.n_leaves
    with torch.cuda.stream(st):
        rho = torch.as_tensor(w.rho, device=dev)
        td = torch.as_tensor(w.td, device=dev)
        ctx.build(w.box_cm, rho, td, n=w.uniform_n, blocks=w.blocks,
                  star_pos=w.star_pos if len(w.star_lum) else None,
                  star_lum=w.star_lum if len(w.star_lum) else None, stream=st)
        wpt, occ, _, _ = ctx.autotune_launch(65536, stream=st)
        J = torch.empty(n, dtype=torch.float32, device=dev)
        F = torch.empty(3 * n, dtype=torch.float64, device=dev)
        for _ in range(3):
            ctx.evaluate(J, F, stream=st)
        ts = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ctx.evaluate(J, F, stream=st)
            e1.record(st)
            st.synchronize()
            ts.append(e0.elapsed_time(e1))
        ctx.check(st)
        tot = ctx.walk_stats(stream=st).cpu().numpy().astype(np.int64)
    ctx.close()
    ms = statistics.mean(ts)
    visits, acc, ent = (int(x) for x in tot)
    return {"ms": ms, "cells": n, "npix": w.params["npix"], "warps_per_target": wpt, "occupancy_pct": occ,
            "ray_evals_per_s": n * w.params["npix"] / (ms * 1e-3),
            "node_stream_GBps": node_stream_bytes(visits, acc) / (ms * 1e-3) / 1e9,
            "walk": {"visits": visits, "accepted": acc, "alpha_entries": ent}}


def run_ours(args):
    import numpy as np
    import torch

    import paper_2204_09072_gb300 as tr

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tr.lib()
    dev = torch.device("cuda", local)
    w = workload(args.npix)
    n = w.n_leaves
    npix = args.npix
    ctx = tr.Context(w.params)
    st = torch.cuda.Stream(device=dev)
    rho = torch.as_tensor(w.rho, device=dev)
    td = torch.as_tensor(w.td, device=dev)
    tgas = torch.as_tensor(w.tgas, device=dev)
    J = torch.empty(n, dtype=torch.float32, device=dev)
    F = torch.empty(3 * n, dtype=torch.float64, device=dev)
    u = torch.empty(n, dtype=torch.float32, device=dev)
    a_rp = torch.empty(3 * n, dtype=torch.float32, device=dev)
    force = torch.empty(3 * n, dtype=torch.float32, device=dev)
    p_src = torch.empty(n, dtype=torch.float32, device=dev)
    Td = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # one-time set-up outside the timed region: build once and let the autotuner pick the
    # evaluate kernel's warps per target for this tree
    with torch.cuda.stream(st):
        ctx.build(w.box_cm, rho, td, n=w.uniform_n, star_pos=w.star_pos, star_lum=w.star_lum, stream=st)
        if args.wpt:
            # a fixed team size: under a profiler the autotuner's timings are serialised and
            # cold-cache, so a capture pins the choice that the plain run made
            ctx.set_warps_per_target(args.wpt)
            ctx.set_occupancy(100)
            best_wpt, best_occ, tune_ms, tune_occ = args.wpt, 100, None, None
        else:
            best_wpt, best_occ, tune_ms, tune_occ = ctx.autotune_launch(65536, stream=st)

    def step(ev=None):
        if ev:
            ev[0].record(st)
        ctx.build(w.box_cm, rho, td, n=w.uniform_n, star_pos=w.star_pos, star_lum=w.star_lum, stream=st)
        if ev:
            ev[1].record(st)
        ctx.evaluate(J, F, stream=st)
        if ev:
            ev[2].record(st)
        ctx.radpressure(J, F, u, a_rp, force, p_src, stream=st)
        ctx.dust_temperature(tgas, J, Td, stream=st)
        if ev:
            ev[3].record(st)

    with torch.cuda.stream(st):
        for _ in range(args.warmup):
            step()
            flush.zero_()
        ctx.check(st)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        l0 = ctx.kernel_launches
        with ClockSampler(local) as clk:
            for k in range(args.steps):
                flush.zero_()
                step(evs[k])
            torch.cuda.synchronize()
        launches = ctx.kernel_launches - l0
        ctx.check(st)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    eval_ms = [e[1].elapsed_time(e[2]) for e in evs]
    build_ms = [e[0].elapsed_time(e[1]) for e in evs]
    post_ms = [e[2].elapsed_time(e[3]) for e in evs]
    ms = statistics.mean(step_ms)
    ms_eval = statistics.mean(eval_ms)
    ms, ms_eval = job_times([ms, ms_eval], dist, dev)
    value = job_value(n, npix, world, ms)

    # ---- roofline of the evaluate kernel: node-stream bytes per launch / measured duration
    with torch.cuda.stream(st):
        tot = ctx.walk_stats(stream=st).cpu().numpy().astype(np.int64)
    visits, acc, ent = (int(x) for x in tot)
    ns_bytes = node_stream_bytes(visits, acc)
    wide_bytes = (BYTES_VISIT * visits + BYTES_ACCEPT * (acc - n) + BYTES_ENTRY * ent
                  + BYTES_TARGET * n)
    peak, peak_kind = measured_peak()
    achieved = ns_bytes / (ms_eval * 1e-3) / 1e9
    traffic = ncu_traffic(f"turb128_npix{npix}")
    l2_bytes = ncu_traffic(f"turb128_npix{npix}", key="lts_bytes_per_launch")

    # ---- the other configurations' evaluate kernels (second ray count; collapsing core)
    import synth
    extra = {}
    if not args.no_extra_configs:
        w192 = workload(192) if npix != 192 else None
        if w192 is not None:
            extra["turb128_npix192"] = time_evaluate(tr, torch, w192, dev, args.steps, flush)
        extra["amr_core_npix48"] = time_evaluate(tr, torch, synth.amr_core(), dev, args.steps, flush)

    # ---- end to end through the public API with host buffers
    rho_h = torch.as_tensor(w.rho).pin_memory()
    td_h = torch.as_tensor(w.td).pin_memory()
    tg_h = torch.as_tensor(w.tgas).pin_memory()
    J_h = torch.empty(n, dtype=torch.float32).pin_memory()
    F_h = torch.empty(3 * n, dtype=torch.float64).pin_memory()
    Td_h = torch.empty(n, dtype=torch.float32).pin_memory()
    a_h = torch.empty(3 * n, dtype=torch.float32).pin_memory()
    h2d = 3 * 4 * n
    d2h = 4 * n + 24 * n + 4 * n + 12 * n

    def e2e_step():
        rho.copy_(rho_h, non_blocking=True)
        td.copy_(td_h, non_blocking=True)
        tgas.copy_(tg_h, non_blocking=True)
        step()
        J_h.copy_(J, non_blocking=True)
        F_h.copy_(F, non_blocking=True)
        Td_h.copy_(Td, non_blocking=True)
        a_h.copy_(a_rp, non_blocking=True)

    with torch.cuda.stream(st):
        for _ in range(max(1, args.warmup)):
            e2e_step()
        st.synchronize()
        e_ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            e2e_step()
            e1.record(st)
            st.synchronize()
            e_ms.append(e0.elapsed_time(e1))
    e2e_val = job_value(n, npix, world, job_times([statistics.mean(e_ms)], dist, dev)[0])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded lognormal turbulent cloud)",
            "config": config(npix, {"parallelism": f"replicas x{world}",
                                    "ms_build": statistics.mean(build_ms),
                                    "ms_evaluate": ms_eval,
                                    "ms_radpressure_dust": statistics.mean(post_ms),
                                    "warps_per_target": best_wpt,
                                    "autotune_ms_wpt2_3_4_8": tune_ms,
                                    "occupancy_pct": best_occ,
                                    "autotune_ms_occupancy_100_75_50": tune_occ,
                                    "ms_evaluate_npix192": extra.get("turb128_npix192", {}).get("ms"),
                                    "ms_evaluate_amr_core": extra.get("amr_core_npix48", {}).get("ms"),
                                    "other_configs": extra}),
            # The walk's node records are served by L1/L2 (DRAM moves only the compulsory
            # bytes); the kernel is bound by the SM's L1 data pipe (shared-memory deposits and
            # node loads). `frac` is the node-stream rate against the measured HBM copy peak.
            "roofline": {"bound": "l1", "kernel": "k_evaluate", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind,
                         "peak_basis": "measured HBM copy bandwidth (node-stream model)",
                         "traffic": traffic,
                         "dram_frac": None if traffic is None else traffic / (ms_eval * 1e-3) / 1e9 / peak,
                         "l2_GBps": None if l2_bytes is None else l2_bytes / (ms_eval * 1e-3) / 1e9,
                         "algorithmic_bytes_per_launch": ns_bytes,
                         "bytes_model": f"{NODE_BYTES_VISIT} B per visited node + {NODE_BYTES_ACCEPT} B per accepted node",
                         "with_angular_tables": {"bytes_per_launch": wide_bytes,
                                                 "achieved": wide_bytes / (ms_eval * 1e-3) / 1e9,
                                                 "frac": wide_bytes / (ms_eval * 1e-3) / 1e9 / peak},
                         "walk": {"visits": visits, "accepted": acc, "alpha_entries": ent}},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()


def cpu_baseline(w, seconds: float):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of targets;
    the full-workload time is its tree build plus the sample time scaled to every cell."""
    import numpy as np

    import oracle
    import synth
    oracle.build()
    t0 = time.perf_counter()
    tree = oracle.Tree(w)
    t_build = time.perf_counter() - t0
    m = 4096
    while True:  # grow the calibration sample until it takes a measurable time
        cal = synth.sample_targets(w.n_leaves, m, seed=21)
        t0 = time.perf_counter()
        tree.evaluate(cal)
        t_cal = time.perf_counter() - t0
        if t_cal > 0.5 or m >= w.n_leaves:
            break
        m = min(w.n_leaves, m * 4)
    m = int(min(w.n_leaves, max(1024, m * seconds / max(t_cal, 1e-3))))
    tg = synth.sample_targets(w.n_leaves, m, seed=22)
    t0 = time.perf_counter()
    J, F = tree.evaluate(tg)
    tree.radpressure(J, F, tg)
    oracle.dust_temperature(w.params, w.rho[tg], w.tgas[tg], J)
    t_s = time.perf_counter() - t0
    t_full = t_build + t_s * w.n_leaves / m
    cores = os.cpu_count()
    # one core: the same steps on a smaller sample (about a quarter of the time budget)
    m1 = int(max(256, min(m, m * 0.25 * seconds / max(t_s * cores, 1e-3))))
    tg1 = synth.sample_targets(w.n_leaves, m1, seed=23)
    t0 = time.perf_counter()
    J1, F1 = tree.evaluate(tg1, threads=1)
    tree.radpressure(J1, F1, tg1)
    oracle.dust_temperature(w.params, w.rho[tg1], w.tgas[tg1], J1)
    t_1 = time.perf_counter() - t0
    return {"value": w.n_leaves * w.params["npix"] / t_full, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{m} random cells of {w.n_leaves} (evaluate+radpressure+dust T, "
                      f"{t_s:.1f} s) plus the full tree build ({t_build:.1f} s), scaled to all cells",
            "threads": cores,
            "one_core": {"value": w.n_leaves * w.params["npix"] / (t_build + t_1 * w.n_leaves / m1),
                         "sample": f"{m1} random cells on 1 thread ({t_1:.1f} s), same tree build "
                                   f"time, scaled to all cells"}}


def run_batch64(args):
    """Independent boxes evaluated together: one batched persistent launch (per kernel
    variant), also replayed as a CUDA graph, against one evaluate launch per box with each
    box's autotuned team size. --batch64: 64 AMR boxes of 32^3-128^3 finest resolution
    (12.3 M leaves); --batch512: 512 boxes of 16^3-32^3 (1-2 levels); --batch-tiny: 1024
    boxes of 8^3, too small to fill the GPU one launch at a time. Prints one JSON line."""
    import torch

    import paper_2204_09072_gb300 as tr
    import synth
    dev = torch.device("cuda:0")
    if args.batch_tiny:
        boxes = synth.batch_of_tiny_boxes(1024, seed=10, npix=args.npix)
        name = "batch1024_tiny8"
    elif args.batch512:
        boxes = synth.batch_of_small_boxes(512, seed=9, npix=args.npix)
        name = "batch512_small"
    else:
        boxes = synth.batch_of_boxes(64, seed=5, npix=args.npix)
        name = "batch64_amr"
    ctxs, Js, Fs = [], [], []
    t0 = time.perf_counter()
    for w in boxes:
        c = tr.Context(w.params)
        c.build(w.box_cm, torch.as_tensor(w.rho, device=dev), torch.as_tensor(w.td, device=dev),
                blocks=w.blocks)
        c.autotune_launch(min(65536, w.n_leaves))
        ctxs.append(c)
        Js.append(torch.empty(w.n_leaves, dtype=torch.float32, device=dev))
        Fs.append(torch.empty(3 * w.n_leaves, dtype=torch.float64, device=dev))
    t_build = time.perf_counter() - t0
    batch = tr.Batch(ctxs)
    n = sum(w.n_leaves for w in boxes)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.mean(ts)

    ms_graph = timed(lambda: batch.evaluate(Js, Fs, use_graph=True), args.steps)
    ms_plain = timed(lambda: batch.evaluate(Js, Fs, use_graph=False), args.steps)

    def per_box():
        for c, J, F in zip(ctxs, Js, Fs):
            c.evaluate(J, F)
    ms_seq = timed(per_box, args.steps)
    for c in ctxs:
        c.check()
    print(json.dumps({"metric": METRIC, "unit": UNIT, "workload": name,
                      "speedup_graph_vs_per_box": ms_seq / ms_graph,
                      "boxes": len(boxes), "cells": n, "npix": args.npix,
                      "value_batched_graph": n * args.npix / (ms_graph * 1e-3),
                      "value_batched_plain": n * args.npix / (ms_plain * 1e-3),
                      "value_per_box_launches": n * args.npix / (ms_seq * 1e-3),
                      "ms_batched_graph": ms_graph, "ms_batched_plain": ms_plain,
                      "ms_per_box_launches": ms_seq, "host_build_s": t_build,
                      "steps": args.steps, "warmup": args.warmup}))


def run_sweep(args):
    """Cost of the 128^3 cloud's evaluation over N_pix x segments, with the autotuner's
    team size for each; then 48 and 192 rays with the opening angle matched to the ray
    size (theta = sqrt(4 pi / N_pix)) and quadratic radii, the setting in which the paper
    quotes its cost ratio; one JSON line per combination."""
    import torch

    import paper_2204_09072_gb300 as tr
    import synth
    dev = torch.device("cuda:0")
    combos = [(npix, nb, {}) for npix in (12, 48, 192) for nb in (10, 20, 40)] + [(768, 20, {})]
    combos += [(npix, 20, {"theta": -1.0, "bin_spacing": sp}) for sp in (0, 1) for npix in (48, 192, 768)]
    for npix, nb, extra in combos:
        w = synth.turbulent_cloud(128, npix=npix, nbins=nb, **extra)
        c = tr.Context(w.params)
        c.build(w.box_cm, torch.as_tensor(w.rho, device=dev), torch.as_tensor(w.td, device=dev), n=128,
                star_pos=w.star_pos, star_lum=w.star_lum)
        best, occ, tune, _ = c.autotune_launch(65536)
        J = torch.empty(w.n_leaves, dtype=torch.float32, device=dev)
        F = torch.empty(3 * w.n_leaves, dtype=torch.float64, device=dev)
        c.evaluate(J, F)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c.evaluate(J, F)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        c.check()
        st = c.walk_stats().cpu().numpy().tolist()
        print(json.dumps({"sweep": "turb128", "npix": npix, "nbins": nb,
                          "theta": "ray-matched" if extra.get("theta", 0.5) < 0 else 0.5,
                          "bin_spacing": "quadratic" if extra.get("bin_spacing", 0) == 1 else "geometric",
                          "warps_per_target": best, "occupancy_pct": occ,
                          "autotune_ms_wpt2_3_4_8_on_65536": tune, "ms_evaluate": ms,
                          "ray_evals_per_s": w.n_leaves * npix / (ms * 1e-3),
                          "walk_visits_accepted_entries": st}))
        c.close()


def run_orientations(args):
    """Several HEALPix orientations (Sec. 7.6) on the 128^3 cloud and on the collapsing-core
    AMR grid (the paper's ray pattern shows around its embedded sources): evaluate time for
    k turned ray sets (one seeded random orientation per cell) against the single unturned
    set, and the residual of J at 48 rays against 192 rays (ray-matched opening angles, as
    the paper's ray-count study): mean and spread over all cells, and the part of the
    spread that survives averaging over blocks of 4^3 cells (uniform grid) or over the 8^3
    blocks (AMR), the coherent ray pattern, versus the part left inside the blocks
    (cell-to-cell noise). One JSON line per workload and k."""
    import torch

    import paper_2204_09072_gb300 as tr
    import synth
    dev = torch.device("cuda:0")
    for wl in ("turb128", "amr_core"):
        _orientations_on(tr, synth, torch, dev, wl)


def _orientations_on(tr, synth, torch, dev, wl):
    def ctx_for(npix):
        if wl == "turb128":
            w = synth.turbulent_cloud(128, npix=npix, theta=-1.0)
        else:
            w = synth.amr_core(npix=npix, theta=-1.0)
        c = tr.Context(w.params)
        c.build(w.box_cm, torch.as_tensor(w.rho, device=dev), torch.as_tensor(w.td, device=dev),
                n=w.uniform_n, blocks=w.blocks, star_pos=w.star_pos, star_lum=w.star_lum)
        return w, c

    def blocks_of(r):
        if wl == "turb128":  # x-fastest cells -> 4^3 blocks
            b = r.reshape(32, 4, 32, 4, 32, 4)
            m = b.mean(axis=(1, 3, 5))
            return m, b - m[:, None, :, None, :, None]
        b = r.reshape(-1, 512)  # block-major leaves -> the 8^3 blocks
        m = b.mean(axis=1)
        return m, b - m[:, None]

    def timed_eval(c, n):
        J = torch.empty(n, dtype=torch.float32, device=dev)
        F = torch.empty(3 * n, dtype=torch.float64, device=dev)
        c.evaluate(J, F)
        ms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c.evaluate(J, F)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        c.check()
        return J.double().cpu().numpy(), statistics.median(ms)

    w, c192 = ctx_for(192)
    c192.autotune(65536)
    J192, ms192 = timed_eval(c192, w.n_leaves)
    c192.close()
    w, c = ctx_for(48)
    c.autotune(65536)
    n = w.n_leaves
    for k in (0, 4, 16, 64):
        t0 = time.time()
        if k:
            rot = synth.random_rotations(k, seed=100 + k)
            m = np.random.Generator(np.random.PCG64(200 + k)).integers(0, k, n).astype(np.uint8)
            c.set_orientations(rot, torch.as_tensor(m, device=dev))
        else:
            c.set_orientations(np.zeros((0, 3, 3)))
        t_tab = time.time() - t0
        J, ms = timed_eval(c, n)
        r = J / J192 - 1.0
        blk, inner = blocks_of(r)
        print(json.dumps({"orientations": k, "workload": f"{wl}_npix48_raytheta", "ms_evaluate": ms,
                          "ray_evals_per_s": n * 48 / (ms * 1e-3), "table_build_s": t_tab,
                          "ms_evaluate_192": ms192, "resid_mean": float(r.mean()), "resid_std": float(r.std()),
                          "resid_block_std": float(blk.std()), "resid_in_block_std": float(inner.std()),
                          "resid_abs_p50_p99": [float(np.percentile(np.abs(r), 50)),
                                                float(np.percentile(np.abs(r), 99))]}))
    c.close()


def run_blob(args):
    """The optically thick blob suite (S, M, L, S-, S+: 0.75-3 pc blobs at 30 K in a
    (15 pc)^3 box, Sec. 5.2) on 128^3 cells: evaluate throughput of the thick kernel and the
    radial structure of J on the GPU: the plateau inside the blob (J / J(30 K)), the
    ambient level between 3.5 and 5.5 pc (J / J(10 K)), and the far field 4.5-7 pc
    (J r^2 in units of the one-node-one-ray value sigma T^4 V^(2/3) / (4 pi^2)) with the
    radial fraction of the flux. One JSON line per variant."""
    import torch

    import paper_2204_09072_gb300 as tr
    import synth
    dev = torch.device("cuda:0")
    n, pc, sig = 128, 3.0857e18, 5.670374419e-5
    for v in ("S", "M", "L", "S-", "S+"):
        w = synth.blob_suite(v, n)
        c = tr.Context(w.params)
        c.build(w.box_cm, torch.as_tensor(w.rho, device=dev), torch.as_tensor(w.td, device=dev), n=n)
        best, occ, tune, _ = c.autotune_launch(65536)
        J = torch.empty(w.n_leaves, dtype=torch.float32, device=dev)
        F = torch.empty(3 * w.n_leaves, dtype=torch.float64, device=dev)
        c.evaluate(J, F)
        ms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c.evaluate(J, F)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        c.check()
        Jh = J.double().cpu().numpy()
        Fh = F.cpu().numpy().reshape(-1, 3)
        cen = synth.cell_centres(n, w.box_cm) - 0.5 * w.box_cm
        r = np.sqrt((cen ** 2).sum(1))
        core = w.rho > 5e-18
        R = 0.5 * synth.BLOB_DIAMETER_PC[v[0]] * pc
        dx = w.box_cm / n
        inside = r < R - 1.5 * dx
        amb = (r > 3.5 * pc) & (r < 5.5 * pc)
        far = (r > 4.5 * pc) & (r < 7.0 * pc)
        unit = sig * 30.0 ** 4 * (core.sum() * dx ** 3) ** (2.0 / 3.0) / (4 * math.pi ** 2)
        radial = (Fh[far] * cen[far]).sum(1) / r[far] / (4 * math.pi * Jh[far])
        print(json.dumps({"blob": v, "grid": f"{n}^3", "core_cells": int(core.sum()), "warps_per_target": best,
                          "ms_evaluate": statistics.median(ms),
                          "ray_evals_per_s": w.n_leaves * 48 / (statistics.median(ms) * 1e-3),
                          "J_inside_over_J30": float((Jh[inside] / (sig * 30.0 ** 4 / math.pi)).mean())
                          if inside.any() else None,
                          "J_ambient_over_J10": float((Jh[amb] / (sig * 10.0 ** 4 / math.pi)).mean()),
                          "far_Jr2_over_one_node": float((Jh[far] * r[far] ** 2 / unit).mean()),
                          "far_radial_flux_fraction": float(radial.mean())}))
        c.close()


def _cloud(n, seed, sigma, n_stars, npix, uv_heating=False):
    """Turbulent cloud with stars and an ionising flux field. The flux is a network
    feature; its UV dust heating is left out unless asked for: with it, dense cells near
    the stars turn optically thick, and a thick cell's own segment (tau_thick,0 = 0) passes
    all outside radiation, so their dust balance has no equilibrium."""
    import synth
    w = synth.turbulent_cloud(n, seed=seed, t_seed=seed + 1, sigma_ln=sigma, n_stars=n_stars, npix=npix)
    w = synth.with_gas(w, seed=seed + 2, tgas_lo=10.0, tgas_hi=100.0)
    w = synth.ionising_field(w)
    if not uv_heating:
        w.heat_extra = np.zeros_like(w.heat_extra)
    return w


def _clump(n, seed, npix):
    """The Gaussian clump (config 1) with a seeded gas temperature, a Planck-mean opacity
    (so that T_d feeds back on the field) and no stars or ionising flux."""
    import synth
    w = synth.gaussian_clump(n, npix=npix)
    w.params = dict(w.params, kappa_model=1)
    w = synth.with_gas(w, seed=seed, tgas_lo=10.0, tgas_hi=100.0)
    w.phi = np.zeros(w.n_leaves, np.float32)
    w.heat_extra = np.zeros(w.n_leaves, np.float32)
    w.star_pos = np.zeros((0, 3))
    w.star_lum = np.zeros(0)
    return w


def run_warmstart(args):
    import numpy as np  # noqa: F401  (used by _cloud)
    """Learned warm start of the dust-temperature fixed point.

    Training: plain fixed points (tol 1e-4) of seven seeded 128^3 clouds (sigma_lnrho 1.5
    and 2, 1-4 stars with ionising fields) and --warm-train-big clouds at the test size
    (sigma_lnrho 2, 4 stars, seeds 200, 201, ...); the features come from one evaluation
    at a uniform reference T_d (--warm-feature-td), so that they depend on the cloud alone
    and not on the random initial T_d; solves that do not converge are left out. Test: a --warm-n^3 cloud (sigma_lnrho 2, 4
    stars, ionising field, seed 777), plain fixed point from T_d ~ U[10, 40] K against
    features -> network -> fixed point."""
    import torch

    import paper_2204_09072_gb300 as tr
    dev = torch.device("cuda:0")

    def make(w):
        c = tr.Context(w.params)
        c.build(w.box_cm, torch.as_tensor(w.rho, device=dev), torch.as_tensor(w.td, device=dev), n=w.uniform_n,
                star_pos=w.star_pos, star_lum=w.star_lum)
        tg = torch.as_tensor(w.tgas, device=dev)
        he = torch.as_tensor(w.heat_extra, device=dev)
        ph = torch.as_tensor(w.phi, device=dev)
        return c, tg, he, ph

    t0 = time.perf_counter()
    Xs, ys, its = [], [], []
    solves = [(128, 101, 1.5, 1), (128, 102, 2.0, 2), (128, 103, 1.5, 4), (128, 104, 2.0, 3), (128, 105, 2.0, 4),
              (128, 106, 2.0, 4), (128, 107, 1.5, 2)]
    solves += [(args.warm_n, 200 + k, 2.0, 4) for k in range(args.warm_train_big)]
    # the 32^3 Gaussian clump (sigma 0: no turbulence) with gas temperatures of several seeds
    solves += [(32, 300 + k, 0.0, 0) for k in range(4)]
    for k, (nn, seed, sig, ns) in enumerate(solves):
        w = _cloud(nn, seed, sig, ns, args.npix) if sig > 0 else _clump(nn, seed, args.npix)
        c, tg, he, ph = make(w)
        c.refresh(torch.full((w.n_leaves,), args.warm_feature_td, device=dev))
        X = c.features(tg, phi=ph)[0].clone()
        td = torch.as_tensor(w.td, device=dev).clone()
        it = c.fixed_point(tg, td, heat_extra=he, tol=1e-4, max_iter=60, raise_on_noconv=False)
        its.append(it)
        if it > 0:  # solves that run away (thick emission over-counted) are left out
            Xs.append(X)
            ys.append(torch.log10(td))
        c.close()
    X = torch.cat(Xs).reshape(-1).contiguous()
    y = torch.cat(ys).contiguous()
    t_data = time.perf_counter() - t0
    net = tr.MLP(seed=2)
    net.fit_normalization(X, y)
    t0 = time.perf_counter()
    hist = net.train(X, y, steps=args.train_steps, batch=8192, lr=2e-3, seed=7)
    hist2 = net.train(X, y, steps=args.train_steps // 2, batch=8192, lr=3e-4, seed=8)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    per_seed = []
    for seed in args.warm_test_seeds:
        w = _cloud(args.warm_n, seed, 2.0, 4, args.npix)
        c, tg, he, ph = make(w)
        td0 = torch.as_tensor(w.td, device=dev)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        td_plain = td0.clone()
        torch.cuda.synchronize()
        e[0].record()
        it_plain = c.fixed_point(tg, td_plain, heat_extra=he, tol=1e-4, max_iter=60, raise_on_noconv=False)
        e[1].record()
        torch.cuda.synchronize()
        td_warm = td0.clone()
        torch.cuda.synchronize()
        e[2].record()
        c.refresh(torch.full_like(td0, args.warm_feature_td))
        Xw = c.features(tg, phi=ph)[0]
        c.warm_start(net, Xw.reshape(-1).contiguous(), td_warm)
        guess = td_warm.clone()
        it_warm = c.fixed_point(tg, td_warm, heat_extra=he, tol=1e-4, max_iter=60, raise_on_noconv=False)
        e[3].record()
        torch.cuda.synchronize()
        c.check()
        ms_plain = e[0].elapsed_time(e[1])
        ms_warm = e[2].elapsed_time(e[3])
        gerr = (guess / td_plain - 1).abs()
        ferr = (td_warm / td_plain - 1).abs()
        gq = torch.quantile(gerr[torch.randperm(gerr.numel(), device=gerr.device)[:1 << 22]],
                            torch.tensor([0.5, 0.9, 0.99, 0.999], device=gerr.device)).tolist()
        per_seed.append({
            "seed": seed, "iterations_plain": it_plain, "iterations_warm": it_warm,
            "evaluations_plain": it_plain, "evaluations_warm": it_warm + 1,
            "evaluation_ratio": it_plain / (it_warm + 1), "iteration_ratio": it_plain / max(it_warm, 1),
            "ms_fixed_point_plain": ms_plain, "ms_warm_total": ms_warm, "speedup": ms_plain / ms_warm,
            "guess_rel_err_p50_p90_p99_p999": gq, "guess_rel_err_max": float(gerr.max()),
            "final_rel_diff_max": float(ferr.max())})
        c.close()
    print(json.dumps({
        "workload": f"learned warm start, test clouds {args.warm_n}^3 sigma_lnrho 2, 4 stars, ionising flux "
                    f"as a feature (no UV dust heating); features at uniform T_d = {args.warm_feature_td} K",
        "train_samples": int(y.numel()), "train_solves_iterations": its, "train_steps": len(hist) + len(hist2),
        "train_loss_first_last": [float(hist[:20].mean()), float(hist2[-50:].mean())],
        "s_training_data": t_data, "s_training": t_train, "training_solves": [list(x) for x in solves],
        "evaluations_note": "warm path = feature pass (one evaluation) + fixed-point iterations",
        "per_seed": per_seed,
        "evaluation_ratio_min": min(p["evaluation_ratio"] for p in per_seed),
        "final_rel_diff_max": max(p["final_rel_diff_max"] for p in per_seed)}))


def run_rays_study(args):
    """The paper's ray-count study (Sec. 7.6) on the collapsing-core AMR grid: evaluate cost at
    48, 192 and 768 rays with the opening angle matched to the ray size (theta = sqrt(4 pi /
    N_pix): the paper opens nodes further as the rays get finer), and the residual of the
    radiation temperature T_J = (pi J / sigma)^(1/4) (eq. radtemp) of 48 and 192 rays against
    768 rays, as mean +- standard deviation over the cells of the central half of the domain
    (the half-width cube) and of the whole domain. Same T_d field for all ray counts (T_d =
    20 K inside, as generated). Prints one JSON line."""
    import numpy as np
    import torch

    import paper_2204_09072_gb300 as tr
    import synth
    dev = torch.device("cuda:0")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    w0 = synth.amr_core() if args.rays_workload == "amr_core" else synth.turbulent_cloud(128)
    sig = 5.670374419e-5
    res, T = {}, {}
    for npix in (48, 192, 768):
        w = w0
        w.params = dict(w0.params, npix=npix, theta=-1.0)
        t0 = time.perf_counter()
        r = time_evaluate(tr, torch, w, dev, args.steps, flush)
        r["s_setup_and_timing"] = time.perf_counter() - t0
        ctx = tr.Context(w.params)
        ctx.build(w.box_cm, torch.as_tensor(w.rho, device=dev), torch.as_tensor(w.td, device=dev),
                  n=w.uniform_n, blocks=w.blocks, star_pos=w.star_pos, star_lum=w.star_lum)
        n = w.n_leaves
        J = torch.empty(n, dtype=torch.float32, device=dev)
        F = torch.empty(3 * n, dtype=torch.float64, device=dev)
        ctx.evaluate(J, F)
        ctx.check()
        T[npix] = (np.pi * J.double().cpu().numpy() / sig) ** 0.25
        ctx.close()
        res[npix] = r
    cen = (w0.leaf_ijk.astype(np.float64) + 0.5) / (2.0 ** w0.leaf_level)[:, None]  # in box units
    half = (np.abs(cen - 0.5) < 0.25).all(axis=1)
    out = {}
    for npix in (48, 192):
        d = T[npix] / T[768] - 1
        out[f"residual_{npix}_vs_768"] = {
            "half_domain_mean_std_pct": [100 * float(d[half].mean()), 100 * float(d[half].std())],
            "full_domain_mean_std_pct": [100 * float(d.mean()), 100 * float(d.std())]}
    base = res[48]["ms"]
    print(json.dumps({"workload": f"{args.rays_workload}, ray-matched opening angle", "cells": int(w0.n_leaves),
                      "cells_half_domain": int(half.sum()),
                      "ms_evaluate": {k: v["ms"] for k, v in res.items()},
                      "cost_ratio_48_192_768": [1.0, res[192]["ms"] / base, res[768]["ms"] / base],
                      "paper_cost_ratio": [1.0, 4.39, 15.98],
                      "walk": {k: v["walk"] for k, v in res.items()},
                      "warps_per_target": {k: v["warps_per_target"] for k, v in res.items()},
                      "paper_residuals_pct": {"48_half": [-15.4, 14.0], "192_half": [-3.77, 5.31],
                                              "48_full": [-31.0, 17.9], "192_full": [-13.2, 10.5]},
                      **out}))


def run_amr_core(args):
    """Collapsing-core AMR grid (~1.9 M leaves of 8^3 blocks on levels 5-9, 10 stars of
    1e2-1e5 Lsun, optically thick centre): evaluation throughput with the step as in the
    main bench, then the plain GPU fixed point of T_d and the IR field to 1e-4 from
    T_d = 20 K; when it does not converge, the largest relative change per iteration."""
    import numpy as np
    import torch

    import paper_2204_09072_gb300 as tr
    import synth
    dev = torch.device("cuda:0")
    t0 = time.perf_counter()
    w = synth.amr_core()
    t_gen = time.perf_counter() - t0
    n = w.n_leaves
    npix = w.params["npix"]
    ctx = tr.Context(w.params)
    st = torch.cuda.Stream(device=dev)
    rho = torch.as_tensor(w.rho, device=dev)
    td0 = torch.as_tensor(w.td, device=dev)
    tgas = torch.as_tensor(w.tgas, device=dev)
    J = torch.empty(n, dtype=torch.float32, device=dev)
    F = torch.empty(3 * n, dtype=torch.float64, device=dev)
    u = torch.empty(n, device=dev)
    a_rp = torch.empty(3 * n, device=dev)
    force = torch.empty(3 * n, device=dev)
    p_src = torch.empty(n, device=dev)
    Td = torch.empty(n, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def build():
        ctx.build(w.box_cm, rho, td0, blocks=w.blocks, star_pos=w.star_pos, star_lum=w.star_lum, stream=st)

    with torch.cuda.stream(st):
        build()
        best, tune = ctx.autotune(65536, stream=st)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps + args.warmup)]
        for k in range(args.steps + args.warmup):
            flush.zero_()
            e = ev[k]
            e[0].record(st)
            build()
            e[1].record(st)
            ctx.evaluate(J, F, stream=st)
            e[2].record(st)
            ctx.radpressure(J, F, u, a_rp, force, p_src, stream=st)
            ctx.dust_temperature(tgas, J, Td, stream=st)
            e[3].record(st)
        torch.cuda.synchronize()
        ctx.check(st)
        tot = ctx.walk_stats(stream=st).cpu().numpy().astype(np.int64)
    ev = ev[args.warmup:]
    ms_step = statistics.mean(e[0].elapsed_time(e[3]) for e in ev)
    ms_eval = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    visits, acc, ent = (int(x) for x in tot)
    alg = node_stream_bytes(visits, acc)
    peak, kind = measured_peak()
    # plain GPU fixed point (graph of unrolled iterations)
    ctx.refresh(td0)
    td = td0.clone()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    it = ctx.fixed_point(tgas, td, tol=1e-4, max_iter=args.fp_max_iter, raise_on_noconv=False)
    f1.record()
    torch.cuda.synchronize()
    ms_fp = f0.elapsed_time(f1)
    out = {
        "workload": f"amr_core: collapsing-core AMR, {n} leaves, levels {sorted(set(np.asarray(w.leaf_level).tolist()))}, "
                    f"{len(w.star_lum)} stars, N_pix {npix}, {w.params['nbins']} segments",
        "s_generate": t_gen, "warps_per_target": best, "autotune_ms_wpt2_3_4_8": tune,
        "ms_per_step": ms_step, "ms_evaluate": ms_eval,
        "ray_evals_per_s": n * npix / (ms_step * 1e-3), "ray_evals_per_s_evaluate": n * npix / (ms_eval * 1e-3),
        "roofline": {"bound": "l1", "achieved": alg / (ms_eval * 1e-3) / 1e9, "peak": peak, "peak_kind": kind,
                     "frac": alg / (ms_eval * 1e-3) / 1e9 / peak, "algorithmic_bytes_per_launch": alg,
                     "bytes_model": f"{NODE_BYTES_VISIT} B per visited node + {NODE_BYTES_ACCEPT} B per accepted node"},
        "walk": {"visits": visits, "accepted": acc, "alpha_entries": ent},
        "fixed_point": {"tol": 1e-4, "iterations": it, "converged": it > 0, "ms": ms_fp,
                        "Td_min": float(td.min()), "Td_max": float(td.max())},
    }
    if it <= 0:
        # one iteration at a time: the largest relative change and where it sits, and how many
        # cells still change by more than the tolerance, thin and thick (the class of the
        # iteration's T_d) and per refinement level
        ctx.refresh(td0)
        td = td0.clone()
        hist, above = [], []
        lev = torch.as_tensor(np.asarray(w.leaf_level), device=dev)
        levels = sorted(set(np.asarray(w.leaf_level).tolist()))
        for _ in range(args.fp_diag_iter):
            prev = td.clone()
            ctx.fixed_point(tgas, td, tol=1e-30, max_iter=1, unroll=0, raise_on_noconv=False)
            ch = (td / prev - 1).abs()
            k = int(torch.argmax(ch))
            hist.append([float(ch[k]), k, float(prev[k]), float(td[k]), float(rho[k])])
            thick = torch.as_tensor(ctx.leaf_export()["thick"], device=dev) != 0
            big = ch > 1e-4
            above.append({"above_tol": int(big.sum()), "thick": int((big & thick).sum()),
                          "thin": int((big & ~thick).sum()), "thick_cells": int(thick.sum()),
                          "by_level": {int(L): int((big & (lev == L)).sum()) for L in levels}})
        out["fixed_point"]["history_max_change_cell_T_before_after_rho"] = hist
        out["fixed_point"]["history_cells_above_tol"] = above
    ctx.close()
    print(json.dumps(out))


def run_profile(args):
    """Profiling driver for ncu: build the full tree once, then launch the evaluate
    kernel on a seeded subset of targets: two warm-up launches, then one more."""
    import numpy as np
    import torch

    import paper_2204_09072_gb300 as tr
    import synth
    w = workload(args.npix) if args.profile_workload == "turb128" else synth.amr_core(npix=args.npix)
    ctx = tr.Context(w.params)
    dev = torch.device("cuda:0")
    rho = torch.as_tensor(w.rho, device=dev)
    td = torch.as_tensor(w.td, device=dev)
    ctx.build(w.box_cm, rho, td, n=w.uniform_n, blocks=w.blocks, star_pos=w.star_pos, star_lum=w.star_lum)
    ctx.set_warps_per_target(args.profile_wpt)  # the team size the bench's autotuner picks
    m = min(args.profile_targets, w.n_leaves)
    tg = torch.as_tensor(np.sort(synth.sample_targets(w.n_leaves, m, seed=5)).astype(np.int32),
                         device=dev)
    J = torch.empty(m, dtype=torch.float32, device=dev)
    F = torch.empty(3 * m, dtype=torch.float64, device=dev)
    for _ in range(3):
        ctx.evaluate(J, F, targets=tg)
    ctx.check()
    print(json.dumps({"profile": "evaluate", "workload": f"{args.profile_workload}_npix{args.npix}", "targets": m,
                      "warps_per_target": args.profile_wpt,
                      "J_mean": float(J.double().mean())}))
    ctx.close()


def run_profile_others(args):
    """Profiling driver for ncu: every kernel of the path other than the evaluate kernel on
    the 128^3 cloud, twice (a warm-up pass, then the captured one): tree build (leaf
    quantities, Morton keys and radix sort, levels, moments, records), radiation pressure,
    dust temperature, warm-start features, network inference and training steps."""
    import torch

    import paper_2204_09072_gb300 as tr
    w = workload(args.npix)
    n = w.n_leaves
    dev = torch.device("cuda:0")
    ctx = tr.Context(w.params)
    rho = torch.as_tensor(w.rho, device=dev)
    td = torch.as_tensor(w.td, device=dev)
    tg = torch.as_tensor(w.tgas, device=dev)
    J = torch.empty(n, dtype=torch.float32, device=dev)
    F = torch.empty(3 * n, dtype=torch.float64, device=dev)
    u, Td = torch.empty(n, device=dev), torch.empty(n, device=dev)
    a_rp, force, p_src = torch.empty(3 * n, device=dev), torch.empty(3 * n, device=dev), torch.empty(n, device=dev)
    net = tr.MLP(seed=1)
    for rep in range(2):
        ctx.build(w.box_cm, rho, td, n=w.uniform_n, star_pos=w.star_pos, star_lum=w.star_lum)
        ctx.evaluate(J, F)
        ctx.radpressure(J, F, u, a_rp, force, p_src)
        ctx.dust_temperature(tg, J, Td)
        X = ctx.features(tg)[0].reshape(-1).contiguous()
        y = torch.log10(Td)
        if rep == 0:
            net.fit_normalization(X, y)
        net.train(X, y, steps=4, batch=8192, lr=1e-3, seed=rep + 1)
        guess = torch.empty(n, device=dev)
        ctx.warm_start(net, X, guess)
        ctx.check()
    torch.cuda.synchronize()
    print(json.dumps({"profile": "others", "workload": f"turb128_npix{args.npix}", "cells": n,
                      "Td_mean": float(Td.double().mean()), "guess_mean": float(guess.double().mean())}))
    ctx.close()
    net.close()


def run_reference(args):
    """The oracle timed as the reference arm: each step evaluates a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    w = workload(args.npix)
    tree = oracle.Tree(w)
    m = args.ref_sample
    times = []
    for k in range(args.warmup + args.steps):
        tg = synth.sample_targets(w.n_leaves, m, seed=100 + k)
        t0 = time.perf_counter()
        J, F = tree.evaluate(tg)
        tree.radpressure(J, F, tg)
        oracle.dust_temperature(w.params, w.rho[tg], w.tgas[tg], J)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = statistics.mean(times) * 1e3
    value = m * args.npix / (ms * 1e-3)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded lognormal turbulent cloud)",
            "config": config(args.npix, {"sample_per_step": m}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{m} random cells per step (evaluate+radpressure+dust T)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    if "--impl" not in sys.argv or "reference" not in sys.argv:
        import paper_2204_09072_gb300 as tr
        tr.build_library()  # no-op when the in-tree library is up to date
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--npix", type=int, default=48, choices=[12, 48, 192, 768])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-sample", type=int, default=16384)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--wpt", type=int, default=0, choices=[0, 2, 3, 4, 8],
                    help="headline step: fixed warps per target instead of the autotuner (0)")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the 192-ray and collapsing-core evaluate timings")
    ap.add_argument("--profile-evaluate", action="store_true",
                    help="ncu driver: evaluate kernel only, on --profile-targets cells")
    ap.add_argument("--profile-targets", type=int, default=262144)
    ap.add_argument("--profile-others", action="store_true",
                    help="ncu driver: every kernel but the evaluate kernel, on the 128^3 cloud")
    ap.add_argument("--profile-workload", default="turb128", choices=["turb128", "amr_core"])
    ap.add_argument("--profile-wpt", type=int, default=3, choices=[2, 3, 4, 8],
                    help="warps per target of the profiled launches (thick trees run 3 as 4)")
    ap.add_argument("--batch64", action="store_true", help="64-box AMR batch: batched vs per-box launches")
    ap.add_argument("--batch512", action="store_true", help="512 small boxes: batched vs per-box launches")
    ap.add_argument("--batch-tiny", action="store_true", help="1024 boxes of 8^3: batched vs per-box launches")
    ap.add_argument("--rays-study", action="store_true",
                    help="cost and T_J residuals at 48 / 192 / 768 rays, ray-matched opening angle")
    ap.add_argument("--rays-workload", default="amr_core", choices=["amr_core", "turb128"])
    ap.add_argument("--sweep", action="store_true", help="N_pix x segments sweep with the autotuner")
    ap.add_argument("--warmstart", action="store_true", help="learned warm start of the T_d fixed point")
    ap.add_argument("--warm-n", type=int, default=256)
    ap.add_argument("--warm-test-seeds", type=int, nargs="+", default=[777, 778, 779])
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--warm-feature-td", type=float, default=20.0,
                    help="uniform T_d of the feature pass (training and test)")
    ap.add_argument("--warm-train-big", type=int, default=2,
                    help="training solves at the test resolution (seeds 200, 201, ...)")
    ap.add_argument("--amr-core", action="store_true",
                    help="collapsing-core AMR grid: throughput and the plain fixed point to 1e-4")
    ap.add_argument("--orientations", action="store_true",
                    help="several HEALPix orientations: cost and J residuals against 192 rays")
    ap.add_argument("--blob", action="store_true", help="optically thick blob suite S, M, L, S-, S+ on 128^3")
    ap.add_argument("--fp-max-iter", type=int, default=100)
    ap.add_argument("--fp-diag-iter", type=int, default=20)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.profile_evaluate:
        run_profile(args)
    elif args.profile_others:
        run_profile_others(args)
    elif args.rays_study:
        run_rays_study(args)
    elif args.batch64 or args.batch512 or args.batch_tiny:
        run_batch64(args)
    elif args.sweep:
        run_sweep(args)
    elif args.warmstart:
        run_warmstart(args)
    elif args.amr_core:
        run_amr_core(args)
    elif args.orientations:
        run_orientations(args)
    elif args.blob:
        run_blob(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
