#!/usr/bin/env python
"""Benchmark: family scores per second of the all-families Givens walk.

One step = one call of score_all_families on the m=26, n=5000 SEM workload
(two near-collinear columns): CholeskyQR2 R0 in FP64, the sub-walk roots and
the Givens walk writing all m*2^(m-1) = 872,415,232 BIC scores to HBM.  The
headline is the FP32 walk; the plain FP64 walk is timed beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank scores its
own dataset (seed + rank): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import ctypes
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "family scores/sec (all m*2^(m-1)) at m=26, FP32 vs plain FP64, on 1 GB300"
UNIT = "family scores/s"
FALLBACK_HBM_GBS = 6800.0
WALK_SOURCES = ["paper_1901_07643_gb300/csrc/walk3.cuh", "paper_1901_07643_gb300/csrc/walk_inst.cu",
                "paper_1901_07643_gb300/csrc/walk_dispatch.cu",
                "paper_1901_07643_gb300/csrc/gbn_internal.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "walk_traffic.json")
LAUNCHES_PER_STEP = 16  # colsum, mean, (gram, gram sum, cholesky) x2, column scaling,
                        # fix-up flags, roots top + leaves, walk, fix-up scan + solve,
                        # score correction of scaled columns


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="m26", choices=["m26", "m24", "m20", "m10"])
    ap.add_argument("--q", type=int, default=0)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-extras", action="store_true",
                    help="skip the batched-workload and adjoint legs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="take the automatic (q, consumer warps) instead of timing the candidates")
    return ap.parse_args()


def _workload(name):
    from paper_1901_07643_gb300 import synthetic
    return {"m26": synthetic.LARGE_M26, "m24": synthetic.PROFILE_M24, "m20": synthetic.MEDIUM_M20,
            "m10": synthetic.SMALL_M10}[name]


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _source_hash():
    h = hashlib.sha256()
    for p in WALK_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _walk_kernel_name(m, q):
    """The FP32 walk kernel a single-dataset call launches (the library's choice for full warps
    of sub-walks and an even number of roots CTAs, which every bench workload has)."""
    return f"walk_ring_kernel<{q}, true>" if q <= 6 else f"walk_kernel_pair<{q}>"


def _traffic(workload_name, q=None):
    """Per-launch DRAM bytes of the walk kernel from the committed ncu summary, if current."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != _source_hash() or d.get("workload") != workload_name:
        return None
    if q is not None and d.get("q") != q:
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def _gpu_id(dev_index):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev_index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev_index] if vis else str(dev_index)


def _error_sample(X, m, count, seed=12345):
    """Seeded random families plus families of each near-collinear column pair (child one
    column of the pair, parents holding the other): the families the CPU baseline times and
    the error statistics compare."""
    rng = np.random.default_rng(seed)
    child = rng.integers(0, m, count).astype(np.int64)
    mask = rng.integers(0, 1 << m, count, dtype=np.int64).astype(np.uint64)
    mask &= ~(np.uint64(1) << child.astype(np.uint64))
    C = np.corrcoef(X, rowvar=False)
    pairs = [(a, b) for a in range(m) for b in range(m) if a != b and abs(C[a, b]) > 0.99]
    if pairs:
        pick = rng.integers(0, len(pairs), count // 8)
        cc = np.array([pairs[i][0] for i in pick], np.int64)
        pp = np.array([pairs[i][1] for i in pick], np.uint64)
        mm = rng.integers(0, 1 << m, len(pick), dtype=np.int64).astype(np.uint64)
        mm = (mm & ~(np.uint64(1) << cc.astype(np.uint64))) | (np.uint64(1) << pp)
        child = np.concatenate([child, cc])
        mask = np.concatenate([mask, mm])
    order = rng.permutation(len(child))  # a prefix of the sample is a sample too
    return child[order].astype(np.int32), mask[order]


def _slots(child, mask, m):
    """Table slots idx(c,S) = c 2^(m-1) + compress(S, c) of the sampled families."""
    c = child.astype(np.uint64)
    low = mask & ((np.uint64(1) << c) - np.uint64(1))
    high = (mask >> (c + np.uint64(1))) << c
    return ((c << np.uint64(m - 1)) + (low | high)).astype(np.int64)


def _cpu_baseline(X, n, m, seconds, gathered):  # noqa: C901
    """Oracle (direct FP64 Householder per family) on a bounded sample of the workload,
    and the GPU tables' errors against it on the same families (`gathered`: precision ->
    the table's values at the sampled slots)."""
    import oracle
    cores = _cores()
    c, k = _error_sample(X, m, max(cores * 4, 32), seed=1)
    t0 = time.perf_counter()
    oracle.scores_sampled(X, c, k, nthreads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    count = int(min(2_000_000, max(len(c), len(c) * seconds / dt)))
    c, k = gathered["families"]
    c, k = c[:count], k[:count]
    t0 = time.perf_counter()
    _, ref = oracle.scores_sampled(X, c, k, nthreads=cores)
    dt = time.perf_counter() - t0
    errors = {}
    for name, got in gathered.items():
        if name == "families":
            continue
        if name == "bge":  # BGe scores against the BGe oracle on a prefix of the sample
            from oracle import bge
            cb, kb = gathered["families"]
            ref_b = bge.scores_sampled(X, cb[:len(got)], kb[:len(got)])
            scaled = np.abs(np.asarray(got, np.float64) - ref_b) / np.maximum(np.abs(ref_b), n)
            errors[name] = {"max_scaled": float(scaled.max()), "count": int(len(ref_b)),
                            "tolerance": 1e-4}
            continue
        got = np.asarray(got[:len(ref)], np.float64)
        d = got - ref
        scaled = np.abs(d) / np.maximum(np.abs(ref), n)
        errors[name] = {"max_scaled": float(scaled.max()),
                        "max_rel_rss": float(np.max(np.abs(np.expm1(d / n)))),
                        "count": int(len(ref)),
                        "tolerance": 1e-4 if name == "fp32" else 1e-10}
    return ({"value": len(ref) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"{len(ref)} families of the m={m}, n={n} workload (seeded random, 1/9 "
                       f"of them near-collinear-pair families), direct FP64 Householder QR per "
                       f"family, OpenMP over families; {dt:.1f} s"}, errors)


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_1901_07643_gb300 import synthetic
    import oracle
    w = _workload(args.workload)
    X = synthetic.workload_sample(w)
    cores = _cores()
    rng = np.random.default_rng(777)
    fam_total = w.m << (w.m - 1)

    def step(count):
        child = rng.integers(0, w.m, count).astype(np.int32)
        mask = np.array([int(rng.integers(0, 1 << w.m)) & ~(1 << int(c)) for c in child], np.uint64)
        t0 = time.perf_counter()
        oracle.scores_sampled(X, child, mask, nthreads=cores)
        return time.perf_counter() - t0

    dt = step(max(4 * cores, 32))
    per_step = int(max(4 * cores, 32) * min(8.0, 160.0 / max(1, args.steps + args.warmup)) /
                   max(dt, 1e-3))
    per_step = max(per_step, cores)
    for _ in range(args.warmup):
        step(per_step)
    times = [step(per_step) for _ in range(args.steps)]
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "families": fam_total,
                   "step": f"{per_step} sampled families (bounded sample of the workload)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random families per step, direct FP64 "
                                   "Householder QR per family"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _time_steps(fn, steps, flush, stream):
    """Per-step CUDA-event durations (ms) and walk-stage durations (ms)."""
    import torch
    step_ms, walk_ms = [], []
    pairs = []
    for _ in range(steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[4].record(stream)
        fn(ev[:4])
        ev[5].record(stream)
        pairs.append(ev)
    torch.cuda.synchronize()
    for ev in pairs:
        step_ms.append(ev[4].elapsed_time(ev[5]))   # the whole call
        walk_ms.append(ev[2].elapsed_time(ev[3]))   # the walk kernel alone
    return step_ms, walk_ms


def _e2e(X, Xd, fam, q32, cw32, w, world, dev, args):
    """End to end through the public call: pinned host X copied in, the table
    delivered to pinned host memory, both inside the timed region.  Three ways
    of delivering the table are timed and the fastest is reported: a device
    table copied back (one copy, or four concurrent chunks), and the kernels
    writing straight into host memory."""
    import torch
    import torch.distributed as dist
    from paper_1901_07643_gb300 import binding
    Xh = torch.from_numpy(X).pin_memory()
    outh = torch.empty(fam, dtype=torch.float32, pin_memory=True)
    Xd2 = torch.empty_like(Xd)
    outd = torch.empty(fam, dtype=torch.float32, device=dev)
    wsd = torch.empty(binding.workspace_size(w.n, w.m, 0, q32, consumer_warps=cw32),
                      dtype=torch.uint8, device=dev)
    kw = dict(q=q32, consumer_warps=cw32, workspace=wsd, check=False)

    def via_copy():
        Xd2.copy_(Xh, non_blocking=True)
        binding.score_all_families(Xd2, outd, **kw)
        outh.copy_(outd, non_blocking=True)

    def direct():
        Xd2.copy_(Xh, non_blocking=True)
        binding.score_all_families(Xd2, outh, **kw)

    streams = [torch.cuda.Stream(dev) for _ in range(4)]

    def via_copy_streams():  # the table copied back as four concurrent chunks
        Xd2.copy_(Xh, non_blocking=True)
        binding.score_all_families(Xd2, outd, **kw)
        done = torch.cuda.Event()
        done.record()
        part = (fam + len(streams) - 1) // len(streams)
        for i, st in enumerate(streams):
            st.wait_event(done)
            with torch.cuda.stream(st):
                outh[i * part:(i + 1) * part].copy_(outd[i * part:(i + 1) * part], non_blocking=True)
        for st in streams:
            torch.cuda.current_stream(dev).wait_stream(st)

    res = {}
    for name, fn in (("device_table_copied", via_copy), ("kernels_write_host", direct),
                     ("device_table_copied_4_streams", via_copy_streams)):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        evs = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        tot = sum(a.elapsed_time(b) for a, b in evs)
        if world > 1:
            t = torch.tensor([tot], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tot = float(t.item())
        res[name] = tot / args.steps
    best = min(res, key=res.get)
    # the host link alone: the same table, device -> pinned host, one copy, nothing else
    cp = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        outh.copy_(outd, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        cp.append(a.elapsed_time(b))
    d2h = int(outh.numel() * outh.element_size())
    copy_ms = min(cp)
    return {"value": world * fam / (res[best] / 1e3), "unit": UNIT,
            "h2d_bytes_per_step": int(Xh.numel() * Xh.element_size()),
            "d2h_bytes_per_step": d2h,
            "ms_per_step": res[best], "method": best,
            "ms_per_step_by_method": res,
            "host_link": {"d2h_copy_ms": copy_ms, "d2h_gbs": d2h / (copy_ms / 1e3) / 1e9,
                          "how": "one cudaMemcpyAsync of the table, device to pinned host "
                                 "(best of 5, CUDA events)"},
            "note": "value is the fastest of the three delivery methods listed"}


def _extras(dev, flush, args):
    """Secondary legs: the 256-dataset bootstrap batch and the adjoint of the
    64-dataset gradient workload, each timed with CUDA events."""
    import torch
    from paper_1901_07643_gb300 import binding, synthetic
    out = {}
    Xs = [torch.from_numpy(X).to(dev) for X in synthetic.batched_bootstrap()]
    offs, total = binding.batch_offsets(Xs)
    q, cw, tune = 0, 0, None
    if not args.no_autotune:
        q, cw, ms, table = binding.autotune_batched(Xs)
        tune = {"q": q, "consumer_warps": cw, "median_ms": ms,
                "candidates": [{"q": a, "consumer_warps": b, "median_ms": t} for a, b, t in table]}
        torch.cuda.empty_cache()
    kw = dict(q=q, consumer_warps=cw)
    tbl = torch.empty(total, dtype=torch.float32, device=dev)
    ws = torch.empty(binding.batched_workspace_size(Xs, **kw), dtype=torch.uint8, device=dev)
    for _ in range(2):
        binding.score_all_families_batched(Xs, tbl, workspace=ws, **kw)
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            binding.score_all_families_batched(Xs, tbl, workspace=ws, **kw)
    torch.cuda.current_stream(dev).wait_stream(s)
    ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    out["batched"] = {"workload": "bootstrap_256 (m~U{12..20}, n~U{100..5000})", "datasets": len(Xs),
                      "families": total, "ms_per_batch": t, "value": total / (t / 1e3),
                      "unit": UNIT, "launch": "one captured CUDA graph",
                      "q": q or None, "consumer_warps": cw or None, "autotune": tune,
                      "hbm_floor_frac": 4 * total / (t / 1e3) / 1e9 / _peak_hbm()[0],
                      "hbm_floor_note": "4 B per score written once, against the measured copy "
                                        "bandwidth, over the whole batch call"}
    del tbl, ws, graph
    Gs, w = synthetic.gradient_workload()
    Gd = [torch.from_numpy(X).to(dev) for X in Gs]
    wt = torch.from_numpy(w).to(dev).float()
    fam = len(Gd) * (16 << 15)
    wsb = torch.empty(binding.backward_batched_workspace_size(Gd), dtype=torch.uint8, device=dev)
    grads = [torch.empty_like(X) for X in Gd]
    for _ in range(2):
        binding.score_all_families_backward_batched(Gd, wt, workspace=wsb, grads=grads)
    torch.cuda.synchronize()
    ms = []
    for _ in range(5):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        binding.score_all_families_backward_batched(Gd, wt, workspace=wsb, grads=grads)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    del wsb
    ws1 = torch.empty(binding.backward_workspace_size(Gs[0].shape[0], Gs[0].shape[1]),
                      dtype=torch.uint8, device=dev)
    binding.score_all_families_backward(Gd[0], wt, workspace=ws1, check=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for X in Gd:
        binding.score_all_families_backward(X, wt, workspace=ws1, check=False)
    b.record()
    torch.cuda.synchronize()
    t1 = a.elapsed_time(b)
    out["adjoint"] = {"workload": "gradient_64 (m=16, n=2000)", "datasets": len(Gd),
                      "ms_total": t, "value": fam / (t / 1e3), "unit": "family adjoints/s",
                      "launch": "score_all_families_backward_batched (one call, 64 datasets)",
                      "ms_total_64_single_calls": t1,
                      "dtype": "f32 walk, f64 accumulation"}
    return out


def _bge_leg(Xd, w, flush, slots_t, gathered):
    """The BGe score of every family (score="bge": a factor of the posterior matrix, the
    unchanged walk, the log-determinant recursion and an in-place pass over the table),
    timed with CUDA events like the RSS-score call; its sampled values join the errors."""
    import torch
    from paper_1901_07643_gb300 import binding
    dev = Xd.device
    fam = w.m << (w.m - 1)
    out = torch.empty(fam, dtype=torch.float32, device=dev)
    ws = torch.empty(binding.workspace_size(w.n, w.m, score="bge"), dtype=torch.uint8,
                     device=dev)
    binding.score_all_families(Xd, out, workspace=ws, score="bge")  # warm-up and status check
    ms = []
    for _ in range(3):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        binding.score_all_families(Xd, out, workspace=ws, score="bge", check=False)
        e[1].record()
        torch.cuda.synchronize()
        ms.append(e[0].elapsed_time(e[1]))
    if slots_t is not None:
        gathered["bge"] = out[slots_t[:4096]].double().cpu().numpy()
    t = statistics.median(ms)
    del out, ws
    # algorithmic HBM bytes of the whole call: the walk writes the table, the log-determinant
    # recursion reads one block per level and writes L (2^m sets), the rewrite pass reads and
    # writes the table and reads L once
    algo = 4 * fam + 8 * fam + 4 * 3 * (1 << w.m) + 4 * (1 << w.m)
    return {"workload": f"{w.name}, BGe score (alpha_mu 1, alpha_w m + 2)", "ms": t,
            "value": fam / (t / 1e3), "unit": UNIT,
            "hbm_frac": algo / (t / 1e3) / 1e9 / _peak_hbm()[0], "algorithmic_bytes": algo}


def _search_leg(table, m, flush, args):
    """Exact structure search (best parents + subset dynamic programme) over the FP32 table
    just scored, timed with CUDA events; the best-parent transform's algorithmic HBM bytes
    (one read and one write of value + argmin per slot and pass) give its roofline."""
    import torch
    from paper_1901_07643_gb300 import binding
    dev = table.device
    b = ctypes.c_size_t(0)
    binding.load().givensbn_structure_search_workspace_size(m, ctypes.byref(b))
    ws = torch.empty(int(b.value), dtype=torch.uint8, device=dev)
    parents, order, total = binding.structure_search(table, workspace=ws)  # warm-up
    ms, ms_bp = [], []
    best = torch.empty_like(table)
    bset = torch.empty(table.numel(), dtype=torch.int32, device=dev)
    for _ in range(3):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        binding.structure_search(table, workspace=ws)
        e[1].record()
        flush.zero_()
        e[2].record()
        binding.best_parents(table)
        e[3].record()
        torch.cuda.synchronize()
        ms.append(e[0].elapsed_time(e[1]))
        ms_bp.append(e[2].elapsed_time(e[3]))
    del best, bset, ws
    slots = m << (m - 1)
    passes = 1 + -(-max(0, (m - 1) - 12) // 7)
    bp_bytes = slots * (4 + 8) + (passes - 1) * slots * 16
    t_bp = statistics.median(ms_bp)
    peak, kind = _peak_hbm()
    return {"workload": f"optimal DAG over the m={m} FP32 table", "ms": statistics.median(ms),
            "best_parents_ms": t_bp, "best_parents_passes": passes,
            "best_parents_roofline": {"bound": "hbm", "achieved": bp_bytes / (t_bp / 1e3) / 1e9,
                                      "peak": peak, "unit": "GB/s",
                                      "frac": bp_bytes / (t_bp / 1e3) / 1e9 / peak,
                                      "algorithmic_bytes": bp_bytes, "peak_kind": kind},
            "network_score": total, "edges": int(sum(bin(p).count("1") for p in parents))}


def rotation_flops(m):
    """T(m) = 3m 2^m + 6 2^m - 3m^2 - 9m - 6: the flops of the Givens walk's rotations for m
    variables (the complexity count of Sec. 5, Table 1)."""
    return 3 * m * 2 ** m + 6 * 2 ** m - 3 * m * m - 9 * m - 6


def _aggregate(total_ms, fam, steps, world, device):
    """Whole-job throughput: every rank scores its own dataset (weak scaling),
    the timed total is the maximum over ranks (all-reduce MAX on `device`, a
    CUDA device under NCCL, the CPU under gloo), and the value counts the
    families of all ranks.  Returns (total_ms, value)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * fam * steps / (total_ms / 1e3)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1901_07643_gb300 import binding, synthetic

    rank, world, local = _dist()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = _workload(args.workload)
    X = synthetic.sem_sample(w.m, w.n, w.edge_p, w.seed + rank, w.collinear)
    fam = w.m << (w.m - 1)
    stream = torch.cuda.current_stream(dev)
    Xd = torch.from_numpy(X).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    tuned = {}

    def make(precision):
        q = args.q if (args.q and (precision == 0 or args.q <= 8)) else 0
        cw = 0
        if not q and not args.no_autotune:  # time the candidate plans, take the fastest
            q, cw, ms, table = binding.autotune(Xd, precision=precision)
            tuned["fp64" if precision else "fp32"] = {
                "q": q, "consumer_warps": cw, "median_ms": ms,
                "candidates": [{"q": a, "consumer_warps": b, "median_ms": t}
                               for a, b, t in table]}
            torch.cuda.empty_cache()
        out = torch.empty(fam, dtype=torch.float64 if precision else torch.float32, device=dev)
        ws = torch.empty(binding.workspace_size(w.n, w.m, precision, q, consumer_warps=cw),
                         dtype=torch.uint8, device=dev)

        def fn(ev):
            binding.score_all_families(Xd, out, precision=precision, q=q, consumer_warps=cw,
                                       workspace=ws, stage_events=ev, check=False)
        return fn, out, ws, q, cw

    want_errors = rank == 0 and world == 1 and not args.skip_cpu_baseline
    gathered = {}
    if want_errors:
        gathered["families"] = _error_sample(X, w.m, 1 << 18)
        slots_t = torch.from_numpy(_slots(*gathered["families"], w.m)).to(dev)

    peaks = None
    try:  # measured FMA throughput: the FP64 walk's compute roofline
        f32, f64 = binding.pipe_peaks(local)
        peaks = {"fp32_tflops": f32, "fp64_tflops": f64, "fp64_mma_tflops": binding.dmma_peak(local),
                 "how": "independent FMA (or mma.sync m8n8k4 f64) chains on every SM, "
                        "best of 3 launches (CUDA events)"}
    except Exception as e:  # noqa: BLE001 - reported, not fatal
        peaks = {"error": str(e)}

    fn32, out32, ws32, q32, cw32 = make(0)
    for _ in range(max(args.warmup, 0)):
        fn32([torch.cuda.Event(enable_timing=True) for _ in range(4)])
    binding.score_all_families(Xd, out32, q=q32, consumer_warps=cw32, workspace=ws32,
                               check=True)  # status check
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out32).all()), "non-finite scores"

    sampler = ClockSampler(_gpu_id(local)) if rank == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, walk_ms = _time_steps(fn32, args.steps, flush, stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    total_ms, value = _aggregate(sum(step_ms), fam, args.steps, world, dev)
    walk_mean = statistics.mean(walk_ms)
    if want_errors:
        gathered["fp32"] = out32[slots_t].double().cpu().numpy()
    search_leg = None if args.skip_extras else _search_leg(out32, w.m, flush, args)
    del out32, ws32
    torch.cuda.empty_cache()
    bge_leg = None if args.skip_extras else _bge_leg(
        Xd, w, flush, slots_t if want_errors else None, gathered)
    torch.cuda.empty_cache()

    fp64 = None
    if not args.skip_fp64:
        fn64, out64, ws64, q64, cw64 = make(1)
        for _ in range(max(args.warmup, 1)):
            fn64([torch.cuda.Event(enable_timing=True) for _ in range(4)])
        k64 = max(3, args.steps // 2)
        s64, w64 = _time_steps(fn64, k64, flush, stream)
        fp64 = {"value": fam * k64 / (sum(s64) / 1e3), "ms_per_step": statistics.mean(s64),
                "walk_ms": statistics.mean(w64),
                "q": q64 or binding.auto_q(w.m, 1), "consumer_warps": cw64 or None,
                "dtype": "f64", "steps": k64}
        if peaks and "fp64_tflops" in peaks:
            wsec = statistics.mean(w64) / 1e3
            ach = rotation_flops(w.m) / wsec / 1e12
            fp64["roofline"] = {
                "bound": "fp64", "achieved": ach, "peak": peaks["fp64_tflops"],
                "unit": "TFLOP/s", "frac": ach / peaks["fp64_tflops"], "peak_kind": "measured",
                "algorithmic_flops": rotation_flops(w.m),
                "note": "rotation flops T(m) of Sec. 5 only; each family also takes an FP64 "
                        "logarithm (a software routine) that the count leaves out",
                "hbm_frac": 8 * fam / wsec / 1e9 / _peak_hbm()[0]}
        if want_errors:
            gathered["fp64"] = out64[slots_t].cpu().numpy()
        del out64, ws64
        torch.cuda.empty_cache()

    e2e = None
    if not args.skip_e2e:
        e2e = _e2e(X, Xd, fam, q32, cw32, w, world, dev, args)

    extras = {} if args.skip_extras else _extras(dev, flush, args)

    cpu, errors = None, None
    if want_errors:
        cpu, errors = _cpu_baseline(X, w.n, w.m, args.cpu_seconds, gathered)

    peak, peak_kind = _peak_hbm()
    algo_bytes = 4 * fam  # the fp32 score table written once
    achieved = algo_bytes / (walk_mean / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "families": fam,
                   "q": q32 or binding.auto_q(w.m, 0), "consumer_warps": cw32 or None,
                   "plan": "autotuned (givensbn_autotune)" if tuned.get("fp32") else "fixed",
                   "precision": "fp32 walk, fp64 CholeskyQR2 R0",
                   "l2": "256 MiB buffer zeroed between timed steps (> 129 MB L2); each step "
                         f"also writes a {fam * 4 / 1e9:.3g} GB table",
                   "parallelism": f"replicas x{world}, one dataset per GPU"},
        "fp64": fp64,
        "speedup_fp32_vs_fp64": (value / world) / fp64["value"] if fp64 else None,
        "walk_ms": walk_mean,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": _traffic(w.name, q32 or binding.auto_q(w.m, 0)),
                     "peak_kind": peak_kind, "kernel": _walk_kernel_name(w.m, q32 or binding.auto_q(w.m, 0)),
                     "algorithmic_bytes_per_launch": algo_bytes},
        "cpu_baseline": cpu,
        "errors": errors,
        "pipe_peaks": peaks,
        "autotune": tuned or None,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
    }
    line.update(extras)
    if search_leg:
        line["structure_search"] = search_leg
    if bge_leg:
        line["bge"] = bge_leg
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
