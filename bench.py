#!/usr/bin/env python3
"""Benchmark: segment-pair evaluations per second of the batched linking-number
verify on one (or N) GB300, mixed precision against the all-FP64 direct sum.

Workload (one "step"): verify every AABB-candidate loop pair of a seeded
synthetic 4-in-1 chainmail sheet (2,048 rings of radius 1 x 256 segments on a
32 x 64 grid, FP32 vertices; 11,653 candidate pairs, 7.6e8 segment pairs) --
the whole hot path: pair frames, persistent tile sweep, careful re-sweep,
FP64 recompute of near segment pairs, per-pair reduction and rounding.  The
step is one replay of the CUDA graph that lk_plan_create captured; inputs are
resident in HBM; L2 is flushed (256 MB write) before every timed step.

`--impl reference` times the FP64 CPU oracle on the same workload instead.
Under torchrun each rank verifies its own sheet (weak scaling, no collective
on the data path).

The other workloads (ring chain, knit yarn, torus links, serving piles and
the paper's stress shapes) are reported in blocks after the headline keys,
and a compact "summary" of them ends the line.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "segment-pair evals/s and p99 verify latency, mixed-prec vs FP64, 1 GB300"
UNIT = "segment-pair evals/s"
# Algorithmic FP32 work per segment pair (FMA = 2 flops): the amortised
# closed-form term with shared grid norms and edge dot products.
FLOPS_PER_SP = 58.0
# FP32 lanes per SM of this GPU generation and its maximum SM clock; the SM
# count is read from the device (152 on a GB300): peak = SMs x 128 x 2 x clock.
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# Kernels one chainmail step launches: pair_frames, sweep_packed, careful_chunk,
# sweep_careful (all fast variant: the sheet has no accurate-variant pair, so
# those launches are skipped), near_fix, reduce.
KERNELS_PER_STEP = 6
# DRAM bytes (read + write) of one sweep_packed_kernel<fast> launch on this
# workload, from one ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum); set to None whenever the kernel changes.
SWEEP_TRAFFIC_BYTES = 10007296


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-stress", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--precise-only", action="store_true",
                    help="verify one woundball pair (nu = 10^3, 2 x 10^5 segments) twice, which the precise "
                         "variant sums: for profiling that kernel")
    ap.add_argument("--accurate-only", action="store_true",
                    help="verify one (5,7) torus link of 2 x 100,000 segments (the accurate variant) three "
                         "times: for profiling that variant of the bulk sweep")
    ap.add_argument("--serving-only", action="store_true",
                    help="the serving capacity alone (closed loop of 32, --serving-requests requests after 40 "
                         "warm-up ones): for launch lists under a profiler")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the headline step only (no tuning, FP64 baseline, end-to-end or other blocks): "
                         "for launch lists under a profiler")
    return ap.parse_args()


def cpu_model() -> str:
    """The host CPU's model string (lscpu), for the CPU baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for key in ("Model name:", "Vendor ID:"):
            for ln in out.splitlines():
                if ln.strip().startswith(key):
                    return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def err_stats(raw, ref):
    """|raw - ref| per result: max, p99 and the index of the max."""
    d = np.abs(np.asarray(raw, np.float64) - np.asarray(ref, np.float64))
    if d.size == 0:
        return {"max": 0.0, "p99": 0.0, "argmax": -1, "n": 0}
    return {"max": float(d.max()), "p99": float(np.percentile(d, 99)), "argmax": int(np.argmax(d)), "n": int(d.size)}


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(rank: int):
    from paper_2106_12655_gb300 import workloads as W

    g = W.chainmail(seed=2 + rank)
    desc = ("4-in-1 chainmail sheet: 32x64 rings of radius 1, 256 segments each, FP32 vertices, "
            "seeded perturbation sigma=0.02, all AABB-candidate pairs")
    return g, desc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def serving_block(args):
    """Open-loop Poisson serving over resident chainmail piles (500-14,000 rings,
    64-256 segments per ring, 1k-20k pairs per request) with the default
    server (lists packed on the device): capacity, then p50/p99 latency at
    50/80/95% of it; then the same at 80% with host packing and with the
    fewest-items-first wave order."""
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import serving as S

    scenes = S.make_scenes(seed=5, n_scenes=6)
    srv = lk.lk_server_create(None)
    try:
        warm = S.request_plan(scenes, 40, seed=99)
        S.run(srv, scenes, warm, None)
        # capacity: a closed loop of at most 32 requests queued or running, so
        # that the host packing of later requests overlaps the device work
        cap_plan = S.request_plan(scenes, max(100, args.serving_requests // 2), seed=1)
        lat, wall, bad, _ = S.run(srv, scenes, cap_plan, None, max_outstanding=32)
        pairs, sps = S.plan_sizes(scenes, cap_plan)
        cap = len(cap_plan) / wall
        out = {"scenes": [{"rings": sc.geometry.n_loops, "vertices": int(sc.geometry.vertices.shape[0]),
                           "pairs": int(sc.geometry.pairs.shape[0])} for sc in scenes],
               "capacity": {"req_per_s": cap, "pairs_per_s": pairs.sum() / wall, "sp_per_s": sps.sum() / wall,
                            "n_requests": len(cap_plan), "nonok_pair_status": bad, "outstanding": 32},
               "loads": []}
        for load in (0.5, 0.8, 0.95):
            plan = S.request_plan(scenes, args.serving_requests, seed=int(load * 100))
            rec = {}
            lat, wall, bad, _ = S.run(srv, scenes, plan, rate_per_s=load * cap, seed=int(load * 1000), record=rec)
            pairs, sps = S.plan_sizes(scenes, plan)
            out["loads"].append({"load": load, "offered_req_per_s": load * cap, "req_per_s": len(plan) / wall,
                                 "pairs_per_s": pairs.sum() / wall, "sp_per_s": sps.sum() / wall,
                                 "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                                 "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                                 "n_requests": len(plan), "nonok_pair_status": bad,
                                 "tail": tail_breakdown(lat, sps, rec)})
        out["server_stats"] = lk.lk_server_get_stats(srv)
        out["host_packing"] = server_variant_block(args, scenes, cap, pack_on_device=0)
        out["fewest_items_first"] = server_variant_block(args, scenes, cap, wave_order=1)
        out["potential_link_search"] = pls_block(scenes)
        out["potential_link_search_large"] = pls_large_block()
        out["batched_same_piles"] = batched_piles_block(scenes)
        return out
    finally:
        lk.lk_server_destroy(srv)
        S.close(scenes)


def server_variant_block(args, scenes, cap, load=0.8, **options):
    """A server with other options on the same piles: its closed-loop capacity
    (32 outstanding), then the 80%-load plan at the default server's offered
    rate (0.8 x `cap`), with the tail breakdown."""
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import serving as S

    o = lk.lk_server_default_options()
    for k, v in options.items():
        setattr(o, k, v)
    srv = lk.lk_server_create(o)
    try:
        S.run(srv, scenes, S.request_plan(scenes, 40, seed=99), None, max_outstanding=32)
        cap_plan = S.request_plan(scenes, max(100, args.serving_requests // 2), seed=1)
        _, wall, bad_cap, _ = S.run(srv, scenes, cap_plan, None, max_outstanding=32)
        plan = S.request_plan(scenes, args.serving_requests, seed=int(load * 100))
        rec = {}
        lat, wall2, bad, _ = S.run(srv, scenes, plan, rate_per_s=load * cap, seed=int(load * 1000), record=rec)
        pairs, sps = S.plan_sizes(scenes, plan)
        return {"options": options, "capacity_req_per_s": len(cap_plan) / wall, "load": load,
                "offered_req_per_s": load * cap, "req_per_s": len(plan) / wall2,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "n_requests": len(plan), "nonok_pair_status": bad + bad_cap, "tail": tail_breakdown(lat, sps, rec)}
    finally:
        lk.lk_server_destroy(srv)


def tail_breakdown(lat, sps, rec):
    """Where the latency tail comes from: p50/p99 of the smallest and the
    largest third of the requests (by segment pairs), of the requests that
    found at most 2 / at least 8 others outstanding when they were submitted,
    and the share of the p99-and-above requests that arrived behind 8 or more."""
    lat = np.asarray(lat) * 1e3
    depth = rec["depth"]
    lo, hi = np.percentile(sps, [33.3, 66.7])
    q99 = np.percentile(lat, 99)

    def pct(mask):
        return ({"n": int(mask.sum()), "p50_ms": float(np.percentile(lat[mask], 50)),
                 "p99_ms": float(np.percentile(lat[mask], 99))} if mask.any() else {"n": 0})

    return {"small_third": pct(sps <= lo), "large_third": pct(sps >= hi),
            "depth_le_2": pct(depth <= 2), "depth_ge_8": pct(depth >= 8),
            "p99_tail_behind_8_or_more": float(np.mean(depth[lat >= q99] >= 8)),
            "mean_depth": float(depth.mean()), "max_submit_late_ms": 1e3 * float(np.max(rec["late"]))}


def geometry_serving_block(args):
    """Requests that carry geometry only: each verifies every potential link of
    one of six resident piles (170-3,500 rings, 64-256 segments per ring, so
    about 1k-20k candidate pairs), after a small displacement of the pile.
    Served two ways on the same piles: the device search and packing of
    lk_server_submit_geometry, and a host round trip (lk_candidates on the
    server's stream, then lk_server_submit of the list).  Closed-loop capacity
    (32 outstanding), then p50/p99 at 50% and 80% of each way's capacity."""
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import serving as S

    scenes = S.make_scenes(seed=7, n_scenes=6, min_rings=170, max_rings=3500)
    srv = lk.lk_server_create(None)
    try:
        out = {"scenes": [{"rings": sc.geometry.n_loops, "pairs": int(sc.geometry.pairs.shape[0])} for sc in scenes]}
        for mode in ("geometry", "host_search"):
            S.run(srv, scenes, S.geometry_plan(scenes, 40, seed=98), None, max_outstanding=32, mode=mode)
            plan = S.geometry_plan(scenes, max(100, args.serving_requests // 2), seed=2)
            lat, wall, bad, verified = S.run(srv, scenes, plan, None, max_outstanding=32, mode=mode)
            cap = len(plan) / wall
            res = {"capacity": {"req_per_s": cap, "pairs_per_s": verified / wall, "n_requests": len(plan),
                                "nonok_pair_status": bad}, "loads": []}
            for load in (0.5, 0.8):
                plan = S.geometry_plan(scenes, args.serving_requests, seed=int(load * 100) + 1)
                lat, wall, bad, verified = S.run(srv, scenes, plan, rate_per_s=load * cap, seed=int(load * 1000) + 1,
                                                 mode=mode)
                res["loads"].append({"load": load, "offered_req_per_s": load * cap, "req_per_s": len(plan) / wall,
                                     "pairs_per_s": verified / wall,
                                     "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                                     "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                                     "n_requests": len(plan), "nonok_pair_status": bad})
            out[mode] = res
        out["server_stats"] = lk.lk_server_get_stats(srv)
        return out
    finally:
        lk.lk_server_destroy(srv)
        S.close(scenes)


def batched_piles_block(scenes):
    """The serving piles verified in one batch each (lk_verify of every
    candidate pair of the pile, device-resident lists and results, CUDA
    events, median of 5 after 2 warm-ups): the device rate the serving
    capacity compares with."""
    import torch
    from paper_2106_12655_gb300 import lk

    stream = torch.cuda.current_stream()
    sp_total, ms_total, per = 0, 0.0, []
    for sc in scenes:
        pairs = torch.from_numpy(np.ascontiguousarray(sc.geometry.pairs)).cuda()
        n = pairs.shape[0]
        o = (torch.zeros(n, dtype=torch.int32, device="cuda"), torch.zeros(n, dtype=torch.float64, device="cuda"),
             torch.zeros(n, dtype=torch.int32, device="cuda"))
        ts = []
        for rep in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lk.lk_verify(sc.ctx, pairs, *o, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if rep >= 2:
                ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        sp = int(sc.geometry.segment_pairs(sc.geometry.pairs))
        per.append({"pairs": n, "ms": ms, "sp_per_s": sp / (ms * 1e-3)})
        sp_total += sp
        ms_total += ms
    return {"sp_per_s": sp_total / (ms_total * 1e-3), "piles": per}


def pls_block(scenes):
    """Device potential link search (lk_candidates) on each resident pile:
    wall time of the synchronous call (median of 10) and whether its list
    equals the pile's candidate list."""
    import torch
    from paper_2106_12655_gb300 import lk

    out = []
    for sc in scenes:
        n = lk.lk_candidates(sc.ctx, np.zeros((0, 2), np.int32))
        buf = torch.zeros((max(n, 1), 2), dtype=torch.int32, device="cuda")
        ts = []
        for _ in range(12):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lk.lk_candidates(sc.ctx, buf)
            ts.append(time.perf_counter() - t0)
        got = buf[:n].cpu().numpy()
        want = np.ascontiguousarray(sc.geometry.pairs)
        out.append({"rings": sc.geometry.n_loops, "candidates": n, "ms": 1e3 * statistics.median(ts[2:]),
                    "box_tests_per_s": sc.geometry.n_loops * (sc.geometry.n_loops - 1) / 2 / statistics.median(ts[2:]),
                    "equals_pile_pairs": bool(got.shape == want.shape and np.array_equal(got, want))})
    return out


def pls_large_block(rows=250, cols=400, nseg=32):
    """The device potential link search on a 100,000-ring chainmail pile
    (sort and sweep: above 2^27 box pairs): wall time of the synchronous call
    into a device buffer (median of 10 after 2), and whether its list equals
    the pile's candidate list from the host's sort and sweep."""
    import torch
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import workloads as W

    g = W.chainmail(seed=31, rows=rows, cols=cols, nseg=nseg)
    ctx = lk.lk_create(g.vertices, g.offsets)
    try:
        n = lk.lk_candidates(ctx, np.zeros((0, 2), np.int32))
        buf = torch.zeros((max(n, 1), 2), dtype=torch.int32, device="cuda")
        ts = []
        for _ in range(12):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lk.lk_candidates(ctx, buf)
            ts.append(time.perf_counter() - t0)
        got = buf[:n].cpu().numpy()
    finally:
        lk.lk_destroy(ctx)
    want = np.ascontiguousarray(g.pairs)
    ms = 1e3 * statistics.median(ts[2:])
    return {"rings": g.n_loops, "segments_per_ring": nseg, "candidates": n, "ms": ms,
            "box_pairs": g.n_loops * (g.n_loops - 1) // 2,
            "equals_pile_pairs": bool(got.shape == want.shape and np.array_equal(got, want))}


def counting_crossings_block(g, v, off, pairs_d, lk_ref, stream, flush, steps=20, search=None):
    """The counting-crossings method (LK_METHOD_CC) on the same sheet and graph
    protocol: device time per step, and whether its linking numbers equal the
    direct sum's.  Its results are exact integers where the crossings decide a
    pair.  ``search`` picks the candidate search (default: the built-in choice,
    here the one-CTA binned search for every pair)."""
    import torch
    from paper_2106_12655_gb300 import lk

    n = g.pairs.shape[0]
    o = lk.lk_default_options()
    o.method = lk.LK_METHOD_CC
    o.timing = 1
    if search is not None:
        o.cc_search = search
    ctx = lk.lk_create(v, off, o, stream)
    plan = lk.lk_plan_create(ctx, pairs_d, stream)
    lo = torch.zeros(n, dtype=torch.int32, device=v.device)
    raw = torch.zeros(n, dtype=torch.float64, device=v.device)
    st = torch.zeros(n, dtype=torch.int32, device=v.device)
    ms, sweep = [], []
    try:
        for k in range(steps + 3):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lk.lk_plan_run(plan, lo, raw, st, stream, ctx=ctx)
            e1.record(stream)
            e1.synchronize()
            if k >= 3:
                ms.append(e0.elapsed_time(e1))
                sweep.append(lk.lk_get_stats(ctx)["sweep_ms"])
        stats = lk.lk_get_stats(ctx)
        lo_h, raw_h, st_h = lo.cpu().numpy(), raw.cpu().numpy(), st.cpu().numpy()
    finally:
        lk.lk_plan_destroy(plan)
        lk.lk_destroy(ctx)
    med = statistics.median(ms)
    return {"value": g.segment_pairs() / (med / 1e3), "unit": UNIT, "ms_per_step": med,
            "sweep_ms": statistics.median(sweep), "candidates": stats["cc_candidates"],
            "fallback_pairs": stats["cc_fallback_pairs"],
            "lk_equal_direct_sum": bool(np.array_equal(lo_h, lk_ref)),
            "exact_integer_raw": bool(np.all(raw_h == lo_h)), "all_status_ok": bool(np.all(st_h == 0))}


def per_pair_block(g, v, off, lk_ref, stream, n_sample=512, seed=9):
    """The sheet verified one pair per call, the structure of the paper's GPU
    path (one kernel launch per loop pair, Sec. 3.4), against the batched step:
    a seeded sample of pairs, each through its own lk_verify (its pair from
    host memory, which the call packs without any device read-back, and its
    results to device memory; the call launches its own kernels), timed with
    CUDA events around the whole sample after one untimed pass; the per-step
    figure scales the per-pair time to all pairs of the sheet."""
    import torch
    from paper_2106_12655_gb300 import lk

    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(g.pairs.shape[0], min(n_sample, g.pairs.shape[0]), replace=False))
    sample = [np.ascontiguousarray(g.pairs[k:k + 1]) for k in pick]
    lo = torch.zeros(len(pick), dtype=torch.int32, device=v.device)
    raw = torch.zeros(len(pick), dtype=torch.float64, device=v.device)
    st = torch.zeros(len(pick), dtype=torch.int32, device=v.device)
    ctx = lk.lk_create(v, off, None, stream)
    try:
        for rep_ in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k, pd in enumerate(sample):
                lk.lk_verify(ctx, pd, lo[k:k + 1], raw[k:k + 1], st[k:k + 1], stream)
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1)
        lo_h = lo.cpu().numpy()
    finally:
        lk.lk_destroy(ctx)
    per_pair = ms / len(pick)
    sps = g.sizes()[g.pairs[pick]].prod(axis=1).sum()
    return {"pairs_sampled": int(len(pick)), "ms_per_pair": per_pair,
            "ms_per_step_scaled": per_pair * g.pairs.shape[0],
            "value": float(sps) / (ms / 1e3), "unit": UNIT,
            "lk_equal_batched": bool(np.array_equal(lo_h, lk_ref[pick])),
            "all_status_ok": bool(np.all(st.cpu().numpy() == 0))}


def early_exit_block(g, v, off, lk_ref, stream, batch=1 << 27, reps=5):
    """Sec. 3.1's fast verification on the sheet (lk_verify_expected, batches
    of 2^27 segment pairs, all enqueued at once; the first batch with a changed
    linking number stops the later ones on the device): CUDA-event time of a
    full check against the sheet's own certificate, and of a check whose
    certificate differs at pair 100 (a "pull-through" among the first items),
    each the median of `reps` after two untimed calls (the second call with the
    same list builds the graph of the batched sequence that later calls
    replay)."""
    import torch
    from paper_2106_12655_gb300 import lk

    cert = np.ascontiguousarray(lk_ref.astype(np.int32))
    bad = cert.copy()
    bad[100] += 1
    pairs_d = torch.from_numpy(np.ascontiguousarray(g.pairs)).cuda()
    ctx = lk.lk_create(v, off, None, stream)
    out = {}
    try:
        for label, c in (("full", cert), ("changed_at_100", bad)):
            cd = torch.from_numpy(c).cuda()
            ms, res = [], None
            for k in range(reps + 2):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = lk.lk_verify_expected(ctx, pairs_d, cd, batch, stream=stream)
                e1.record(stream)
                e1.synchronize()
                if k >= 2:
                    ms.append(e0.elapsed_time(e1))
            out[label] = {"ms": statistics.median(ms), "first_mismatch": int(res[0]), "pairs_checked": int(res[1])}
    finally:
        lk.lk_destroy(ctx)
    out["batch_segment_pairs"] = batch
    out["pairs"] = int(g.pairs.shape[0])
    return out


def timed_verify(ctx, pd, n, stream, warm, reps, device):
    """CUDA-event times (ms) of `reps` verifies of the device pair list after
    `warm` untimed ones, and the last results (host arrays)."""
    import torch
    from paper_2106_12655_gb300 import lk

    lo = torch.zeros(n, dtype=torch.int32, device=device)
    raw = torch.zeros(n, dtype=torch.float64, device=device)
    st = torch.zeros(n, dtype=torch.int32, device=device)
    ms = []
    for k in range(warm + reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lk.lk_verify(ctx, pd, lo, raw, st, stream)
        e1.record(stream)
        e1.synchronize()
        if k >= warm:
            ms.append(e0.elapsed_time(e1))
    est = np.zeros(n)
    try:
        lk.lk_get_error_estimates(ctx, est)
    except lk.LkError:
        est[:] = np.nan
    return ms, lo.cpu().numpy(), raw.cpu().numpy(), st.cpu().numpy(), est


def stress_block(stream):
    """The paper's large-input stress shapes (Sec. 4, Table 1): the two
    double-helix ribbons (2 x 10^5 segments, lk = 10 and 1000), the woundballs
    (nu = 10^3 with 10^6 segments and nu = 10^4 with 2 x 10^6, lk = 0) and the
    two thick square links (1,250 loops, 5x10^5 segments, 390,625 pairs, and
    5,000 loops, 4x10^6 segments, 6,250,000 pairs, all lk = 1, from the
    device's potential link search), each by the direct sum and by counting
    crossings.  Each direct-sum record gives the raw error against the closed
    form, the library's own error estimate and how many pairs the compensated
    (precise) sweep summed again.  Times are CUDA-event medians of the timed
    verifies after untimed ones (the first packs the list and sizes the work
    lists -- the largest shape gets them sized up front --, the second, the
    list's first repeat, builds its graph plan, so the timed verifies replay
    that plan); the largest shapes are timed once."""
    import torch
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import workloads as W

    out = {}
    big = {"near_capacity": 1_400_000_000, "chunk_capacity": 1 << 26, "cc_capacity": 1 << 26}
    for name, make, expect, opts, warm, reps, methods in (
            ("ribbon_lk10", lambda: W.double_helix_ribbon(10, 100_000), 10, {}, 2, 3, ("ds",)),
            ("ribbon_lk1000", lambda: W.double_helix_ribbon(1000, 100_000), 1000, {}, 2, 3, ("ds",)),
            ("woundball_nu1000", lambda: W.woundball(1000, 500_000), 0, {}, 2, 2, ("ds", "cc")),
            ("woundball_nu10000", lambda: W.woundball(10_000, 1_000_000), 0, {"cc_capacity": 1 << 29}, 1, 1,
             ("ds", "cc")),
            ("square_links_1250", lambda: W.square_links(625, 400), 1, {}, 3, 3, ("ds", "cc")),
            ("square_links_5000", lambda: W.square_links(2500, 800), 1, big, 3, 1, ("ds", "cc"))):
        g = make()
        g.vertices = g.vertices.astype(np.float32)
        v = torch.from_numpy(g.vertices).cuda()
        off = torch.from_numpy(g.offsets).cuda()
        rec = {"loops": g.n_loops, "segments": int(g.vertices.shape[0])}
        for label in methods:
            method = lk.LK_METHOD_DS if label == "ds" else lk.LK_METHOD_CC
            o = lk.lk_default_options()
            o.method = method
            for k, val in opts.items():
                setattr(o, k, val)
            ctx = lk.lk_create(v, off, o, stream)
            try:
                if g.pairs.shape[0] == 1:
                    pairs = g.pairs
                else:
                    pairs = lk.lk_candidates(ctx, stream=stream)
                n = pairs.shape[0]
                pd = torch.from_numpy(np.ascontiguousarray(pairs)).cuda()
                ms, lo_h, raw_h, st_h, est = timed_verify(ctx, pd, n, stream, warm, reps, v.device)
                stats = lk.lk_get_stats(ctx)
            finally:
                lk.lk_destroy(ctx)
            sps = g.segment_pairs(pairs)
            med = statistics.median(ms)
            ref = np.sign(lo_h) * float(expect) if expect else np.zeros(n)
            r = {"value": sps / (med / 1e3), "unit": UNIT, "ms": med, "pairs": int(n), "segment_pairs": int(sps),
                 "lk_all_expected": bool(np.all(np.abs(lo_h) == expect)), "all_status_ok": bool(np.all(st_h == 0)),
                 "max_abs_raw_err": float(np.max(np.abs(np.abs(raw_h) - expect))),
                 "raw_err_vs_closed_form": err_stats(raw_h, ref),
                 "max_error_estimate": float(np.nanmax(est)) if n else 0.0,
                 "fp64_recomputed_segment_pairs": stats["fp64_pairs"], "precise_pairs": stats["precise_pairs"]}
            if method == lk.LK_METHOD_CC:
                r["candidates"] = stats["cc_candidates"]
                r["fallback_pairs"] = stats["cc_fallback_pairs"]
            rec["direct_sum" if label == "ds" else "counting_crossings"] = r
        out[name] = rec
    return out


def configs_block(stream, reps=3, oracle_threads=None):
    """The other workloads of the benchmark's configurations, each verified
    through lk_verify with the pair list in pinned host memory and the results
    on the device (CUDA-event medians of `reps` verifies after untimed ones)
    and, where the FP64 oracle can run in seconds, checked against it
    result by result (max, p99 and argmax of |raw - oracle|):
      * ring chain: 16 rings x 128 segments, FP64 vertices, all 120 pairs
        (latency-bound; the oracle runs on every pair);
      * knit yarn: 600 stitch loops of 1k-20k segments, all AABB candidates;
        the all-FP64 GPU direct sum is timed on a seeded ~3% sample of the
        pairs (its rate, extrapolated to the whole sheet), and a seeded 10%
        sample of the pairs (with the 20 largest) is compared with the oracle;
      * torus links (2p,2q), R = 3, r = 1: every (p,q) of {(2,3), (5,7),
        (11,13), (31,37)} at 250k segments per component, and (5,7), (11,13),
        (31,37) at 500k, 750k and 1M; error against the closed form |lk| = pq;
        the all-FP64 GPU path's rate is measured on a 2 x 25k-segment (31,37)
        link and the oracle's on a seeded sample of 64 column segments (row
        sums of Eq. 3) of each link, both extrapolated by segment-pair count
        and labelled so."""
    import torch
    from oracle import oracle as O
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import workloads as W

    threads = oracle_threads or O.default_threads()

    def verify(g, pairs=None, warm=2, reps_=reps, **opts):
        pairs = g.pairs if pairs is None else pairs
        v = torch.from_numpy(np.ascontiguousarray(g.vertices)).cuda()
        off = torch.from_numpy(g.offsets).cuda()
        o = lk.lk_default_options()
        for k, val in opts.items():
            setattr(o, k, val)
        ctx = lk.lk_create(v, off, o, stream)
        try:
            # the list in pinned host memory, where a caller keeps it (a device
            # list is read back to the host, with a synchronisation, each call)
            pd = torch.from_numpy(np.ascontiguousarray(pairs)).pin_memory()
            ms, lo, raw, st, est = timed_verify(ctx, pd, pairs.shape[0], stream, warm, reps_, v.device)
            stats = lk.lk_get_stats(ctx)
        finally:
            lk.lk_destroy(ctx)
        return statistics.median(ms), lo, raw, st, est, stats

    out = {}
    # ring chain (config 1)
    g = W.ring_chain()
    med, lo, raw, st, est, _ = verify(g, warm=3, reps_=10)
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs, threads=threads)
    out["ring_chain"] = {"pairs": int(g.pairs.shape[0]), "segment_pairs": g.segment_pairs(), "ms": med,
                         "value": g.segment_pairs() / (med / 1e3), "unit": UNIT,
                         "lk_equal_oracle": bool(np.array_equal(lo, O.round_lk(ref))),
                         "all_status_ok": bool(np.all(st == 0)), "raw_err_vs_oracle": err_stats(raw, ref),
                         "max_error_estimate": float(np.max(est))}
    # knit yarn (config 3)
    g = W.knit_yarn()
    med, lo, raw, st, est, stats = verify(g)
    sizes = g.sizes()[g.pairs].prod(axis=1)
    rng = np.random.default_rng(31)
    pick64 = np.sort(rng.choice(g.pairs.shape[0], max(1, g.pairs.shape[0] // 32), replace=False))
    med64, _, raw64, _, _, _ = verify(g, g.pairs[pick64], warm=1, reps_=1, precision=lk.LK_ALL_F64)
    sps64 = float(sizes[pick64].sum())
    order = np.argsort(sizes)
    pick = np.unique(np.concatenate([order[-20:], np.random.default_rng(7).choice(
        g.pairs.shape[0], g.pairs.shape[0] // 10, replace=False)]))
    t0 = time.perf_counter()
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs[pick], threads=threads)
    t_or = time.perf_counter() - t0
    e = err_stats(raw[pick], ref)
    e["argmax_pair"] = int(pick[e["argmax"]]) if e["n"] else -1
    out["knit_yarn"] = {"loops": g.n_loops, "pairs": int(g.pairs.shape[0]), "segment_pairs": int(sizes.sum()),
                        "ms": med, "value": float(sizes.sum()) / (med / 1e3), "unit": UNIT,
                        "all_status_ok": bool(np.all(st == 0)), "precise_pairs": stats["precise_pairs"],
                        "fp64_gpu": {"value": sps64 / (med64 / 1e3), "unit": UNIT, "pairs_timed": int(pick64.size),
                                     "segment_pairs_timed": int(sps64),
                                     "ms_whole_sheet_extrapolated": med64 * float(sizes.sum()) / sps64},
                        "speedup_mixed_over_fp64": (float(sizes.sum()) / (med / 1e3)) / (sps64 / (med64 / 1e3)),
                        "max_abs_raw_minus_fp64_gpu": float(np.max(np.abs(raw[pick64] - raw64))),
                        "oracle_sample": {"pairs": int(pick.size), "segment_pairs": int(sizes[pick].sum()),
                                          "seconds": t_or, "threads": threads,
                                          "lk_equal": bool(np.array_equal(lo[pick], O.round_lk(ref)))},
                        "raw_err_vs_oracle": e, "max_abs_raw_minus_lk": float(np.max(np.abs(raw - lo))),
                        "max_error_estimate": float(np.max(est))}
    # torus links (config 4)
    g = W.torus_link(31, 37, 25_000, dtype=np.float32)
    med64, _, _, _, _, _ = verify(g, warm=1, reps_=1, precision=lk.LK_ALL_F64)
    fp64_rate = g.segment_pairs() / (med64 / 1e3)
    tl = []
    for p, q, n in ((2, 3, 250_000), (5, 7, 250_000), (11, 13, 250_000), (31, 37, 250_000),
                    (5, 7, 500_000), (11, 13, 750_000), (31, 37, 1_000_000)):
        g = W.torus_link(p, q, n, dtype=np.float32)
        med, lo, raw, st, est, stats = verify(g, warm=1, reps_=2)
        sps = g.segment_pairs()
        rows = np.sort(np.random.default_rng(p * q).choice(n, 64, replace=False))
        t0 = time.perf_counter()
        O.link_rows(g.loop(0), g.loop(1), rows, threads=threads)
        t_or = time.perf_counter() - t0
        tl.append({"p": p, "q": q, "segments_per_component": n, "segment_pairs": sps, "ms": med,
                   "value": sps / (med / 1e3), "unit": UNIT, "lk": int(lo[0]), "closed_form_abs_lk": p * q,
                   "abs_raw_err_vs_closed_form": float(abs(abs(raw[0]) - p * q)), "status_ok": bool(st[0] == 0),
                   "error_estimate": float(est[0]), "precise": bool(stats["precise_pairs"]),
                   "fp64_gpu_s_extrapolated": sps / fp64_rate,
                   "oracle_s_extrapolated": t_or * n / rows.size,
                   "oracle_sample": "64 seeded column segments of the %d (row sums of Eq. 3), %d threads" % (n, threads)})
    out["torus_links"] = {"fp64_gpu_rate": {"value": fp64_rate, "unit": UNIT,
                                            "measured_on": "(31,37) torus link, 2 x 25,000 segments"},
                          "links": tl}
    return out


def tuning_block(g, v, off, pairs_d, stream, flush, steps=20):
    """The autotuner on the sheet: lk_autotune's table against the built-in
    work-item heights, same graph protocol as the headline (L2 flushed before
    each timed replay); the headline uses whichever was faster."""
    import torch
    from paper_2106_12655_gb300 import lk

    res = {}
    n = g.pairs.shape[0]
    lo = torch.zeros(n, dtype=torch.int32, device=v.device)
    raw = torch.zeros(n, dtype=torch.float64, device=v.device)
    st = torch.zeros(n, dtype=torch.int32, device=v.device)
    table = None
    for label in ("default", "tuned"):
        ctx = lk.lk_create(v, off, None, stream)
        try:
            if label == "tuned":
                t0 = time.perf_counter()
                lk.lk_autotune(ctx, g.pairs, stream)
                res["tune_seconds"] = time.perf_counter() - t0
                table = lk.lk_tune_get(ctx)
                res["table"] = table.reshape(-1, 3).tolist()
            plan = lk.lk_plan_create(ctx, pairs_d, stream)
            ms = []
            for k in range(steps + 3):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                lk.lk_plan_run(plan, lo, raw, st, stream, ctx=ctx)
                e1.record(stream)
                e1.synchronize()
                if k >= 3:
                    ms.append(e0.elapsed_time(e1))
            lk.lk_plan_destroy(plan)
        finally:
            lk.lk_destroy(ctx)
        res[label + "_ms"] = statistics.median(ms)
    res["use_tuned"] = bool(res["tuned_ms"] < res["default_ms"])
    return res, (table if res["use_tuned"] else None)


def tuning_other_block(stream, reps=7):
    """The autotuner on the knit yarn and on the six serving piles: one
    lk_verify of every candidate pair (device lists and results, L2 flushed
    before each, CUDA events, median of `reps` after one warm-up) with the
    built-in work-item heights and with lk_autotune's table, and the largest
    difference between the two tables' raw sums (the tables only reorder the
    FP64 sums)."""
    import torch
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import serving as S

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(ctx, pairs_d, out):
        ms = []
        for k in range(reps + 1):
            flush.fill_(k & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lk.lk_verify(ctx, pairs_d, *out, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if k:
                ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    def compare(geoms):
        res = {"default_ms": 0.0, "tuned_ms": 0.0, "tune_seconds": 0.0, "max_abs_raw_diff": 0.0, "tables": []}
        for g in geoms:
            v = torch.from_numpy(g.vertices).cuda()
            off = torch.from_numpy(g.offsets).cuda()
            pairs_d = torch.from_numpy(np.ascontiguousarray(g.pairs)).cuda()
            n = g.pairs.shape[0]
            raws = []
            for label in ("default", "tuned"):
                out = (torch.zeros(n, dtype=torch.int32, device="cuda"),
                       torch.zeros(n, dtype=torch.float64, device="cuda"),
                       torch.zeros(n, dtype=torch.int32, device="cuda"))
                ctx = lk.lk_create(v, off, None, stream)
                try:
                    if label == "tuned":
                        t0 = time.perf_counter()
                        lk.lk_autotune(ctx, g.pairs, stream)
                        res["tune_seconds"] += time.perf_counter() - t0
                        res["tables"].append(lk.lk_tune_get(ctx).reshape(-1, 3).tolist())
                    res[label + "_ms"] += timed(ctx, pairs_d, out)
                    raws.append(out[1].cpu().numpy())
                finally:
                    lk.lk_destroy(ctx)
            res["max_abs_raw_diff"] = max(res["max_abs_raw_diff"], float(np.max(np.abs(raws[0] - raws[1]))))
        res["tuned_over_default"] = res["tuned_ms"] / res["default_ms"]
        return res

    from paper_2106_12655_gb300 import workloads as W

    scenes = S.make_scenes(seed=5, n_scenes=6)       # the serving block's piles
    piles = [sc.geometry for sc in scenes]
    S.close(scenes)
    return {"knit_yarn": compare([W.knit_yarn()]), "serving_piles": compare(piles)}


def cpu_baseline(g):
    """The FP64 oracle on the sheet: every pair on all host cores (one pass),
    and a seeded 1/16 sample of the pairs on one core."""
    from oracle import oracle as O

    threads = O.default_threads()
    t0 = time.perf_counter()
    raw = O.link_pairs(g.vertices, g.offsets, g.pairs, threads=threads)
    dt = time.perf_counter() - t0
    pick = np.sort(np.random.default_rng(13).choice(g.pairs.shape[0], g.pairs.shape[0] // 16, replace=False))
    t0 = time.perf_counter()
    O.link_pairs(g.vertices, g.offsets, g.pairs[pick], threads=1)
    dt1 = time.perf_counter() - t0
    return raw, {"value": g.segment_pairs() / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                 "sample": "all %d candidate pairs of the sheet, one pass (%.1f s)" % (g.pairs.shape[0], dt),
                 "cpu": cpu_model(), "one_core": {"value": g.segment_pairs(g.pairs[pick]) / dt1, "unit": UNIT,
                                                   "cores": 1, "sample": "%d seeded pairs (1/16 of the sheet), %.1f s"
                                                   % (pick.size, dt1)}}


def workload_config(g, desc):
    return {"workload": desc, "pairs": int(g.pairs.shape[0]), "segment_pairs_per_step": int(g.segment_pairs())}


def run_reference(args):
    """The oracle on the headline workload: each step verifies the whole sheet
    on all host cores when the run fits in about two minutes (the driver's
    --steps/--warmup do), else a seeded sample of the pairs sized to fit."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from oracle import oracle as O

    g, desc = workload(0)
    threads = O.default_threads()
    n = g.pairs.shape[0]
    # one untimed probe of the oracle's rate sizes the per-step sample
    probe = np.random.default_rng(1).choice(n, max(1, n // 64), replace=False)
    t0 = time.perf_counter()
    O.link_pairs(g.vertices, g.offsets, g.pairs[probe], threads=threads)
    full_s = (time.perf_counter() - t0) * n / probe.size
    frac = min(1.0, 120.0 / max(full_s * (args.steps + args.warmup), 1e-9))
    per_step = n if frac >= 1.0 else max(1, int(n * frac))
    rng = np.random.default_rng(0)
    times, sps = [], []
    for s in range(args.warmup + args.steps):
        sub = g.pairs if per_step == n else g.pairs[rng.choice(n, per_step, replace=False)]
        t0 = time.perf_counter()
        O.link_pairs(g.vertices, g.offsets, sub, threads=threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            sps.append(g.segment_pairs(sub))
    value = sum(sps) / sum(times)
    sample = ("all %d candidate pairs of the sheet per step" % n if per_step == n else
              "%d seeded random candidate pairs per step (of %d)" % (per_step, n))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(g, desc),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    from paper_2106_12655_gb300 import build as B
    from paper_2106_12655_gb300 import lk

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    lk.load()
    g, desc = workload(rank)
    n = g.pairs.shape[0]
    sps_per_step = g.segment_pairs()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    v = torch.from_numpy(g.vertices).to(dev)
    off = torch.from_numpy(g.offsets).to(dev)
    pairs_d = torch.from_numpy(g.pairs).to(dev)
    lk_o = torch.zeros(n, dtype=torch.int32, device=dev)
    raw_o = torch.zeros(n, dtype=torch.float64, device=dev)
    st_o = torch.zeros(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # the roofline's denominator, from the unit counts and the maximum clock;
    # beside it the FMA rate measured on this GPU now, with its clocks
    fp32_peak = n_sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    peak_clk = ClockSampler(local)
    peak_clk.start()
    measured = [lk.lk_measure_fp32_peak(stream) for _ in range(3)]
    peak_clocks = peak_clk.stop()
    fp32_measured, peak_ms = max(measured)

    # The autotuner's table against the built-in split; the timed run uses the faster.
    tuning, table = ({}, None) if args.headline_only else tuning_block(g, v, off, pairs_d, stream, flush)

    opt = lk.lk_default_options()
    opt.timing = 1
    ctx = lk.lk_create(v, off, opt, stream)
    if table is not None:
        lk.lk_tune_set(ctx, table)
    plan = lk.lk_plan_create(ctx, pairs_d, stream)

    def step_timed():
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lk.lk_plan_run(plan, lk_o, raw_o, st_o, stream, ctx=ctx)
        e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        step_timed()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    step_ms, sweep_ms = [], []
    w0 = time.perf_counter()
    for _ in range(args.steps):
        e0, e1 = step_timed()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        sweep_ms.append(lk.lk_get_stats(ctx)["sweep_ms"])
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    stats = lk.lk_get_stats(ctx)
    total_ms = sum(step_ms)
    if dist:
        from paper_2106_12655_gb300 import multigpu as MG

        total_ms = MG.max_over_ranks(total_ms, dist, dev)
    value = world * sps_per_step * args.steps / (total_ms / 1e3)
    lk_host = lk_o.cpu().numpy()
    raw_host = raw_o.cpu().numpy()
    st_host = st_o.cpu().numpy()
    est_host = np.zeros(n)
    lk.lk_get_error_estimates(ctx, est_host)
    if args.headline_only:
        lk.lk_plan_destroy(plan)
        lk.lk_destroy(ctx)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                              "headline_only": True}), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    # All-FP64 direct sum on the same GPU and workload (the baseline to beat).
    opt64 = lk.lk_default_options()
    opt64.precision = lk.LK_ALL_F64
    opt64.timing = 1
    ctx64 = lk.lk_create(v, off, opt64, stream)
    plan64 = lk.lk_plan_create(ctx64, pairs_d, stream)
    lk64 = torch.zeros_like(lk_o)
    raw64 = torch.zeros_like(raw_o)
    st64 = torch.zeros_like(st_o)
    lk.lk_plan_run(plan64, lk64, raw64, st64, stream, ctx=ctx64)
    f64_ms = []
    for _ in range(args.fp64_steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lk.lk_plan_run(plan64, lk64, raw64, st64, stream, ctx=ctx64)
        e1.record(stream)
        e1.synchronize()
        f64_ms.append(e0.elapsed_time(e1))
    fp64_value = sps_per_step / (statistics.median(f64_ms) / 1e3)
    raw64_host = raw64.cpu().numpy()
    lk.lk_plan_destroy(plan64)
    lk.lk_destroy(ctx64)

    # End to end through the public C-ABI call with host buffers: each step
    # uploads a displacement of every vertex from pinned host memory, passes
    # the (unchanged) pair list from pinned host memory, verifies, and reads
    # the results back to host memory.  lk_verify compares the list with the
    # previous call's on the host and replays that list's graph plan, so the
    # list itself is not copied to the device.
    rng = np.random.default_rng(11)
    delta = torch.from_numpy(rng.normal(scale=1e-6, size=g.vertices.shape).astype(np.float32)).pin_memory()
    neg = (-delta).pin_memory()
    pairs_h = torch.from_numpy(g.pairs).pin_memory()
    lk_h = torch.zeros(n, dtype=torch.int32).pin_memory()
    raw_h = torch.zeros(n, dtype=torch.float64).pin_memory()
    st_h = torch.zeros(n, dtype=torch.int32).pin_memory()
    e2e_ms = []
    for s in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lk.lk_update(ctx, delta if s % 2 == 0 else neg, True, stream)
        lk.lk_verify(ctx, pairs_h, lk_h, raw_h, st_h, stream)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            e2e_ms.append(dt * 1e3)
    e2e_value = world * sps_per_step * len(e2e_ms) / (sum(e2e_ms) / 1e3)
    h2d = delta.numel() * delta.element_size()
    d2h = n * (4 + 8 + 4) + 80      # the results, and the verify's ten work counters (list sizing)
    e2e_ok = bool(np.all(st_h.numpy() == 0) and np.array_equal(lk_h.numpy(), lk_host))
    lk.lk_plan_destroy(plan)
    lk.lk_destroy(ctx)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    sweep_avg = statistics.mean(sweep_ms)
    achieved = sps_per_step * FLOPS_PER_SP / (sweep_avg / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "precision": "FP32 segment-pair terms, FP64 accumulation, FP64 recompute of near pairs",
        "data": "synthetic",
        "config": workload_config(g, desc),
        "timing": {"l2": "flushed before every timed step (256 MB write)", "step": "one CUDA-graph replay",
                   "work_split": "autotuned" if table is not None else "built-in"},
        "p50_verify_ms": float(np.percentile(step_ms, 50)), "p99_verify_ms": float(np.percentile(step_ms, 99)),
        "fp64_recomputed_segment_pairs": stats["fp64_pairs"], "careful_items": stats["careful_items"],
        "careful_chunks": stats["careful_chunks"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": SWEEP_TRAFFIC_BYTES,
                     "traffic_unit": "bytes per launch", "kernel": "sweep_packed_kernel<fast>",
                     "kernel_ms": sweep_avg, "flops_per_segment_pair": FLOPS_PER_SP,
                     "peak_source": "derived: %d SMs x %d FP32 lanes x 2 x %.0f MHz" % (
                         n_sms, FP32_LANES_PER_SM, SM_MAX_MHZ),
                     "peak_measured": fp32_measured, "frac_of_measured": achieved / fp32_measured,
                     "peak_measured_source": "independent FMAs on every SM, packed and scalar, the faster "
                                             "(lk_measure_fp32_peak, %.1f ms launch, burst)" % peak_ms,
                     "peak_measured_clocks": peak_clocks},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": statistics.mean(e2e_ms), "results_match_device_run": e2e_ok},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "clocks": clk, "wall_s_timed_region": wall, "tuning": tuning,
        "fp64_baseline": {"value": fp64_value, "unit": UNIT, "ms_per_step": statistics.median(f64_ms),
                          "speedup_mixed_over_fp64": value / world / fp64_value,
                          "max_abs_raw_diff_vs_mixed": float(np.max(np.abs(raw64_host - raw_host)))},
    }
    if world == 1:
        line["one_call_per_pair"] = per_pair_block(g, v, off, lk_host, stream)
        line["early_exit"] = early_exit_block(g, v, off, lk_host, stream)
        line["counting_crossings"] = counting_crossings_block(g, v, off, pairs_d, lk_host, stream, flush)
        line["counting_crossings_all_pairs_sweep"] = counting_crossings_block(
            g, v, off, pairs_d, lk_host, stream, flush, search=lk.LK_CC_SEARCH_SWEEP)
    if not args.no_serving and world == 1:
        line["serving"] = serving_block(args)
        line["serving_geometry"] = geometry_serving_block(args)
    if not args.no_stress and world == 1:
        line["stress"] = stress_block(stream)
        line["configs"] = configs_block(stream)
        line["tuning_other"] = tuning_other_block(stream)
    if not args.no_cpu_baseline and world == 1:
        ref_raw, cb = cpu_baseline(g)
        line["cpu_baseline"] = cb
        ref_lk = np.sign(ref_raw) * np.floor(np.abs(ref_raw) + 0.5)
        line["parity_vs_oracle"] = {"lk_bit_exact": bool(np.array_equal(lk_host, ref_lk.astype(np.int32))),
                                    "raw_err_vs_oracle": err_stats(raw_host, ref_raw),
                                    "max_error_estimate": float(np.max(est_host)),
                                    "all_status_ok": bool(np.all(st_host == 0))}
    line["summary"] = summary(line)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _g(x, digits=3):
    """A number rounded to `digits` significant digits (compact JSON)."""
    if x is None or not isinstance(x, (int, float)) or x == 0 or not np.isfinite(x):
        return x
    return float("%.*g" % (digits, x))


def summary(line):
    """The numbers the tail of the line must hold: the FP64 baseline, serving,
    every configuration's rate and its worst raw error against the oracle or
    the closed form."""
    out = {"fp64_gpu": {"sp_s": _g(line["fp64_baseline"]["value"]),
                        "mixed_speedup": _g(line["fp64_baseline"]["speedup_mixed_over_fp64"])},
           "early_exit_ms": ({"full": _g(line["early_exit"]["full"]["ms"]),
                              "changed_at_100": _g(line["early_exit"]["changed_at_100"]["ms"])}
                             if "early_exit" in line else None),
           "roofline_frac": _g(line["roofline"]["frac"]), "e2e_sp_s": _g(line["e2e"]["value"])}
    err, rate = {}, {}
    if "parity_vs_oracle" in line:
        err["chainmail"] = _g(line["parity_vs_oracle"]["raw_err_vs_oracle"]["max"])
    if "serving" in line:
        sv = line["serving"]
        out["serving"] = {"cap_req_s": _g(sv["capacity"]["req_per_s"]), "cap_sp_s": _g(sv["capacity"]["sp_per_s"]),
                          "batched_sp_s": _g(sv["batched_same_piles"]["sp_per_s"]),
                          "pls_100k_ms": _g(sv["potential_link_search_large"]["ms"]),
                          "n_req": sv["loads"][0]["n_requests"],
                          "p50_ms": [_g(x["p50_ms"]) for x in sv["loads"]],
                          "p99_ms": [_g(x["p99_ms"]) for x in sv["loads"]],
                          "variants_cap_p50_p99_80": {k: [_g(sv[k]["capacity_req_per_s"]), _g(sv[k]["p50_ms"]),
                                                          _g(sv[k]["p99_ms"])]
                                                      for k in ("host_packing", "fewest_items_first")}}
    if "serving_geometry" in line:
        sg = line["serving_geometry"]
        out["serving_geometry"] = {m: {"cap_req_s": _g(sg[m]["capacity"]["req_per_s"]),
                                       "p50_ms": [_g(x["p50_ms"]) for x in sg[m]["loads"]],
                                       "p99_ms": [_g(x["p99_ms"]) for x in sg[m]["loads"]]}
                                   for m in ("geometry", "host_search")}
    if "tuning_other" in line:
        out["tuned_over_default"] = {k: _g(v["tuned_over_default"]) for k, v in line["tuning_other"].items()}
        out["tuned_over_default"]["sheet"] = _g(line["tuning"]["tuned_ms"] / line["tuning"]["default_ms"]) \
            if "tuned_ms" in line.get("tuning", {}) else None
    if "configs" in line:
        c = line["configs"]
        err["ring_chain"] = _g(c["ring_chain"]["raw_err_vs_oracle"]["max"])
        err["knit_sample"] = _g(c["knit_yarn"]["raw_err_vs_oracle"]["max"])
        rate["ring_chain"] = _g(c["ring_chain"]["value"])
        rate["knit"] = _g(c["knit_yarn"]["value"])
        rate["knit_fp64"] = _g(c["knit_yarn"]["fp64_gpu"]["value"])
        for t in c["torus_links"]["links"]:
            key = "torus%d_%d_%dk" % (t["p"], t["q"], t["segments_per_component"] // 1000)
            err[key] = _g(t["abs_raw_err_vs_closed_form"])
            rate[key] = _g(t["value"])
        rate["torus_fp64"] = _g(c["torus_links"]["fp64_gpu_rate"]["value"])
    if "stress" in line:
        for k, rec in line["stress"].items():
            err[k] = _g(rec["direct_sum"]["max_abs_raw_err"])
            rate[k] = _g(rec["direct_sum"]["value"])
    if "cpu_baseline" in line:
        out["oracle_sp_s"] = {"cores": line["cpu_baseline"]["cores"], "all": _g(line["cpu_baseline"]["value"]),
                              "one": _g(line["cpu_baseline"]["one_core"]["value"])}
    out["sp_s"] = rate
    out["max_raw_err"] = err
    return out


def run_precise_only(args):
    """One pair that the bulk sweep's error estimate sends to the precise
    variant, verified twice (CUDA-event time of the second)."""
    import torch
    from paper_2106_12655_gb300 import build as B
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import workloads as W

    B.build()
    lk.load()
    g = W.woundball(1000, 100_000)
    g.vertices = g.vertices.astype(np.float32)
    stream = torch.cuda.current_stream()
    v = torch.from_numpy(g.vertices).cuda()
    off = torch.from_numpy(g.offsets).cuda()
    ctx = lk.lk_create(v, off, None, stream)
    try:
        pd = torch.from_numpy(g.pairs).cuda()
        ms, lo, raw, st, est = timed_verify(ctx, pd, 1, stream, 1, 1, v.device)
        stats = lk.lk_get_stats(ctx)
    finally:
        lk.lk_destroy(ctx)
    print(json.dumps({"workload": "woundball nu=1000, 2 x 100,000 segments", "segment_pairs": g.segment_pairs(),
                      "ms": ms[0], "raw": float(raw[0]), "lk": int(lo[0]), "status": int(st[0]),
                      "error_estimate": float(est[0]), "precise_pairs": stats["precise_pairs"]}), flush=True)


def run_accurate_only(args):
    """One pair that takes the bulk sweep's accurate variant (10^10 segment
    pairs) verified three times (CUDA-event time of the last)."""
    import torch
    from paper_2106_12655_gb300 import build as B
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import workloads as W

    B.build()
    lk.load()
    g = W.torus_link(5, 7, 100_000, dtype=np.float32)
    stream = torch.cuda.current_stream()
    v = torch.from_numpy(g.vertices).cuda()
    off = torch.from_numpy(g.offsets).cuda()
    ctx = lk.lk_create(v, off, None, stream)
    try:
        pd = torch.from_numpy(g.pairs).pin_memory()
        ms, lo, raw, st, est = timed_verify(ctx, pd, 1, stream, 2, 1, v.device)
        stats = lk.lk_get_stats(ctx)
    finally:
        lk.lk_destroy(ctx)
    print(json.dumps({"workload": "torus link (5,7), 2 x 100,000 segments", "segment_pairs": g.segment_pairs(),
                      "ms": ms[0], "raw": float(raw[0]), "lk": int(lo[0]), "status": int(st[0]),
                      "error_estimate": float(est[0]), "precise_pairs": stats["precise_pairs"]}), flush=True)


def run_serving_only(args):
    """Closed-loop serving capacity on the six resident piles, alone."""
    from paper_2106_12655_gb300 import build as B
    from paper_2106_12655_gb300 import lk
    from paper_2106_12655_gb300 import serving as S

    B.build()
    lk.load()
    scenes = S.make_scenes(seed=5, n_scenes=6)
    srv = lk.lk_server_create(None)
    try:
        S.run(srv, scenes, S.request_plan(scenes, 40, seed=99), None, max_outstanding=32)
        plan = S.request_plan(scenes, args.serving_requests, seed=1)
        lat, wall, bad, _ = S.run(srv, scenes, plan, None, max_outstanding=32)
        pairs, sps = S.plan_sizes(scenes, plan)
        print(json.dumps({"workload": "serving capacity, six chainmail piles, closed loop of 32",
                          "n_requests": len(plan), "req_per_s": len(plan) / wall, "sp_per_s": float(sps.sum()) / wall,
                          "nonok_pair_status": bad, "server_stats": lk.lk_server_get_stats(srv)}), flush=True)
    finally:
        lk.lk_server_destroy(srv)
        S.close(scenes)


def main():
    args = parse()
    if args.precise_only:
        run_precise_only(args)
        return
    if args.serving_only:
        run_serving_only(args)
        return
    if args.accurate_only:
        run_accurate_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
