"""Open-loop serving driver over the library's continuous-batching server.

Requests arrive as a Poisson process; each asks to verify a window of
1k-20k candidate pairs of one of several resident chainmail piles (the
per-frame verification of a running simulation).  Between requests a pile
receives a small displacement (lk_update) when none of its requests is in
flight.  Latency is measured from a request's scheduled arrival to the moment
lk_server_poll hands its results to the host.  All linking-number work runs in
the library; this module only schedules submissions and reads clocks.

Requests can also carry geometry only (mode "geometry"): verify every
potential link of the pile's current geometry, the search and packing done on
the device by lk_server_submit_geometry.  Mode "host_search" serves the same
requests through a host round trip instead: lk_candidates on the server's
stream (after the pile's update), then lk_server_submit of the list.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import lk
from . import workloads as W


@dataclass
class Scene:
    geometry: W.Geometry
    ctx: int
    delta_pos: object      # device tensors
    delta_neg: object
    flip: bool = False
    in_flight: int = 0


def make_scenes(seed=5, n_scenes=6, min_rings=500, max_rings=14000, sigma=1e-3, stream=None):
    """Resident chainmail piles with log-uniform ring counts and 64-256 segments per ring.
    The per-step displacements live in device memory, as a simulation's would."""
    import torch

    rng = np.random.default_rng(seed)
    scenes = []
    for k in range(n_scenes):
        g = W.serving_pile(int(rng.integers(1 << 30)), min_rings, max_rings)
        ctx = lk.lk_create(g.vertices, g.offsets, None, stream)
        d = rng.normal(scale=sigma, size=g.vertices.shape).astype(g.vertices.dtype)
        scenes.append(Scene(g, ctx, torch.from_numpy(d).cuda(), torch.from_numpy(np.ascontiguousarray(-d)).cuda()))
    return scenes


def request_plan(scenes, n_requests, seed=0, min_pairs=1000, max_pairs=20000):
    """(scene index, pair window) for each request; window sizes log-uniform."""
    rng = np.random.default_rng(seed)
    plan = []
    for _ in range(n_requests):
        k = int(rng.integers(len(scenes)))
        pairs = scenes[k].geometry.pairs
        want = int(np.exp(rng.uniform(np.log(min_pairs), np.log(max_pairs))))
        m = min(want, pairs.shape[0])
        lo = int(rng.integers(0, pairs.shape[0] - m + 1))
        plan.append((k, np.ascontiguousarray(pairs[lo:lo + m])))
    return plan


def geometry_plan(scenes, n_requests, seed=0):
    """Whole-pile requests: (scene index, None) for each request."""
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(len(scenes))), None) for _ in range(n_requests)]


def run(srv, scenes, plan, rate_per_s=None, seed=1, update=True, timeout_s=600.0, max_outstanding=None,
        mode="pairs", record=None):
    """Serve `plan`; arrivals are Poisson at rate_per_s (None: all at t = 0).
    With max_outstanding, a request is submitted only while fewer than that
    many are queued or running (a closed loop: with rate_per_s None this
    measures the sustained capacity, the host packing of later requests
    overlapping the device work of earlier ones).  mode: "pairs" (each plan
    entry carries its pair list), "geometry" or "host_search" (whole-pile
    requests, see the module's head).  Returns per-request latencies (s), the
    wall time, the number of pair results whose status was not LK_OK, and the
    number of pairs verified.  With `record` (a dict), it also receives per
    request the requests outstanding when it was submitted ("depth") and the
    delay between its scheduled arrival and its submission ("late", s)."""
    rng = np.random.default_rng(seed)
    n = len(plan)
    if rate_per_s is None:
        arrivals = np.zeros(n)
    else:
        arrivals = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    stream = lk.lk_server_stream(srv)
    cap = max(p.shape[0] for _, p in plan) if mode == "pairs" else 0
    if mode != "pairs":
        cap = max(sc.geometry.pairs.shape[0] for sc in scenes) * 2 + 1024
    status = np.zeros(cap, np.int32)
    pairs_buf = np.zeros((cap, 2), np.int32)
    bad = 0
    verified = 0
    pending = {}          # ticket -> (request index, scene index)
    lat = np.zeros(n)
    depth = np.zeros(n, np.int64)
    late = np.zeros(n)
    nxt = 0
    done = 0
    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        if now > timeout_s:
            raise TimeoutError("serving run exceeded %.0f s" % timeout_s)
        while nxt < n and arrivals[nxt] <= now and (max_outstanding is None or len(pending) < max_outstanding):
            k, pairs = plan[nxt]
            sc = scenes[k]
            if update and sc.in_flight == 0:
                lk.lk_update(sc.ctx, sc.delta_neg if sc.flip else sc.delta_pos, True, stream)
                sc.flip = not sc.flip
            if mode == "geometry":
                t = lk.lk_server_submit_geometry(srv, sc.ctx)
            elif mode == "host_search":
                m = lk.lk_candidates(sc.ctx, pairs_buf, stream)
                t = lk.lk_server_submit(srv, sc.ctx, pairs_buf[:min(m, cap)])
            else:
                t = lk.lk_server_submit(srv, sc.ctx, pairs)
            sc.in_flight += 1
            depth[nxt] = len(pending)
            late[nxt] = (time.perf_counter() - t0) - arrivals[nxt]
            pending[t] = (nxt, k)
            nxt += 1
            # launch work as soon as it is admitted, not after a burst of submits
            lk.lk_server_step(srv, wait=False)
        lk.lk_server_step(srv, wait=False)
        for t in lk.lk_server_completed(srv):
            got, m = lk.lk_server_poll_pairs(srv, t, None, None, None, status, capacity=cap)
            if got:
                if m > cap:
                    raise RuntimeError("a request returned more pairs than the driver's buffer")
                i, k = pending.pop(t)
                bad += int(np.count_nonzero(status[:m]))
                verified += m
                lat[i] = (time.perf_counter() - t0) - arrivals[i]
                scenes[k].in_flight -= 1
                done += 1
        if not pending and nxt < n and arrivals[nxt] > time.perf_counter() - t0:
            wait = arrivals[nxt] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.001))
    wall = time.perf_counter() - t0
    if record is not None:
        record["depth"] = depth
        record["late"] = late
    return lat, wall, bad, verified


def plan_sizes(scenes, plan):
    pairs = np.array([p.shape[0] for _, p in plan], dtype=np.int64)
    sps = np.array([scenes[k].geometry.segment_pairs(p) for k, p in plan], dtype=np.int64)
    return pairs, sps


def close(scenes):
    for sc in scenes:
        lk.lk_destroy(sc.ctx)
