"""Multi-GPU sharding of a verify (host logic; one process per GPU).

Loop pairs are independent, so a verify shards by pairs with no exchange on
the data path: every rank holds the geometry (tens of MB at most), verifies
its own share of the pairs, and the per-pair results are gathered once at the
end.  Shares are balanced by longest-processing-time assignment on the cost
N_rows * N_cols of each pair.  Collectives go through torch.distributed, so
the same code runs over NCCL on GPUs and over gloo on CPU (where the tests
exercise it).
"""
from __future__ import annotations

import heapq

import numpy as np


def pair_costs(loop_sizes, pairs) -> np.ndarray:
    n = np.asarray(loop_sizes, np.int64)
    pr = np.asarray(pairs, np.int64).reshape(-1, 2)
    ok = (pr >= 0).all(1) & (pr < n.shape[0]).all(1) & (pr[:, 0] != pr[:, 1])
    cost = np.zeros(pr.shape[0], np.int64)
    cost[ok] = n[pr[ok, 0]] * n[pr[ok, 1]]
    return cost


def partition_pairs(loop_sizes, pairs, world: int):
    """Indices of the pairs each of `world` ranks verifies (LPT on cost).
    Deterministic: ties are broken by pair index and rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = pair_costs(loop_sizes, pairs)
    order = np.lexsort((np.arange(cost.shape[0]), -cost))
    heap = [(0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for idx in order:
        load, r = heapq.heappop(heap)
        shares[r].append(int(idx))
        heapq.heappush(heap, (load + int(cost[idx]), r))
    return [np.asarray(sorted(s), np.int64) for s in shares]


def gather_results(share, lk, raw, status, n_pairs: int, dist):
    """Assemble the full per-pair results on every rank from each rank's share
    (pair indices and its results) with one all_gather."""
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, (np.asarray(share), np.asarray(lk), np.asarray(raw), np.asarray(status)))
    out_lk = np.zeros(n_pairs, np.int32)
    out_raw = np.full(n_pairs, np.nan)
    out_st = np.full(n_pairs, -1, np.int32)
    for idx, a, b, c in parts:
        out_lk[idx] = a
        out_raw[idx] = b
        out_st[idx] = c
    return out_lk, out_raw, out_st


def max_over_ranks(value: float, dist, device=None) -> float:
    """The largest value over all ranks (the timing rule for a multi-GPU step)."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
