"""The multi-rank path on CPU: world_size-2 gloo process groups.

Each rank verifies its LPT share of the pairs (here with the FP64 oracle, the
stand-in for one GPU's verify), the shares are gathered with one collective,
and the assembled result must equal the single-rank result.  The timing rule
(maximum over ranks) is checked the same way.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2106_12655_gb300 import multigpu as MG
from paper_2106_12655_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = W.chainmail(seed=21, rows=6, cols=10, nseg=64)
        shares = MG.partition_pairs(g.sizes(), g.pairs, world)
        mine = shares[rank]
        raw = O.link_pairs(g.vertices, g.offsets, g.pairs[mine], threads=2)
        lk = O.round_lk(raw).astype(np.int32)
        st = np.zeros(mine.shape[0], np.int32)
        out = MG.gather_results(mine, lk, raw, st, g.pairs.shape[0], dist)
        slowest = MG.max_over_ranks(10.0 * (rank + 1), dist)
        q.put((rank, out, slowest, [s.tolist() for s in shares]))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_reassemble_the_single_rank_result():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = W.chainmail(seed=21, rows=6, cols=10, nseg=64)
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs, threads=2)
    for rank, (lk, raw, st), slowest, shares in res:
        assert slowest == 20.0
        assert np.array_equal(raw, ref)                  # same fixed-order sums per pair
        assert np.array_equal(lk, O.round_lk(ref).astype(np.int32))
        assert np.all(st == 0)
        assert sorted(shares[0] + shares[1]) == list(range(g.pairs.shape[0]))


def test_lpt_partition_balances_uneven_pairs():
    rng = np.random.default_rng(0)
    sizes = rng.integers(64, 20000, size=300)
    pairs = np.array([[a, b] for a, b in rng.integers(0, 300, size=(2000, 2)) if a != b], np.int32)
    for world in (1, 2, 3, 8):
        shares = MG.partition_pairs(sizes, pairs, world)
        assert sorted(np.concatenate(shares).tolist()) == list(range(pairs.shape[0]))
        cost = MG.pair_costs(sizes, pairs)
        loads = np.array([cost[s].sum() for s in shares])
        assert loads.max() - loads.min() <= cost.max()       # the LPT bound
    again = MG.partition_pairs(sizes, pairs, 3)
    assert all(np.array_equal(a, b) for a, b in zip(again, MG.partition_pairs(sizes, pairs, 3)))
