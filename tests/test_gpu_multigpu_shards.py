"""The sharded verify with the GPU kernels: each rank's share of one pair list
(longest-processing-time partition) is verified by its own context of the full
geometry, as one process per GPU would, here one share after the other on one
GPU; the gather step reassembles the list.  The result must equal the
single-call verify bit for bit (a pair's result does not depend on what else
is in its batch) and the oracle on a sample within 1e-6."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_12655_gb300 import lk
from paper_2106_12655_gb300 import multigpu as MG
from paper_2106_12655_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12655_gb300 import build as B

    B.build()
    lk.load()


class _Gathered:
    """The all_gather of the shares' results, done in one process: every
    rank's contribution is known once all shares have run."""

    def __init__(self, parts):
        self.parts = parts

    def get_world_size(self):
        return len(self.parts)

    def all_gather_object(self, out, obj):
        for k, p in enumerate(self.parts):
            out[k] = p


def verify(ctx, pairs):
    n = pairs.shape[0]
    out = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
    lk.lk_verify(ctx, np.ascontiguousarray(pairs), *out)
    return out


@pytest.mark.parametrize("world", [2, 4])
def test_shards_reassemble_the_single_call_result(world):
    g = W.serving_pile(55, 600, 600)
    whole_ctx = lk.lk_create(g.vertices, g.offsets)
    try:
        ref = verify(whole_ctx, g.pairs)
    finally:
        lk.lk_destroy(whole_ctx)
    shares = MG.partition_pairs(g.sizes(), g.pairs, world)
    assert sorted(np.concatenate(shares).tolist()) == list(range(g.pairs.shape[0]))
    parts = []
    for mine in shares:
        ctx = lk.lk_create(g.vertices, g.offsets)          # each rank holds the whole geometry
        try:
            parts.append((mine,) + verify(ctx, g.pairs[mine]))
        finally:
            lk.lk_destroy(ctx)
    cost = MG.pair_costs(g.sizes(), g.pairs)
    loads = [int(cost[s].sum()) for s in shares]
    assert max(loads) - min(loads) <= int(cost.max())        # LPT balance bound
    out = MG.gather_results(None, None, None, None, g.pairs.shape[0], _Gathered(parts))
    for k in range(3):
        assert np.array_equal(out[k], ref[k])
    rng = np.random.default_rng(world)
    idx = np.sort(rng.choice(g.pairs.shape[0], size=150, replace=False))
    want = O.link_pairs(g.vertices, g.offsets, np.ascontiguousarray(g.pairs[idx]))
    assert np.max(np.abs(out[1][idx] - want)) <= 1e-6
    assert np.array_equal(out[0][idx], O.round_lk(want).astype(np.int32))
