"""GPU potential link search (lk_candidates, Sec. 3.2 Algorithm 2) against the
oracle's all-pairs box-overlap definition: the pair lists must be identical
(exact FP64 box comparisons, sorted by (i, j))."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_12655_gb300 import lk
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


def context(g):
    stream = torch.cuda.current_stream()
    v = torch.from_numpy(np.ascontiguousarray(g.vertices)).cuda()
    off = torch.from_numpy(g.offsets).cuda()
    return lk.lk_create(v, off, None, stream), stream


def gpu_candidates(g):
    ctx, stream = context(g)
    try:
        return lk.lk_candidates(ctx, stream=stream)
    finally:
        lk.lk_destroy(ctx)


def grid_triangles(n, seed, spread=8):
    """Non-degenerate triangles with boxes on a coarse grid (many exact ties)."""
    rng = np.random.default_rng(seed)
    loops = []
    for _ in range(n):
        lo = rng.integers(0, spread, size=3).astype(float) / 4.0
        hi = lo + rng.integers(1, 4, size=3).astype(float) / 4.0
        loops.append(np.array([lo, [hi[0], lo[1], hi[2]], hi]))
    return W.from_loops(loops, dtype=np.float64)


@pytest.mark.parametrize("name", ["ring_chain", "chainmail", "knit_yarn", "triangles", "serving_pile"])
def test_candidates_match_oracle(name):
    g = {"ring_chain": lambda: W.ring_chain(),
         "chainmail": lambda: W.chainmail(),
         "knit_yarn": lambda: W.knit_yarn(),
         "triangles": lambda: grid_triangles(700, 1),
         "serving_pile": lambda: W.serving_pile(12345, 14000, 14000)}[name]()
    got = gpu_candidates(g)
    ref = O.candidates(g.vertices, g.offsets)
    assert got.shape == ref.shape and np.array_equal(got, ref), (got.shape, ref.shape)
    assert ref.shape[0] > 0


def test_tile_boundaries_and_sizes():
    # loop counts around the 8-row block and 256-box tile sizes
    for n in (2, 3, 7, 8, 9, 255, 256, 257, 263, 520):
        g = grid_triangles(n, n, spread=3 + n // 40)
        assert np.array_equal(gpu_candidates(g), O.candidates(g.vertices, g.offsets)), n


def test_capacity_host_and_device_outputs():
    g = grid_triangles(300, 2)
    ref = O.candidates(g.vertices, g.offsets)
    ctx, stream = context(g)
    try:
        n = ref.shape[0]
        assert lk.lk_candidates(ctx, np.zeros((0, 2), np.int32), stream=stream) == n
        half = np.full((n // 2, 2), -7, np.int32)
        assert lk.lk_candidates(ctx, half, stream=stream) == n
        assert np.array_equal(half, ref[: n // 2])
        dev = torch.full((n + 5, 2), -7, dtype=torch.int32, device="cuda")
        assert lk.lk_candidates(ctx, dev, stream=stream) == n
        d = dev.cpu().numpy()
        assert np.array_equal(d[:n], ref) and np.all(d[n:] == -7)
    finally:
        lk.lk_destroy(ctx)


def test_single_loop_and_after_update():
    g1 = grid_triangles(1, 3)
    assert gpu_candidates(g1).shape == (0, 2)
    g = W.chainmail(rows=4, cols=6, dtype=np.float64)
    ctx, stream = context(g)
    try:
        before = lk.lk_candidates(ctx, stream=stream)
        # move loop 5 far away: it loses every candidate
        delta = np.zeros_like(g.vertices)
        delta[g.offsets[5]:g.offsets[6]] = 100.0
        lk.lk_update(ctx, torch.from_numpy(delta).cuda(), True, stream)
        after = lk.lk_candidates(ctx, stream=stream)
    finally:
        lk.lk_destroy(ctx)
    moved = W.Geometry(g.vertices + delta, g.offsets, g.pairs)
    assert np.array_equal(before, O.candidates(g.vertices, g.offsets))
    assert np.array_equal(after, O.candidates(moved.vertices, moved.offsets))
    assert np.any(before == 5) and not np.any(after == 5)


def test_candidates_feed_verify_and_contain_every_linked_pair():
    g = W.chainmail(rows=4, cols=5, nseg=64, dtype=np.float64)
    all_pairs = np.array(list(itertools.combinations(range(g.n_loops), 2)), np.int32)
    raw_all = O.link_pairs(g.vertices, g.offsets, all_pairs)
    linked = {tuple(p) for p, r in zip(all_pairs.tolist(), raw_all) if abs(round(r)) > 0}
    ctx, stream = context(g)
    try:
        cand = torch.zeros((all_pairs.shape[0], 2), dtype=torch.int32, device="cuda")
        n = lk.lk_candidates(ctx, cand, stream=stream)
        cand = cand[:n].contiguous()
        lo = torch.zeros(n, dtype=torch.int32, device="cuda")
        raw = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = torch.zeros(n, dtype=torch.int32, device="cuda")
        lk.lk_verify(ctx, cand, lo, raw, st, stream)
        lk.lk_sync(ctx, stream)
    finally:
        lk.lk_destroy(ctx)
    c = cand.cpu().numpy()
    assert linked <= {tuple(p) for p in c.tolist()}
    assert np.all(st.cpu().numpy() == 0)
    ref = O.link_pairs(g.vertices, g.offsets, c)
    assert np.array_equal(lo.cpu().numpy(), O.round_lk(ref).astype(np.int32))
    assert np.abs(raw.cpu().numpy() - ref).max() <= 1e-6


def test_sort_and_sweep_on_100k_loops():
    """100,000 small triangles scattered so that each box overlaps about ten
    others: the sort and sweep on x finds exactly the oracle's all-pairs set
    (5e9 box tests on the host)."""
    import time

    g = grid_triangles(100_000, 5, spread=104)
    ctx, stream = context(g)
    try:
        lk.lk_candidates(ctx, stream=stream)                  # first call allocates
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = lk.lk_candidates(ctx, stream=stream)
        dt = time.perf_counter() - t0
    finally:
        lk.lk_destroy(ctx)
    ref = O.candidates(g.vertices, g.offsets)
    print(f"100k loops: {got.shape[0]} candidate pairs in {1e3 * dt:.2f} ms")
    assert got.shape == ref.shape and np.array_equal(got, ref)
    assert 100_000 < ref.shape[0] < 10_000_000


def test_sort_and_sweep_with_exact_ties():
    """20,000 triangles whose boxes sit on a coarse grid (many equal bounds,
    boxes touching on faces, edges and corners): past 2^27 box pairs the
    search sorts and sweeps, and must still equal the oracle exactly."""
    g = grid_triangles(20_000, 3, spread=40)
    assert 20_000 * 19_999 // 2 > (1 << 27)
    got = gpu_candidates(g)
    ref = O.candidates(g.vertices, g.offsets)
    assert got.shape == ref.shape and np.array_equal(got, ref)
