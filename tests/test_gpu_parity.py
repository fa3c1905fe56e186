"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bar (per pair): the rounded linking number bit-exact, the raw sum within
1e-6 of the oracle's FP64 sum (the tolerance stated for this method) and
within int_tol = 0.1 of an integer, status LK_OK.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_12655_gb300 import lk
from paper_2106_12655_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RAW_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12655_gb300 import build as B

    B.build()
    lk.load()


def run(g, pairs=None, precision=lk.LK_MIXED, on_device=True, stats=False, **opts):
    pairs = g.pairs if pairs is None else np.asarray(pairs, np.int32).reshape(-1, 2)
    o = lk.lk_default_options()
    o.precision = precision
    for k, v in opts.items():
        setattr(o, k, v)
    stream = torch.cuda.current_stream()
    if on_device:
        v = torch.from_numpy(np.ascontiguousarray(g.vertices)).cuda()
        off = torch.from_numpy(g.offsets).cuda()
        pr = torch.from_numpy(np.ascontiguousarray(pairs)).cuda()
    else:
        v, off, pr = np.ascontiguousarray(g.vertices), g.offsets, np.ascontiguousarray(pairs)
    n = pairs.shape[0]
    ctx = lk.lk_create(v, off, o, stream)
    try:
        if on_device:
            lk_o = torch.zeros(n, dtype=torch.int32, device="cuda")
            raw = torch.zeros(n, dtype=torch.float64, device="cuda")
            st = torch.zeros(n, dtype=torch.int32, device="cuda")
            lk.lk_verify(ctx, pr, lk_o, raw, st, stream)
            lk.lk_sync(ctx, stream)
            res = lk_o.cpu().numpy(), raw.cpu().numpy(), st.cpu().numpy()
        else:
            lk_o, raw, st = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
            lk.lk_verify(ctx, pr, lk_o, raw, st, stream)
            res = lk_o, raw, st
        s = lk.lk_get_stats(ctx)
    finally:
        lk.lk_destroy(ctx)
    return res + (s,) if stats else res


def check_against_oracle(g, pairs=None, tol=RAW_TOL, **kw):
    pairs = g.pairs if pairs is None else np.asarray(pairs, np.int32).reshape(-1, 2)
    lk_o, raw, st = run(g, pairs, **kw)
    ref = O.link_pairs(g.vertices, g.offsets, pairs)
    ref_lk = O.round_lk(ref)
    assert np.all(st == lk.LK_OK), np.unique(st, return_counts=True)
    assert np.array_equal(lk_o, ref_lk.astype(np.int32)), np.nonzero(lk_o != ref_lk)
    err = np.abs(raw - ref)
    assert err.max() <= tol, (err.max(), int(err.argmax()))
    assert np.abs(raw - lk_o).max() <= 0.1
    return raw, ref


# ----------------------------------------------------------------------------- configs

def test_ring_chain_all_pairs():
    g = W.ring_chain()
    raw, ref = check_against_oracle(g)
    assert sorted(set(O.round_lk(ref).tolist())) == [-1, 0, 1]


def test_ring_chain_all_f64_baseline():
    check_against_oracle(W.ring_chain(), precision=lk.LK_ALL_F64, tol=1e-9)


def test_chainmail_sheet_full_size():
    """The benchmarked workload: 2,048 rings x 256 segments, all AABB candidates."""
    g = W.chainmail()
    raw, ref = check_against_oracle(g)
    counts = np.unique(O.round_lk(ref), return_counts=True)
    assert set(counts[0].tolist()) == {-1, 0, 1}


def test_chainmail_sheet_accurate_variant():
    check_against_oracle(W.chainmail(), accurate_threshold=0)


def test_chainmail_plan_graph_matches_oracle():
    g = W.chainmail()
    v = torch.from_numpy(g.vertices).cuda()
    off = torch.from_numpy(g.offsets).cuda()
    pr = torch.from_numpy(g.pairs).cuda()
    n = g.pairs.shape[0]
    stream = torch.cuda.current_stream()
    ctx = lk.lk_create(v, off, None, stream)
    plan = lk.lk_plan_create(ctx, pr, stream)
    try:
        outs = []
        for _ in range(2):
            lk_o = torch.zeros(n, dtype=torch.int32, device="cuda")
            raw = torch.zeros(n, dtype=torch.float64, device="cuda")
            st = torch.zeros(n, dtype=torch.int32, device="cuda")
            lk.lk_plan_run(plan, lk_o, raw, st, stream, ctx=ctx)
            torch.cuda.synchronize()
            outs.append((lk_o.cpu().numpy(), raw.cpu().numpy(), st.cpu().numpy()))
    finally:
        lk.lk_plan_destroy(plan)
        lk.lk_destroy(ctx)
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs)
    for lk_o, raw, st in outs:
        assert np.all(st == 0)
        assert np.array_equal(lk_o, O.round_lk(ref).astype(np.int32))
        assert np.abs(raw - ref).max() <= RAW_TOL
    assert np.array_equal(outs[0][1], outs[1][1])      # graph replays are bit-identical


def test_knit_yarn_sampled_pairs():
    """600 loops of 1k-20k segments: every pair on the GPU; a seeded 10% sample
    of the pairs together with the 20 largest (about 1.3e10 segment pairs)
    against the oracle element by element; every pair integral."""
    g = W.knit_yarn()
    lk_o, raw, st = run(g)
    assert np.all(st == 0)
    assert np.abs(raw - lk_o).max() < 1e-4
    sizes = g.sizes()[g.pairs].prod(axis=1)
    order = np.argsort(sizes)
    rng = np.random.default_rng(7)
    pick = np.unique(np.concatenate([order[-20:], rng.choice(len(order), len(order) // 10, replace=False)]))
    assert pick.size >= 330
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs[pick])
    assert np.array_equal(lk_o[pick], O.round_lk(ref).astype(np.int32))
    err = np.abs(raw[pick] - ref)
    assert err.max() <= RAW_TOL, (err.max(), g.pairs[pick][np.argmax(err)])
    assert set(np.unique(lk_o).tolist()) <= {-1, 0, 1}


@pytest.mark.parametrize("p,q,n", [(2, 3, 250_000), (31, 37, 1_000_000)])
def test_torus_link_closed_form_large(p, q, n):
    """Single huge pairs (intra-pair split): the exact sum is -p*q for this
    orientation; the raw sum must be within 1e-6 of it."""
    g = W.torus_link(p, q, n, dtype=np.float32)
    lk_o, raw, st = run(g)
    assert st[0] == 0
    assert abs(lk_o[0]) == p * q
    assert abs(raw[0] - lk_o[0]) <= RAW_TOL


@pytest.mark.parametrize("twists", [10, 1000])
def test_paper_stress_ribbon_closed_form(twists):
    """The double-helix ribbons of the paper's stress tests at the size of its
    Table 1 (two loops of 1e5 segments, lk = 10 and 10^3): the linking number
    exact and the raw sum within 1e-6 of it.  At 1000 twists the edges wind
    around each other so that the 1e10 terms turn through about 2e5 rad for a
    net 2000 pi; FP32 terms leave an error near 1e-6 there (the paper reports
    its own single-precision GPU sum on these ribbons as mostly under 1e-5,
    Sec. 4.1), so the bulk sweep's error estimate sends the pair to the
    compensated sweep."""
    g = W.double_helix_ribbon(twists, 100_000)
    lk_o, raw, st, stats = run(g, stats=True)
    assert st[0] == 0 and abs(lk_o[0]) == twists
    assert abs(raw[0] - lk_o[0]) <= RAW_TOL
    if twists == 1000:
        assert stats["precise_pairs"] == 1


def test_torus_link_small_matches_oracle_f32_and_f64_inputs():
    for dt in (np.float32, np.float64):
        g = W.torus_link(5, 7, 3000, dtype=dt, n2=2711)
        check_against_oracle(g)


# ----------------------------------------------------------------------------- tiles and edges

@pytest.mark.parametrize("n1,n2", [(3, 3), (3, 4), (4, 5), (5, 129), (127, 128), (128, 129),
                                   (129, 255), (256, 257), (300, 1000)])
def test_tile_edges_random_polygons(n1, n2):
    rng = np.random.default_rng(n1 * 1000 + n2)
    loops = []
    for n in (n1, n2):
        t = np.sort(rng.uniform(0, 2 * np.pi, n))
        r = 1.0 + 0.2 * rng.normal(size=(n, 1))
        c = rng.normal(scale=0.3, size=3)
        loops.append(c + r * np.stack([np.cos(t), np.sin(t), 0.3 * rng.normal(size=n)], 1))
    loops[1] = loops[1][:, [0, 2, 1]] + np.array([1.0, 0.0, 0.0])
    g = W.from_loops(loops, pairs=[[0, 1], [1, 0]])
    for tile_rows in (0, 32, 64, 96):
        for accurate_threshold in (0, 1 << 62):          # both FP32 arithmetic variants
            check_against_oracle(g, tile_rows=tile_rows, accurate_threshold=accurate_threshold)


def test_random_integer_polygons_against_exact_crossings():
    from crossings import linking_number_exact

    rng = np.random.default_rng(12)
    loops, pairs, expect = [], [], []
    while len(pairs) < 40:
        n1, n2 = rng.integers(4, 40, 2)
        l = rng.integers(-40, 41, (n1, 3))
        k = rng.integers(-40, 41, (n2, 3))
        try:
            cc = linking_number_exact(l, k, rng)
        except Exception:
            continue
        pairs.append([len(loops), len(loops) + 1])
        loops += [l.astype(np.float64), k.astype(np.float64)]
        expect.append(cc)
    g = W.from_loops(loops, pairs=pairs)
    lk_o, raw, st = run(g)
    assert np.all(st == 0), st
    assert np.array_equal(lk_o, np.asarray(expect, np.int32))
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs)
    assert np.abs(raw - ref).max() <= RAW_TOL


def test_near_segments_take_the_fp64_path():
    """Two loops with segments within a segment length of each other: the
    careful pass must send those pairs to FP64 and still match the oracle."""
    t = np.arange(400) * 2 * np.pi / 400
    a = np.stack([np.cos(t), np.sin(t), 0 * t], 1)
    # b threads a's disk and passes 0.004 outside a at (1.004, 0, 0); a's
    # segments are ~0.0157 long, b's ~0.0079
    b = np.stack([0.5 + 0.504 * np.cos(t + 0.01), 0 * t, 0.504 * np.sin(t + 0.01)], 1)
    g = W.from_loops([a, b], pairs=[[0, 1]])
    lk_o, raw, st, s = run(g, stats=True)
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs)
    assert st[0] == 0 and lk_o[0] == O.round_lk(ref)[0]
    assert abs(raw[0] - ref[0]) <= RAW_TOL
    assert s["fp64_pairs"] > 0
    assert s["careful_chunks"] > 0 and s["careful_items"] == 0
    # a one-entry chunk list hands whole items to the careful pass instead;
    # that pass sums every segment pair's arctangent, the bulk sweep sums its
    # chunks by angle summation, so the two agree to FP32 rounding of the sums
    lk3, raw3, st3, s3 = run(g, stats=True, chunk_capacity=1)
    assert s3["careful_items"] > 0
    assert st3[0] == 0 and lk3[0] == lk_o[0] and abs(raw3[0] - raw[0]) <= 1e-8
    assert abs(raw3[0] - ref[0]) <= RAW_TOL
    # a tiny list forces the in-place FP64 evaluation of the overflow
    lk2, raw2, st2, s2 = run(g, stats=True, near_capacity=3)
    assert s2["near_overflow"] > 0
    assert st2[0] == 0 and lk2[0] == lk_o[0] and abs(raw2[0] - ref[0]) <= RAW_TOL


@pytest.mark.parametrize("chunk_capacity", [1, 3, 8, 40, 1 << 20])
def test_chunk_list_overflow_part_way_through_an_item(chunk_capacity):
    """Square links put near segment pairs in two chunks of one work item (each
    rectangle passes within w = L/2 of both long sides of the other, which lie
    in the two halves of its 60 rows).  When the chunk list fills after some
    of an item's chunks went to it, the item is swept again whole; its near
    pairs must be counted once, in both paths."""
    g = W.square_links(12, 60)
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs)
    for near_capacity in (1 << 20, 7):
        lk_o, raw, st, s = run(g, stats=True, chunk_capacity=chunk_capacity, near_capacity=near_capacity)
        assert np.all(st == 0) and np.array_equal(lk_o, O.round_lk(ref).astype(np.int32))
        assert np.max(np.abs(raw - ref)) <= RAW_TOL, (near_capacity, np.max(np.abs(raw - ref)))
        assert s["careful_chunks"] > 0 and s["fp64_pairs"] > 0
        assert (s["careful_items"] > 0) == (chunk_capacity <= 40)


def test_overflowed_lists_grow_for_later_verifies():
    """A verify that overflowed the recompute and chunk lists leaves its need on
    the context; the next verify runs with lists that fit (and with a memory
    budget the sizes stay as configured).  Every call matches the oracle."""
    g = W.square_links(12, 60)
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs)
    stream = torch.cuda.current_stream()
    v = torch.from_numpy(g.vertices).cuda()
    off = torch.from_numpy(g.offsets).cuda()
    pr = torch.from_numpy(g.pairs).cuda()
    n = g.pairs.shape[0]
    for budget in (0, 1 << 40):
        o = lk.lk_default_options()
        o.near_capacity, o.chunk_capacity, o.mem_budget = 7, 1, budget
        ctx = lk.lk_create(v, off, o, stream)
        try:
            runs = []
            for _ in range(3):       # plain, grown plain, plan replay of the same list
                lk_o = torch.zeros(n, dtype=torch.int32, device="cuda")
                raw = torch.zeros(n, dtype=torch.float64, device="cuda")
                st = torch.zeros(n, dtype=torch.int32, device="cuda")
                lk.lk_verify(ctx, pr, lk_o, raw, st, stream)
                torch.cuda.synchronize()
                runs.append((lk_o.cpu().numpy(), raw.cpu().numpy(), st.cpu().numpy(), lk.lk_get_stats(ctx)))
            grown = lk.lk_get_options(ctx)
        finally:
            lk.lk_destroy(ctx)
        for lk_o, raw, st, _ in runs:
            assert np.all(st == 0) and np.array_equal(lk_o, O.round_lk(ref).astype(np.int32))
            assert np.max(np.abs(raw - ref)) <= RAW_TOL
        first = runs[0][3]
        assert first["near_overflow"] > 0 and first["careful_items"] > 0
        if budget:
            assert (grown.near_capacity, grown.chunk_capacity) == (7, 1)
            assert runs[2][3]["near_overflow"] > 0
        else:
            assert grown.near_capacity >= first["fp64_pairs"] and grown.chunk_capacity > 1
            for _, _, _, s in runs[1:]:
                assert s["near_overflow"] == 0 and s["careful_items"] == 0
            assert np.array_equal(runs[1][1], runs[2][1])      # replay of the grown plan: bit-identical


def threaded_ring(n_small, n_big, centre_row=16, r_small=0.1, seed=7, jitter=1e-4):
    """A unit ring (n_big segments, seeded jitter) threaded by a ring of radius
    r_small centred on its wire next to row segment centre_row, in the plane
    normal to the wire: linked (lambda = -1), every vertex-vertex distance
    about r_small, the small ring's segments 2*pi*r_small/n_small long."""
    rng = np.random.default_rng(seed)
    t = 2 * np.pi * np.arange(n_big) / n_big
    big = np.stack([np.cos(t), np.sin(t), np.zeros_like(t)], 1)
    phi = 2 * np.pi * (centre_row + 0.5) / n_big
    radial, up = np.array([np.cos(phi), np.sin(phi), 0.0]), np.array([0.0, 0.0, 1.0])
    u = 2 * np.pi * (np.arange(n_small) + 0.5) / n_small
    small = radial + r_small * (np.cos(u)[:, None] * radial + np.sin(u)[:, None] * up)
    big += rng.normal(scale=jitter, size=big.shape)
    return W.from_loops([big, small], dtype=np.float64, pairs=[[0, 1]])


@pytest.mark.parametrize("accurate_threshold", [0, 1 << 40])
def test_far_cells_below_the_distance_floor(accurate_threshold):
    """A ring of radius 5e-5 (64 segments) threading a unit ring of 640,000
    segments: around it the cells are far in segment lengths (corners beyond
    4.5 L) but closer than 1e-4 of the pair's frame, where the product of a
    cell's four edge terms nears the FP32 underflow.  Those chunks must go to
    the careful pass, in both arithmetic variants, and the pair must match the
    oracle."""
    g = threaded_ring(64, 640_000, centre_row=1000, r_small=5e-5, jitter=1e-7)
    raw, ref = check_against_oracle(g, accurate_threshold=accurate_threshold)
    assert ref[0] == pytest.approx(-1.0, abs=1e-9)
    _, _, _, s = run(g, stats=True, accurate_threshold=accurate_threshold)
    assert s["careful_chunks"] > 0


@pytest.mark.parametrize("n_small,n_big,bulk", [(29, 314, True), (48, 512, True), (24, 400, False)])
def test_angle_summation_large_chunk_angles(n_small, n_big, bulk):
    """Fast variant.  (29, 314): nearest corners at 4.6 segment lengths, every
    column of the first chunk turns by about 0.2 rad, so the chunk angle is
    taken by atan2f; (48, 512): 7.6 lengths, mostly the polynomial; (24, 400):
    3.8 lengths, closer than the angle-summation bound, so the chunk goes to
    the per-pair careful pass.  All must match the oracle, and no segment pair
    is near (m >= 3L), so nothing is recomputed in FP64."""
    g = threaded_ring(n_small, n_big)
    raw, ref = check_against_oracle(g)
    assert ref[0] == pytest.approx(-1.0, abs=1e-9)
    _, _, _, s = run(g, stats=True)
    assert s["fp64_pairs"] == 0
    assert (s["careful_chunks"] == 0) == bulk


def test_intersecting_loops_are_reported():
    t = np.arange(64) * 2 * np.pi / 64
    a = np.stack([np.cos(t), np.sin(t), 0 * t], 1)
    b = np.stack([np.cos(t), 0 * t, np.sin(t)], 1)          # shares vertices (+-1,0,0) with a
    c = np.stack([5 + np.cos(t), np.sin(t), 0 * t], 1)
    g = W.from_loops([a, b, c], pairs=[[0, 1], [0, 2]])
    for prec in (lk.LK_MIXED, lk.LK_ALL_F64):
        lk_o, raw, st = run(g, precision=prec)
        assert st[0] == lk.LK_ERR_INTERSECT and lk_o[0] == 0
        assert st[1] == lk.LK_OK and lk_o[1] == 0


def test_invalid_pairs_only_affect_themselves():
    g = W.ring_chain()
    pairs = np.array([[0, 1], [3, 3], [0, 99], [-1, 2], [2, 3]], np.int32)
    lk_o, raw, st = run(g, pairs)
    assert st.tolist() == [0, lk.LK_ERR_ARG, lk.LK_ERR_ARG, lk.LK_ERR_ARG, 0]
    ref = O.link_pairs(g.vertices, g.offsets, pairs[[0, 4]])
    assert np.abs(raw[[0, 4]] - ref).max() <= RAW_TOL


def test_empty_pair_list():
    g = W.ring_chain()
    lk_o, raw, st = run(g, np.zeros((0, 2), np.int32), on_device=False)
    assert lk_o.shape == (0,)


def test_host_and_device_buffers_agree():
    g = W.ring_chain()
    a = run(g, on_device=True)
    b = run(g, on_device=False)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_result_independent_of_batch_and_rerun():
    g = W.chainmail(rows=6, cols=10)
    full = run(g)[1]
    again = run(g)[1]
    assert np.array_equal(full, again)
    rng = np.random.default_rng(3)
    pick = rng.choice(g.pairs.shape[0], 7, replace=False)
    for k in pick:
        alone = run(g, g.pairs[k:k + 1])[1]
        assert alone[0] == full[k]
    shuffled = rng.permutation(g.pairs.shape[0])
    assert np.array_equal(run(g, g.pairs[shuffled])[1], full[shuffled])


def test_repeated_pair_list_replays_a_plan():
    """lk_verify with the same list again reuses its work tables (a graph plan)
    and must give, after every lk_update, what a fresh context gives; a
    different list in between, and a tune-table change, start over."""
    g = W.ring_chain()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    v = torch.from_numpy(np.ascontiguousarray(g.vertices)).cuda()
    off = torch.from_numpy(g.offsets).cuda()
    ctx = lk.lk_create(v, off, None, stream)
    n = g.pairs.shape[0]
    other = np.ascontiguousarray(g.pairs[::3])
    try:
        for step in range(5):
            d = rng.normal(scale=2e-3, size=g.vertices.shape)
            lk.lk_update(ctx, torch.from_numpy(d).cuda(), True, stream)
            if step == 2:
                lo2, raw2, st2 = np.zeros(other.shape[0], np.int32), np.zeros(other.shape[0]), np.zeros(other.shape[0], np.int32)
                lk.lk_verify(ctx, other, lo2, raw2, st2, stream)
            if step == 3:
                lk.lk_tune_set(ctx, np.array([[7, 7, 64]], np.int32))
            lo, raw, st = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
            lk.lk_verify(ctx, np.ascontiguousarray(g.pairs), lo, raw, st, stream)
            g = W.Geometry(g.vertices + d, g.offsets, g.pairs, g.name, {})
            ref_lo, ref_raw, ref_st = run(g)
            assert np.array_equal(st, ref_st) and np.array_equal(lo, ref_lo)
            # a changed tune table only regroups the FP64 sums
            assert np.abs(raw - ref_raw).max() <= (1e-12 if step >= 3 else 0.0)
    finally:
        lk.lk_destroy(ctx)


def test_update_matches_fresh_context():
    g = W.chainmail(rows=6, cols=10, dtype=np.float32)
    rng = np.random.default_rng(5)
    delta = rng.normal(scale=1e-3, size=g.vertices.shape).astype(np.float32)
    stream = torch.cuda.current_stream()
    v = torch.from_numpy(g.vertices).cuda()
    off = torch.from_numpy(g.offsets).cuda()
    n = g.pairs.shape[0]
    ctx = lk.lk_create(v, off, None, stream)
    try:
        lk.lk_update(ctx, torch.from_numpy(delta).cuda(), True, stream)
        lk_o, raw, st = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
        lk.lk_verify(ctx, g.pairs, lk_o, raw, st, stream)
    finally:
        lk.lk_destroy(ctx)
    moved = W.Geometry((g.vertices.astype(np.float64) + delta.astype(np.float64)), g.offsets, g.pairs)
    fresh = run(moved)
    assert np.array_equal(lk_o, fresh[0])
    assert np.abs(raw - fresh[1]).max() <= 1e-9
    ref = O.link_pairs(moved.vertices, moved.offsets, moved.pairs)
    assert np.abs(raw - ref).max() <= RAW_TOL


def test_update_boxes_of_long_and_short_loops():
    """Loop boxes are reduced over fixed vertex chunks: two torus-link
    components of 60,001 and 50,003 vertices span hundreds of chunks, and 300
    seven-vertex rings put many loops in one chunk.  After delta and absolute
    updates (FP32 and FP64 data), the candidate pairs and every result must be
    those of a fresh context built from the moved vertices."""
    rng = np.random.default_rng(9)
    tor = W.torus_link(5, 7, 60_001, n2=50_003)
    small = [W.circle(rng.uniform(-3, 3, 3), np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), 7, radius=0.2)
             for _ in range(300)]
    g = W.from_loops([tor.loop(0)] + small + [tor.loop(1)])
    stream = torch.cuda.current_stream()
    ctx = lk.lk_create(torch.from_numpy(g.vertices).cuda(), torch.from_numpy(g.offsets).cuda(), None, stream)
    x = g.vertices.copy()
    try:
        for step in range(4):
            if step % 2 == 0:
                d = rng.normal(scale=1e-3, size=x.shape).astype(np.float32)
                lk.lk_update(ctx, torch.from_numpy(d).cuda(), True, stream)
                x = x + d.astype(np.float64)
            else:
                x = x + rng.normal(scale=1e-3, size=x.shape)
                lk.lk_update(ctx, torch.from_numpy(x).cuda(), False, stream)
            pairs = lk.lk_candidates(ctx, stream=stream)
            n = pairs.shape[0]
            out = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
            lk.lk_verify(ctx, pairs, *out, stream)
            moved = W.Geometry(x.copy(), g.offsets, pairs)
            fresh_ctx = lk.lk_create(torch.from_numpy(moved.vertices).cuda(), torch.from_numpy(g.offsets).cuda(),
                                     None, stream)
            try:
                fresh_pairs = lk.lk_candidates(fresh_ctx, stream=stream)
            finally:
                lk.lk_destroy(fresh_ctx)
            assert np.array_equal(pairs, fresh_pairs)
            fresh = run(moved)
            for a, b in zip(out, fresh):
                assert np.array_equal(a, b)
            k = pairs.tolist().index([0, 301])
            assert out[2][k] == 0 and abs(out[0][k]) == 35
    finally:
        lk.lk_destroy(ctx)


def test_autotune_changes_only_the_split(tmp_path):
    from paper_2106_12655_gb300 import tuning

    g = W.chainmail(rows=12, cols=24)
    stream = torch.cuda.current_stream()
    ctx = lk.lk_create(g.vertices, g.offsets, None, stream)
    try:
        n = g.pairs.shape[0]
        base = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
        lk.lk_verify(ctx, g.pairs, *base)
        lk.lk_autotune(ctx, g.pairs, stream)
        table = lk.lk_tune_get(ctx)
        assert table.shape[0] >= 1 and np.all(table[:, 2] >= 32)
        tuned = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
        lk.lk_verify(ctx, g.pairs, *tuned)
        assert np.array_equal(tuned[0], base[0]) and np.array_equal(tuned[2], base[2])
        assert np.max(np.abs(tuned[1] - base[1])) <= 1e-9
        # and both against the oracle
        ref = O.link_pairs(g.vertices, g.offsets, g.pairs)
        assert np.array_equal(tuned[0], O.round_lk(ref).astype(np.int32)) and np.all(tuned[2] == 0)
        assert np.max(np.abs(tuned[1] - ref)) <= RAW_TOL
        # the cache round-trips the table
        path = str(tmp_path / "tune.json")
        tuning.save(ctx, "test-gpu", path)
        lk.lk_tune_set(ctx, np.zeros((0, 3), np.int32))
        assert lk.lk_tune_get(ctx).shape[0] == 0
        assert tuning.restore(ctx, "test-gpu", path)
        assert np.array_equal(lk.lk_tune_get(ctx), table)
        # a forced split gives the same answer too
        forced = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
        lk.lk_tune_set(ctx, np.array([[r, c, 64] for r, c, _ in table], np.int32))
        lk.lk_verify(ctx, g.pairs, *forced)
        assert np.max(np.abs(forced[1] - base[1])) <= 1e-9
    finally:
        lk.lk_destroy(ctx)


def test_early_exit_stops_at_the_first_changed_link():
    """Sec. 3.1's fast verification against a certificate taken from the
    oracle: every batch is enqueued at once, the first batch holding a changed
    linking number stops the later ones on the device, and the results of the
    checked prefix equal the certificate."""
    g = W.chainmail(rows=10, cols=20)
    n = g.pairs.shape[0]
    cert = O.round_lk(O.link_pairs(g.vertices, g.offsets, g.pairs)).astype(np.int32)
    per_batch = (1 << 22) // (256 * 256)                  # pairs of 256-segment rings in a 2^22 batch
    ctx = lk.lk_create(g.vertices, g.offsets)
    try:
        out = np.zeros(n, np.int32)
        raw = np.zeros(n)
        fm, checked = lk.lk_verify_expected(ctx, g.pairs, cert, 1 << 22, out, raw)
        assert fm == -1 and checked == n and np.array_equal(out, cert)
        ref = O.link_pairs(g.vertices, g.offsets, g.pairs)
        assert np.max(np.abs(raw - ref)) <= RAW_TOL
        k = (2 * n) // 3
        bad = cert.copy()
        bad[k] += 1                                   # a "pull-through" at pair k
        out = np.full(n, 77, np.int32)
        fm, checked = lk.lk_verify_expected(ctx, g.pairs, bad, 1 << 22, out)
        assert fm == k and k < checked <= k + per_batch and checked < n   # stopped after k's batch
        assert np.array_equal(out[:checked], cert[:checked]) and np.all(out[checked:] == 77)
        # a change among the first pairs: only the first batch is verified
        bad0 = cert.copy()
        bad0[3] = 5
        fm, checked = lk.lk_verify_expected(ctx, g.pairs, bad0, 1 << 22)
        assert fm == 3 and checked == per_batch
        dev = torch.from_numpy(bad).cuda()
        assert lk.lk_verify_expected(ctx, torch.from_numpy(g.pairs).cuda(), dev, 0)[0] == k
    finally:
        lk.lk_destroy(ctx)
