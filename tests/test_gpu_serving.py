"""Serving (continuous batching): results alone and in the mix, admission by
memory, geometry kept resident and updated between requests."""
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


def alone(ctx, pairs):
    n = pairs.shape[0]
    out = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
    lk.lk_verify(ctx, pairs, *out)
    return out


def drain(srv, tickets, sizes, max_steps=100000):
    res = {}
    for _ in range(max_steps):
        lk.lk_server_step(srv, wait=True)
        for t in list(tickets):
            if t in res:
                continue
            n = sizes[t]
            out = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
            if lk.lk_server_poll(srv, t, *out):
                res[t] = out
        if len(res) == len(tickets):
            return res
    raise AssertionError("server did not finish")


def scenes():
    # several resident geometries: small piles of various ring and segment counts
    gs = [W.chainmail(seed=40 + k, rows=6 + 2 * k, cols=8 + 3 * k, nseg=None,
                      nseg_per_ring=np.random.default_rng(k).integers(64, 257, size=(6 + 2 * k) * (8 + 3 * k)))
          for k in range(4)]
    gs.append(W.torus_link(2, 3, 3000, dtype=np.float32, n2=2900))     # an accurate-variant request
    return gs


def test_results_alone_and_in_the_mix_are_identical():
    gs = scenes()
    ctxs = [lk.lk_create(g.vertices, g.offsets) for g in gs]
    o = lk.lk_server_default_options()
    o.wave_items = 512                       # small waves: requests span several, and share them
    srv = lk.lk_server_create(o)
    try:
        refs, tickets, sizes, which = {}, [], {}, {}
        rng = np.random.default_rng(0)
        for rep in range(3):
            for k, (g, ctx) in enumerate(zip(gs, ctxs)):
                pairs = g.pairs if rep == 0 else g.pairs[rng.permutation(g.pairs.shape[0])][: max(1, g.pairs.shape[0] // 2)]
                pairs = np.ascontiguousarray(pairs)
                t = lk.lk_server_submit(srv, ctx, pairs)
                tickets.append(t)
                sizes[t] = pairs.shape[0]
                which[t] = (k, pairs)
                if rep == 1:
                    lk.lk_server_step(srv)           # let some run while the rest arrive
        res = drain(srv, tickets, sizes)
        st = lk.lk_server_get_stats(srv)
        assert st["completed"] == len(tickets)
        assert st["max_requests_per_wave"] >= 2          # work of several requests overlapped
        for t in tickets:
            k, pairs = which[t]
            ref = alone(ctxs[k], pairs)
            got = res[t]
            assert np.array_equal(got[2], ref[2])
            assert np.array_equal(got[0], ref[0])
            assert np.max(np.abs(got[1] - ref[1])) <= 1e-12
        # and against the oracle for one request of each scene
        for k, g in enumerate(gs):
            t = next(t for t in tickets if which[t][0] == k)
            ref = O.link_pairs(g.vertices, g.offsets, which[t][1])
            assert np.max(np.abs(res[t][1] - ref)) <= 1e-6
            assert np.array_equal(res[t][0], O.round_lk(ref).astype(np.int32))
    finally:
        lk.lk_server_destroy(srv)
        for c in ctxs:
            lk.lk_destroy(c)


def test_admission_waits_for_arena_memory():
    g = W.chainmail(seed=7, rows=8, cols=16)
    ctx = lk.lk_create(g.vertices, g.offsets)
    # measure one request's arena footprint, then give the server room for
    # one such request at a time
    # (host packing: a request's whole footprint is known when it is submitted)
    o0 = lk.lk_server_default_options()
    o0.pack_on_device = 0
    probe = lk.lk_server_create(o0)
    t = lk.lk_server_submit(probe, ctx, g.pairs)
    lk.lk_server_step(probe)
    one = lk.lk_server_get_stats(probe)["arena_used"]
    drain(probe, [t], {t: g.pairs.shape[0]})
    lk.lk_server_destroy(probe)
    assert one > 0
    o = lk.lk_server_default_options()
    o.pack_on_device = 0
    o.arena_bytes = int(one * 1.5)
    o.wave_items = 256
    srv = lk.lk_server_create(o)
    try:
        tickets, sizes = [], {}
        for _ in range(4):
            t = lk.lk_server_submit(srv, ctx, g.pairs)
            tickets.append(t)
            sizes[t] = g.pairs.shape[0]
        lk.lk_server_step(srv)
        st = lk.lk_server_get_stats(srv)
        assert st["running"] == 1 and st["queued"] == 3       # admission held back by memory
        assert st["arena_used"] <= o.arena_bytes
        res = drain(srv, tickets, sizes)
        ref = alone(ctx, g.pairs)
        for t in tickets:
            assert np.array_equal(res[t][1], ref[1])
        too_big = W.chainmail(seed=8, rows=32, cols=64)
        ctx2 = lk.lk_create(too_big.vertices, too_big.offsets)
        with pytest.raises(lk.LkError) as ei:
            lk.lk_server_submit(srv, ctx2, too_big.pairs)
        assert ei.value.status == lk.LK_ERR_OOM
        lk.lk_destroy(ctx2)
    finally:
        lk.lk_server_destroy(srv)
        lk.lk_destroy(ctx)


def test_resident_geometry_updated_between_requests():
    g = W.chainmail(seed=11, rows=6, cols=10)
    ctx = lk.lk_create(g.vertices, g.offsets)
    srv = lk.lk_server_create(None)
    stream = lk.lk_server_stream(srv)
    rng = np.random.default_rng(2)
    verts = g.vertices.astype(np.float64).copy()
    try:
        for step in range(3):
            delta = rng.normal(scale=2e-3, size=g.vertices.shape).astype(np.float32)
            lk.lk_update(ctx, delta, True, stream)   # ordered before the request on the server's stream
            verts += delta.astype(np.float64)
            t = lk.lk_server_submit(srv, ctx, g.pairs)
            res = drain(srv, [t], {t: g.pairs.shape[0]})[t]
            ref = O.link_pairs(verts, g.offsets, g.pairs)
            assert np.all(res[2] == 0)
            assert np.array_equal(res[0], O.round_lk(ref).astype(np.int32))
            assert np.max(np.abs(res[1] - ref)) <= 1e-6
    finally:
        lk.lk_server_destroy(srv)
        lk.lk_destroy(ctx)


def test_completed_reports_each_finished_ticket_once():
    gs = scenes()[:3]
    ctxs = [lk.lk_create(g.vertices, g.offsets) for g in gs]
    srv = lk.lk_server_create(None)
    try:
        sizes, tickets = {}, []
        for k, g in enumerate(gs):
            for w in range(3):
                p = np.ascontiguousarray(g.pairs[w::3])
                t = lk.lk_server_submit(srv, ctxs[k], p)
                sizes[t] = (p.shape[0], k, p)
                tickets.append(t)
        seen = []
        for _ in range(100000):
            lk.lk_server_step(srv, wait=True)
            seen += lk.lk_server_completed(srv)
            if len(seen) == len(tickets):
                break
        assert sorted(seen) == sorted(tickets) and len(set(seen)) == len(seen)
        assert lk.lk_server_completed(srv) == []
        for t in seen:
            n, k, p = sizes[t]
            out = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
            assert lk.lk_server_poll(srv, t, *out)
            ref = alone(ctxs[k], p)
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[2], ref[2])
            assert np.array_equal(out[1], ref[1])
    finally:
        lk.lk_server_destroy(srv)
        for c in ctxs:
            lk.lk_destroy(c)


def test_fp64_list_overflow_is_reported_and_exact():
    """A server whose per-request FP64 list holds 8 entries evaluates the rest
    in place: the results must equal lk_verify's, and the statistics must show
    the overflow."""
    g = W.serving_pile(77, 400, 400)            # 64-256-segment rings: many near segment pairs
    ctx = lk.lk_create(g.vertices, g.offsets)
    o = lk.lk_server_default_options()
    o.near_capacity = 8
    srv = lk.lk_server_create(o)
    try:
        pairs = np.ascontiguousarray(g.pairs)
        t = lk.lk_server_submit(srv, ctx, pairs)
        res = drain(srv, [t], {t: pairs.shape[0]})[t]
        ref = alone(ctx, pairs)
        assert np.array_equal(res[0], ref[0]) and np.array_equal(res[2], ref[2])
        assert np.abs(res[1] - ref[1]).max() <= 1e-12
        st = lk.lk_server_get_stats(srv)
        assert st["near_overflow"] > 0 and st["careful_chunks"] > 0
    finally:
        lk.lk_server_destroy(srv)
        lk.lk_destroy(ctx)


def test_fewest_items_first_order_changes_no_result():
    gs = scenes()
    ctxs = [lk.lk_create(g.vertices, g.offsets) for g in gs]
    o = lk.lk_server_default_options()
    o.wave_items = 512
    o.wave_order = 1
    srv = lk.lk_server_create(o)
    try:
        tickets, sizes, which = [], {}, {}
        for rep in range(2):
            for k, (g, ctx) in enumerate(zip(gs, ctxs)):
                pairs = np.ascontiguousarray(g.pairs if rep == 0 else g.pairs[: max(1, g.pairs.shape[0] // 3)])
                t = lk.lk_server_submit(srv, ctx, pairs)
                tickets.append(t)
                sizes[t] = pairs.shape[0]
                which[t] = (k, pairs)
        res = drain(srv, tickets, sizes)
        assert lk.lk_server_get_stats(srv)["max_requests_per_wave"] >= 2
        for t in tickets:
            k, pairs = which[t]
            ref = alone(ctxs[k], pairs)
            for a, b in zip(res[t], ref):
                assert np.array_equal(a, b)
    finally:
        lk.lk_server_destroy(srv)
        for c in ctxs:
            lk.lk_destroy(c)
    bad = lk.lk_server_default_options()
    bad.wave_order = 2
    with pytest.raises(lk.LkError):
        lk.lk_server_create(bad)


def test_lists_packed_on_the_device_equal_host_packing():
    gs = scenes()
    ctxs = [lk.lk_create(g.vertices, g.offsets) for g in gs]
    # a tune table on one context reaches the device packer too
    lk.lk_tune_set(ctxs[1], np.array([[r, c, 64] for r in range(6, 9) for c in range(6, 9)], np.int32))
    lists = []
    rng = np.random.default_rng(3)
    for k, g in enumerate(gs):
        p = np.ascontiguousarray(g.pairs[rng.permutation(g.pairs.shape[0])])
        if k == 0:       # invalid pairs: a loop with itself, an index past the end, a negative one
            bad = np.array([[0, 0], [1, g.n_loops], [-1, 2]], np.int32)
            p = np.ascontiguousarray(np.concatenate([p[:5], bad, p[5:]]))
        lists.append((k, p))
    results = []
    for on_device in (0, 1):
        o = lk.lk_server_default_options()
        o.wave_items = 512
        o.pack_on_device = on_device
        srv = lk.lk_server_create(o)
        try:
            tickets, sizes = [], {}
            for k, p in lists:
                t = lk.lk_server_submit(srv, ctxs[k], p)
                tickets.append(t)
                sizes[t] = p.shape[0]
            res = drain(srv, tickets, sizes)
            results.append([res[t] for t in tickets])
        finally:
            lk.lk_server_destroy(srv)
    for a, b in zip(*results):
        for x, y in zip(a, b):
            # invalid pairs have no raw sum (NaN) on both servers
            assert np.array_equal(x, y, equal_nan=bool(np.issubdtype(x.dtype, np.floating)))
    st0 = results[1][0][2]
    assert (st0[5:8] == lk.LK_ERR_ARG).all() and (np.delete(st0, [5, 6, 7]) == 0).all()
    # a list of invalid pairs only
    o = lk.lk_server_default_options()
    o.pack_on_device = 1
    srv = lk.lk_server_create(o)
    try:
        bad = np.array([[0, 0], [3, 3]], np.int32)
        t = lk.lk_server_submit(srv, ctxs[0], bad)
        res = drain(srv, [t], {t: 2})[t]
        assert (res[2] == lk.LK_ERR_ARG).all()
    finally:
        lk.lk_server_destroy(srv)
        for c in ctxs:
            lk.lk_destroy(c)
    o.pack_on_device = 2
    with pytest.raises(lk.LkError):
        lk.lk_server_create(o)


def test_device_packed_requests_wait_for_room_and_fail_at_poll_when_too_large():
    g = W.chainmail(seed=7, rows=8, cols=16)
    ctx = lk.lk_create(g.vertices, g.offsets)
    torus = W.torus_link(2, 3, 100_000, dtype=np.float32)
    ctx2 = lk.lk_create(torus.vertices, torus.offsets)
    # one request's largest footprint (pack block, then its work buffers too)
    probe = lk.lk_server_create(None)
    t = lk.lk_server_submit(probe, ctx, g.pairs)
    peak, out = 0, np.zeros(g.pairs.shape[0])
    for _ in range(100000):
        lk.lk_server_step(probe)
        peak = max(peak, lk.lk_server_get_stats(probe)["arena_used"])
        if lk.lk_server_poll(probe, t, None, out, None):
            break
    lk.lk_server_destroy(probe)
    assert peak > 0
    o = lk.lk_server_default_options()
    o.arena_bytes = int(peak * 1.5)
    o.wave_items = 256
    srv = lk.lk_server_create(o)
    try:
        tickets, sizes = [], {}
        for _ in range(4):
            t = lk.lk_server_submit(srv, ctx, g.pairs)
            tickets.append(t)
            sizes[t] = g.pairs.shape[0]
        # the four footprints together exceed the arena, so requests had to
        # wait for room (their pack blocks or their work buffers) ...
        assert 4 * peak > o.arena_bytes
        for _ in range(20):
            lk.lk_server_step(srv)
            assert lk.lk_server_get_stats(srv)["arena_used"] <= o.arena_bytes   # ... and never overran it
        res = drain(srv, tickets, sizes)
        ref = alone(ctx, g.pairs)
        for t in tickets:
            assert np.array_equal(res[t][0], ref[0]) and np.array_equal(res[t][1], ref[1])
        # one pair (a small list) whose work buffers, for its 65k items and
        # 2.4M chunks, exceed the arena
        t = lk.lk_server_submit(srv, ctx2, np.ascontiguousarray(torus.pairs))
        with pytest.raises(lk.LkError) as ei:
            for _ in range(100000):
                lk.lk_server_step(srv, wait=True)
                if lk.lk_server_poll_pairs(srv, t)[0]:
                    break
        assert ei.value.status == lk.LK_ERR_OOM
        assert lk.lk_server_get_stats(srv)["arena_used"] == 0
    finally:
        lk.lk_server_destroy(srv)
        lk.lk_destroy(ctx)
        lk.lk_destroy(ctx2)
