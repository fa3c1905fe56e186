"""Serving requests that carry geometry only: the potential link search (Sec.
3.2, Algorithm 2) and the packing of its pairs run on the device.  The pairs
must equal the oracle's candidate list, and each pair's result must equal a
pair-list request's bit for bit and the oracle's within 1e-6."""
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


def take_all(srv, tickets, max_steps=200000):
    """{ticket: (pairs, lk, raw, status)} once every ticket has finished."""
    res = {}
    for _ in range(max_steps):
        lk.lk_server_step(srv, wait=True)
        for t in tickets:
            if t not in res:
                r = lk.server_take_pairs(srv, t)
                if r is not None:
                    res[t] = r
        if len(res) == len(tickets):
            return res
    raise AssertionError("server did not finish")


def check_against_oracle(g, got, n_sample=200, seed=0, vertices=None):
    pairs, lkv, raw, st = got
    v = g.vertices if vertices is None else vertices
    assert np.array_equal(pairs, O.candidates(v, g.offsets))
    assert np.all(st == 0)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(pairs.shape[0], size=min(n_sample, pairs.shape[0]), replace=False))
    ref = O.link_pairs(v, g.offsets, np.ascontiguousarray(pairs[idx]))
    assert np.max(np.abs(raw[idx] - ref)) <= 1e-6
    assert np.array_equal(lkv[idx], O.round_lk(ref).astype(np.int32))


def geometries():
    return [W.serving_pile(101, 300, 300),                                  # 64-256-segment rings
            W.chainmail(seed=3, rows=10, cols=14),
            W.torus_link(2, 3, 3000, dtype=np.float32, n2=2900)]             # one accurate-variant pair


def test_geometry_request_equals_candidates_and_pair_list_request():
    gs = geometries()
    ctxs = [lk.lk_create(g.vertices, g.offsets) for g in gs]
    o = lk.lk_server_default_options()
    o.wave_items = 512                       # requests span several waves and share them
    srv = lk.lk_server_create(o)
    try:
        geo = [lk.lk_server_submit_geometry(srv, c) for c in ctxs]
        res = take_all(srv, geo)
        st = lk.lk_server_get_stats(srv)
        assert st["geometry_requests"] == len(gs)
        assert st["candidate_pairs"] == sum(res[t][0].shape[0] for t in geo)
        # the same lists as pair-list requests, on the same server
        lists = [lk.lk_server_submit(srv, c, np.ascontiguousarray(res[t][0])) for c, t in zip(ctxs, geo)]
        ref = take_all(srv, lists)
        for g, t, u in zip(gs, geo, lists):
            assert np.array_equal(res[t][0], ref[u][0])
            for k in (1, 2, 3):
                assert np.array_equal(res[t][k], ref[u][k])
            check_against_oracle(g, res[t])
    finally:
        lk.lk_server_destroy(srv)
        for c in ctxs:
            lk.lk_destroy(c)


def test_sort_and_sweep_search_feeds_the_packer():
    # 16,900 rings: above 2^27 box pairs the search sorts and sweeps
    g = W.chainmail(seed=9, rows=130, cols=130, nseg=32)
    ctx = lk.lk_create(g.vertices, g.offsets)
    srv = lk.lk_server_create(None)
    try:
        t = lk.lk_server_submit_geometry(srv, ctx)
        got = take_all(srv, [t])[t]
        assert got[0].shape[0] > 0
        assert np.array_equal(got[0], lk.lk_candidates(ctx))
        u = lk.lk_server_submit(srv, ctx, np.ascontiguousarray(got[0]))
        ref = take_all(srv, [u])[u]
        # every handed-over chunk found room in its request's list (no item
        # was handed over whole), so the two results agree bit for bit
        assert lk.lk_server_get_stats(srv)["careful_items"] == 0
        for k in (1, 2, 3):
            assert np.array_equal(got[k], ref[k])
        check_against_oracle(g, got)
    finally:
        lk.lk_server_destroy(srv)
        lk.lk_destroy(ctx)


def test_tune_table_reaches_the_device_packer():
    g = W.serving_pile(102, 200, 200)
    ctx = lk.lk_create(g.vertices, g.offsets)
    srv = lk.lk_server_create(None)
    try:
        def items_of(submit):
            before = lk.lk_server_get_stats(srv)["items_launched"]
            t = submit()
            out = take_all(srv, [t])[t]
            return lk.lk_server_get_stats(srv)["items_launched"] - before, out

        n0, base = items_of(lambda: lk.lk_server_submit_geometry(srv, ctx))
        # 32 rows per item for every size class of these rings (64-256 segments)
        lk.lk_tune_set(ctx, np.array([[r, c, 32] for r in range(6, 9) for c in range(6, 9)], np.int32))
        n1, tuned = items_of(lambda: lk.lk_server_submit_geometry(srv, ctx))
        n2, listed = items_of(lambda: lk.lk_server_submit(srv, ctx, np.ascontiguousarray(tuned[0])))
        assert n1 == n2 and n1 > n0                 # the same split as the host packer, not the default
        assert np.array_equal(tuned[0], base[0])
        for k in (1, 2, 3):
            assert np.array_equal(tuned[k], listed[k])
        assert np.array_equal(tuned[1], base[1])
        assert np.max(np.abs(tuned[2] - base[2])) <= 1e-9
    finally:
        lk.lk_server_destroy(srv)
        lk.lk_destroy(ctx)


def test_search_follows_an_update_on_the_server_stream():
    g = W.chainmail(seed=12, rows=6, cols=10)
    ctx = lk.lk_create(g.vertices, g.offsets)
    srv = lk.lk_server_create(None)
    stream = lk.lk_server_stream(srv)
    rng = np.random.default_rng(4)
    verts = g.vertices.astype(np.float64).copy()
    try:
        for step in range(3):
            # large enough to change which boxes overlap
            delta = rng.normal(scale=0.05, size=g.vertices.shape).astype(np.float32)
            lk.lk_update(ctx, delta, True, stream)
            verts += delta.astype(np.float64)
            t = lk.lk_server_submit_geometry(srv, ctx)
            got = take_all(srv, [t])[t]
            check_against_oracle(g, got, seed=step, vertices=verts)
    finally:
        lk.lk_server_destroy(srv)
        lk.lk_destroy(ctx)


def test_no_candidates_small_buffer_and_arena_limits():
    srv = lk.lk_server_create(None)
    ctxs = []
    try:
        # three rings far apart: no candidate pair
        ring = W.chainmail(seed=1, rows=1, cols=1, nseg=64)
        v = np.concatenate([ring.vertices + np.float32(10 * k) for k in range(3)])
        off = np.array([0, 64, 128, 192], np.int64)
        ctxs.append(lk.lk_create(v, off))
        # one loop only
        ctxs.append(lk.lk_create(ring.vertices, ring.offsets))
        for c in ctxs:
            t = lk.lk_server_submit_geometry(srv, c)
            got = take_all(srv, [t])[t]
            assert got[0].shape == (0, 2)
        # a buffer too small keeps the ticket
        g = W.chainmail(seed=5, rows=4, cols=6)
        ctxs.append(lk.lk_create(g.vertices, g.offsets))
        t = lk.lk_server_submit_geometry(srv, ctxs[-1])
        for _ in range(100000):
            lk.lk_server_step(srv, wait=True)
            done, n = lk.lk_server_poll_pairs(srv, t, capacity=0)
            if done:
                break
        assert done and n == g.pairs.shape[0]
        got = lk.server_take_pairs(srv, t)
        assert np.array_equal(got[0], g.pairs)
        with pytest.raises(lk.LkError):
            lk.lk_server_poll_pairs(srv, t)          # released
        with pytest.raises(lk.LkError):
            lk.lk_server_poll(srv, lk.lk_server_submit_geometry(srv, ctxs[-1]))   # not for geometry tickets
    finally:
        lk.lk_server_destroy(srv)
        for c in ctxs:
            lk.lk_destroy(c)
    # an arena that holds the search but not the packed candidates
    g = W.serving_pile(103, 2000, 2000)
    ctx = lk.lk_create(g.vertices, g.offsets)
    o = lk.lk_server_default_options()
    o.arena_bytes = 1 << 20
    srv = lk.lk_server_create(o)
    try:
        t = lk.lk_server_submit_geometry(srv, ctx)
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


def test_mixed_geometry_and_list_requests_equal_their_solo_results():
    gs = [W.serving_pile(110 + k, 150, 600) for k in range(3)]
    ctxs = [lk.lk_create(g.vertices, g.offsets) for g in gs]
    o = lk.lk_server_default_options()
    o.wave_items = 1024                      # several requests share each wave
    try:
        # each request alone on a fresh server
        solo = {}
        for k, c in enumerate(ctxs):
            srv = lk.lk_server_create(o)
            try:
                t = lk.lk_server_submit_geometry(srv, c)
                solo[("g", k)] = take_all(srv, [t])[t]
                half = np.ascontiguousarray(gs[k].pairs[::2])
                t = lk.lk_server_submit(srv, c, half)
                solo[("l", k)] = take_all(srv, [t])[t]
            finally:
                lk.lk_server_destroy(srv)
        # all of them interleaved, twice over, on one server
        srv = lk.lk_server_create(o)
        try:
            which = {}
            for rep in range(2):
                for k, c in enumerate(ctxs):
                    which[lk.lk_server_submit_geometry(srv, c)] = ("g", k)
                    which[lk.lk_server_submit(srv, c, np.ascontiguousarray(gs[k].pairs[::2]))] = ("l", k)
                    lk.lk_server_step(srv)
            res = take_all(srv, list(which))
            assert lk.lk_server_get_stats(srv)["max_requests_per_wave"] >= 2
        finally:
            lk.lk_server_destroy(srv)
        for t, key in which.items():
            for a, b in zip(res[t], solo[key]):
                assert np.array_equal(a, b)
        for k, g in enumerate(gs):
            check_against_oracle(g, solo[("g", k)], n_sample=100, seed=k)
    finally:
        for c in ctxs:
            lk.lk_destroy(c)
