"""The paper's large-input stress shapes (Sec. 4, Table 1 and Fig. "Large-Input
Stress Tests") through both exact methods: woundballs, whose linking number 0
comes from many terms that cancel, and thick square links, L^2/4 linked pairs
of lk = 1 found by the device's potential link search.  At the oracle's sizes
the results are compared with the oracle; at the paper's sizes with the
closed forms (the oracle would need hours of host time there)."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_12655_gb300 import lk
from paper_2106_12655_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RAW_TOL = 1e-6      # the raw-sum tolerance of the method, as in the parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12655_gb300 import build as B

    B.build()
    lk.load()


METHODS = {"ds": lk.LK_METHOD_DS, "cc": lk.LK_METHOD_CC}


def run(g, pairs=None, method="ds", candidates=False, **opts):
    """Verify ``pairs`` (or the device's candidate pairs) with one method; returns
    (pairs, lk, raw, status, stats, seconds)."""
    o = lk.lk_default_options()
    o.method = METHODS[method]
    for k, v in opts.items():
        setattr(o, k, v)
    stream = torch.cuda.current_stream()
    v = torch.from_numpy(np.ascontiguousarray(g.vertices)).cuda()
    off = torch.from_numpy(g.offsets).cuda()
    ctx = lk.lk_create(v, off, o, stream)
    try:
        if candidates:
            pairs = lk.lk_candidates(ctx, stream=stream)
        pairs = np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1, 2))
        n = pairs.shape[0]
        out = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lk.lk_verify(ctx, pairs, *out, stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = lk.lk_get_stats(ctx)
    finally:
        lk.lk_destroy(ctx)
    return (pairs,) + out + (st, dt)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("method", ["ds", "cc"])
def test_woundball_matches_oracle(method, dtype):
    g = W.woundball(20, 4000, n2=3001)
    g.vertices = g.vertices.astype(dtype)
    _, lk_o, raw, status, st, _ = run(g, g.pairs, method)
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs)
    assert status[0] == lk.LK_OK and lk_o[0] == 0 == O.round_lk(ref)[0]
    if method == "cc":
        assert st["cc_fallback_pairs"] == 0 and raw[0] == 0.0
    else:
        assert abs(raw[0] - ref[0]) <= RAW_TOL, (raw[0], ref[0])


@pytest.mark.parametrize("nu,n", [(1000, 500_000), (10_000, 1_000_000)])
def test_woundball_paper_sizes(nu, n):
    """Table 1's woundballs: nu = 10^3 with 10^6 segments and nu = 10^4 with
    2x10^6 segments in two loops (up to 10^12 segment pairs in one pair)."""
    g = W.woundball(nu, n)
    g.vertices = g.vertices.astype(np.float32)
    _, lk_d, raw_d, st_d, stats_d, t_d = run(g, g.pairs, "ds")
    # about 1.5 nu^2 projected crossings: give the candidate list room for all
    _, lk_c, raw_c, st_c, stats_c, t_c = run(g, g.pairs, "cc", cc_capacity=3 * nu * nu)
    print(f"woundball nu={nu} n={n}: ds raw {raw_d[0]:.3e} in {t_d:.3f} s (precise pairs "
          f"{stats_d['precise_pairs']}); cc raw {raw_c[0]} in {t_c:.3f} s, {stats_c['cc_candidates']} candidates")
    assert st_d[0] == lk.LK_OK and lk_d[0] == 0
    # 10^11-10^12 terms whose angles sum to about 5e8 rad and cancel: FP32
    # terms alone would leave a random error near 1e-5, so the bulk sweep's
    # error estimate sends the pair to the compensated sweep, which meets 1e-6
    assert abs(raw_d[0]) <= RAW_TOL, raw_d[0]
    if nu == 10_000:
        assert stats_d["precise_pairs"] == 1
    assert st_c[0] == lk.LK_OK and lk_c[0] == 0 and raw_c[0] == 0.0
    assert stats_c["cc_fallback_pairs"] == 0


@pytest.mark.parametrize("method", ["ds", "cc"])
def test_square_links_match_oracle(method):
    g = W.square_links(12, 200)
    pairs, lk_o, raw, status, st, _ = run(g, method=method, candidates=True)
    # the device's box search finds exactly the cross-family pairs
    assert np.array_equal(pairs, g.pairs)
    ref = O.link_pairs(g.vertices, g.offsets, pairs)
    assert np.all(status == lk.LK_OK)
    assert np.array_equal(lk_o, O.round_lk(ref).astype(np.int32)) and np.all(lk_o == 1)
    if method == "cc":
        assert st["cc_fallback_pairs"] == 0 and np.array_equal(raw, lk_o.astype(np.float64))
    else:
        assert np.max(np.abs(raw - ref)) <= RAW_TOL, np.max(np.abs(raw - ref))


@pytest.mark.parametrize("method", ["ds", "cc"])
def test_square_links_paper_size(method):
    """Table 1's thick square link: 1,250 loops, 5x10^5 segments, 390,625 linked
    pairs from the device's potential link search, every one lk = 1."""
    g = W.square_links(625, 400, dtype=np.float32)
    assert g.vertices.shape[0] == 500_000
    # about four projected crossings per pair: room for all of them
    opts = {"cc_capacity": 1 << 23} if method == "cc" else {}
    pairs, lk_o, raw, status, st, dt = run(g, method=method, candidates=True, **opts)
    print(f"square links {method}: {pairs.shape[0]} pairs in {dt:.3f} s; fp64 pairs {st['fp64_pairs']}, "
          f"careful items {st['careful_items']}, near overflow {st['near_overflow']}")
    assert np.array_equal(pairs, g.pairs)
    assert np.all(status == lk.LK_OK), np.unique(status, return_counts=True)
    assert np.all(lk_o == 1)
    if method == "cc":
        assert st["cc_fallback_pairs"] == 0 and np.array_equal(raw, lk_o.astype(np.float64))
    else:
        assert np.max(np.abs(raw - 1.0)) <= RAW_TOL, np.max(np.abs(raw - 1.0))


@pytest.mark.parametrize("method", ["ds", "cc"])
def test_square_links_paper_largest(method):
    """Table 1's larger thick square link: 5,000 loops, 4x10^6 segments,
    6,250,000 linked pairs (4x10^12 segment pairs, about 1e9 of them near
    enough for the FP64 path), every one lk = 1; the work lists are sized for
    it up front."""
    g = W.square_links(2500, 800, dtype=np.float32)
    assert g.vertices.shape[0] == 4_000_000
    opts = ({"cc_capacity": 1 << 26} if method == "cc"
            else {"near_capacity": 1_400_000_000, "chunk_capacity": 1 << 26})
    pairs, lk_o, raw, status, st, dt = run(g, method=method, candidates=True, **opts)
    print(f"square links 5000 {method}: {pairs.shape[0]} pairs in {dt:.2f} s; fp64 pairs {st['fp64_pairs']}, "
          f"near overflow {st['near_overflow']}, candidates {st['cc_candidates']}")
    assert np.array_equal(pairs, g.pairs)
    assert np.all(status == lk.LK_OK) and np.all(lk_o == 1)
    if method == "cc":
        assert st["cc_fallback_pairs"] == 0 and np.array_equal(raw, lk_o.astype(np.float64))
    else:
        assert st["near_overflow"] == 0 and np.max(np.abs(raw - 1.0)) <= RAW_TOL
