"""Counting crossings (LK_METHOD_CC; Sec. 3.4, Method 1, Algorithm 4): the
linking numbers must equal the FP64 direct-sum oracle's exactly, and a pair
decided by its crossings returns the exact integer as its raw value.  Pairs
the projection cannot decide (forced here by a tiny candidate list) fall
back to the direct sum in the same call.  Each candidate search (the
all-pairs sweep, the one-CTA binned search, the device-wide grid) must give
the same results."""
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


def run_cc(g, pairs=None, **opts):
    pairs = g.pairs if pairs is None else np.asarray(pairs, np.int32).reshape(-1, 2)
    o = lk.lk_default_options()
    o.method = lk.LK_METHOD_CC
    for k, v in opts.items():
        setattr(o, k, v)
    stream = torch.cuda.current_stream()
    ctx = lk.lk_create(np.ascontiguousarray(g.vertices), g.offsets, o, stream)
    try:
        n = pairs.shape[0]
        out = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
        lk.lk_verify(ctx, np.ascontiguousarray(pairs), *out, stream)
        st = lk.lk_get_stats(ctx)
    finally:
        lk.lk_destroy(ctx)
    return out + (st,)


def check(g, pairs=None, **opts):
    pairs = g.pairs if pairs is None else np.asarray(pairs, np.int32).reshape(-1, 2)
    lk_o, raw, status, st = run_cc(g, pairs, **opts)
    ref = O.round_lk(O.link_pairs(g.vertices, g.offsets, pairs)).astype(np.int32)
    assert np.all(status == lk.LK_OK), np.unique(status, return_counts=True)
    assert np.array_equal(lk_o, ref), np.nonzero(lk_o != ref)
    return lk_o, raw, st


SEARCH = {"auto": lk.LK_CC_SEARCH_AUTO, "sweep": lk.LK_CC_SEARCH_SWEEP, "binned": lk.LK_CC_SEARCH_BINNED}


@pytest.mark.parametrize("search", list(SEARCH))
@pytest.mark.parametrize("name", ["ring_chain", "chainmail", "torus_small", "whitehead", "ribbon", "hopf"])
def test_cc_matches_oracle_and_is_exact(name, search):
    g = {"ring_chain": lambda: W.ring_chain(),
         "chainmail": lambda: W.chainmail(),
         "torus_small": lambda: W.torus_link(5, 7, 3000, dtype=np.float32, n2=2711),
         "whitehead": lambda: W.whitehead(),
         "ribbon": lambda: W.double_helix_ribbon(25, 6000),
         "hopf": lambda: W.hopf(24, 30)}[name]()
    lk_o, raw, st = check(g, cc_search=SEARCH[search])
    # decided by crossings: the raw value is the integer itself
    assert st["cc_fallback_pairs"] == 0
    assert np.array_equal(raw, lk_o.astype(np.float64))
    assert st["fp64_pairs"] == 0


def test_cc_knit_yarn_sampled_pairs():
    g = W.knit_yarn()
    rng = np.random.default_rng(4)
    pick = np.sort(rng.choice(g.pairs.shape[0], 12, replace=False))
    lk_o, raw, st = check(g, g.pairs[pick])
    assert np.array_equal(raw, lk_o.astype(np.float64))


def test_cc_large_torus_closed_form():
    g = W.torus_link(31, 37, 250_000, dtype=np.float32)
    lk_o, raw, status, st = run_cc(g)
    assert status[0] == lk.LK_OK and lk_o[0] == -31 * 37
    assert st["cc_fallback_pairs"] == 0 and raw[0] == -31 * 37


@pytest.mark.parametrize("search", list(SEARCH))
def test_cc_random_polygons_against_exact_crossings(search):
    import crossings as C

    rng = np.random.default_rng(12)
    loops, pairs, expect = [], [], []
    for k in range(40):
        a = rng.normal(size=(rng.integers(4, 30), 3))
        b = rng.normal(size=(rng.integers(4, 30), 3)) + rng.normal(scale=0.3, size=3)
        try:
            lam = C.linking_number_exact(a, b, rng=rng)
        except C.Intersecting:
            continue
        base = len(loops)
        loops += [a, b]
        pairs.append([base, base + 1])
        expect.append(lam)
    g = W.from_loops(loops, dtype=np.float64, pairs=pairs)
    lk_o, raw, status, st = run_cc(g, cc_search=SEARCH[search])
    assert np.all(status == lk.LK_OK)
    assert np.array_equal(lk_o, np.asarray(expect, np.int32))


@pytest.mark.parametrize("search", ["sweep", "binned"])
def test_cc_fallback_to_direct_sum(search):
    """A one-entry candidate list: every pair with more than one candidate is
    computed by the direct sum instead; the linking numbers do not change."""
    g = W.chainmail(rows=6, cols=10, dtype=np.float64)
    lk_full, raw_full, _ = check(g, cc_search=SEARCH[search])
    lk_o, raw, st = check(g, cc_capacity=1, cc_search=SEARCH[search])
    assert np.array_equal(lk_o, lk_full)
    fell_back = raw != lk_o.astype(np.float64)
    assert fell_back.any() and not fell_back.all()
    assert st["cc_fallback_pairs"] == int(fell_back.sum())
    ref = O.link_pairs(g.vertices, g.offsets, g.pairs)
    assert np.abs(raw[fell_back] - ref[fell_back]).max() <= 1e-6


@pytest.mark.parametrize("search", list(SEARCH))
def test_cc_reports_intersections(search):
    t = np.arange(64) * 2 * np.pi / 64
    a = np.stack([np.cos(t), np.sin(t), 0 * t], 1)
    b = np.stack([np.cos(t), 0 * t, np.sin(t)], 1)          # shares vertices (+-1,0,0) with a
    c = np.stack([5 + np.cos(t), np.sin(t), 0 * t], 1)
    g = W.from_loops([a, b, c], pairs=[[0, 1], [0, 2]])
    lk_o, raw, status, st = run_cc(g, cc_search=SEARCH[search])
    assert status[0] == lk.LK_ERR_INTERSECT and lk_o[0] == 0
    assert status[1] == lk.LK_OK and lk_o[1] == 0 and raw[1] == 0.0


@pytest.mark.parametrize("name", ["woundball", "torus", "ribbon", "whitehead"])
def test_cc_binned_search_matches_oracle(name):
    """Pairs of at least 2^28 segment pairs take the binned candidate search
    (Algorithm 4's accelerated query, as a uniform grid over the projection):
    the linking numbers must equal the oracle's, decided by crossings alone
    (raw exact, no fallback)."""
    g = {"woundball": lambda: W.woundball(100, 20_000),
         "torus": lambda: W.torus_link(5, 7, 20_000, n2=17_001),
         "ribbon": lambda: W.double_helix_ribbon(25, 20_000),
         "whitehead": lambda: W.whitehead(20_000, 30_000)}[name]()
    assert g.segment_pairs() >= 1 << 28
    lk_o, raw, st = check(g)
    assert st["cc_fallback_pairs"] == 0
    assert np.array_equal(raw, lk_o.astype(np.float64))


@pytest.mark.parametrize("search", ["sweep", "binned"])
def test_cc_search_boundary_sizes(search):
    """Loops at and just past the one-CTA limit (2,048 segments), loops of a few
    segments, a pair whose projections cross but do not link and one whose
boxes lie apart:
    every search gives the oracle's linking numbers, decided by crossings."""
    rng = np.random.default_rng(31)
    loops, pairs = [], []
    for n1, n2 in [(2048, 2048), (2049, 2048), (2048, 3000), (3, 5), (4, 2048), (700, 9)]:
        t1 = np.arange(n1) * 2 * np.pi / n1
        t2 = np.arange(n2) * 2 * np.pi / n2
        a = np.stack([np.cos(t1), np.sin(t1), 0.05 * np.sin(3 * t1)], 1)
        b = np.stack([1 + np.cos(t2), 0.1 * np.sin(2 * t2), np.sin(t2)], 1)
        a += rng.normal(scale=1e-3, size=a.shape)
        b += rng.normal(scale=1e-3, size=b.shape)
        base = len(loops)
        loops += [a, b]
        pairs.append([base, base + 1])
    # a ring above the first one whose projection crosses it (lk = 0 from
    # crossings that cancel), and one whose box lies apart from it
    t = np.arange(300) * 2 * np.pi / 300
    loops.append(np.stack([1.3 + 0.5 * np.cos(t), 0.5 * np.sin(t), 0.3 + 0 * t], 1))
    pairs.append([0, len(loops) - 1])
    loops.append(np.stack([2.5 + 0.5 * np.cos(t), 0.5 * np.sin(t), 0 * t], 1))
    pairs.append([0, len(loops) - 1])
    g = W.from_loops(loops, dtype=np.float64, pairs=pairs)
    lk_o, raw, st = check(g, cc_search=SEARCH[search])
    assert st["cc_fallback_pairs"] == 0
    assert np.array_equal(raw, lk_o.astype(np.float64))


def test_cc_one_cta_search_many_candidates():
    """An interwound pair of loops under the one-CTA limit (2,000 and 1,999
    segments, nu = 20: about 600 projected crossings) produces more candidates
    than a CTA buffers (256); the rest go to the list directly.  lk = 0 from
    crossings that cancel, raw exact."""
    g = W.woundball(20, 2000, n2=1999)
    lk_o, raw, st = check(g)
    assert st["cc_candidates"] > 256 and st["cc_fallback_pairs"] == 0
    assert lk_o[0] == 0 and raw[0] == 0.0


def test_cc_one_cta_search_halves_its_grid():
    """A row loop that zigzags across the whole intersection of the two loops'
    boxes: at the starting grid (16 x 16) its segments' entries exceed four per
    segment, so the grid halves (down to 2 x 2) before the binning; the result
    still equals the oracle's, decided by crossings."""
    n_zz = 128
    ys = np.linspace(-1, 1, n_zz)
    xs = np.where(np.arange(n_zz) % 2 == 0, -1.0, 1.0)
    zz = np.stack([xs, ys, 0.05 * np.sin(np.arange(n_zz))], 1)
    ret = np.stack([np.full(8, 1.6), np.linspace(1, -1, 8), np.zeros(8)], 1)   # return path
    a = np.concatenate([zz, ret], 0)
    t = np.arange(300) * 2 * np.pi / 300
    b = np.stack([0.2 + 0.9 * np.cos(t), 0.1 * np.sin(3 * t), 0.9 * np.sin(t)], 1)
    g = W.from_loops([a, b], pairs=[[0, 1]])
    for search in ("auto", "sweep"):
        lk_o, raw, st = check(g, cc_search=SEARCH[search])
        assert st["cc_fallback_pairs"] == 0 and raw[0] == lk_o[0] == -1
