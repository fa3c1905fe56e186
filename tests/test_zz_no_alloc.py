"""The allocation-free verify (lk_verify_noalloc) against the regular one.

Callers that cannot allocate device memory when they verify (a no-allocation
simulation step, a process whose pool owns all device memory) use
lk_verify_noalloc, whose work buffers live in a static device array.  This
file is collected last on purpose: it must pass both alone in a fresh process
and after every other test.  Two calls in a row are compared with lk_verify on
the same inputs (linking numbers exact, raw sums within the 1e-6 tolerance of
the parity tests); the second call also checks that what the first left in the
shared array does not leak into the next result.
"""
import numpy as np
import pytest

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


def regular(g, pairs):
    n = pairs.shape[0]
    out = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
    ctx = lk.lk_create(g.vertices, g.offsets)
    try:
        lk.lk_verify(ctx, pairs, *out)
    finally:
        lk.lk_destroy(ctx)
    return out


def noalloc(g, pairs, on_device):
    n = pairs.shape[0]
    stream = torch.cuda.current_stream()
    if on_device:
        v = torch.from_numpy(np.ascontiguousarray(g.vertices)).cuda()
        lk_o = torch.zeros(n, dtype=torch.int32, device="cuda")
        raw = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = torch.zeros(n, dtype=torch.int32, device="cuda")
        lk.lk_verify_noalloc(v, g.offsets, pairs, lk_o, raw, st, stream)
        torch.cuda.synchronize()
        return lk_o.cpu().numpy(), raw.cpu().numpy(), st.cpu().numpy()
    out = np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.int32)
    lk.lk_verify_noalloc(g.vertices, g.offsets, pairs, *out, stream=stream)
    return out


def check_same(a, b):
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[0], b[0])
    ok = b[2] == 0
    assert np.max(np.abs(a[1][ok] - b[1][ok]), initial=0.0) <= RAW_TOL


def test_noalloc_matches_regular_verify_two_calls_in_a_row():
    chain = W.ring_chain()                                   # FP64 vertices, 120 pairs
    mail = W.chainmail(seed=9, rows=8, cols=16)              # FP32 vertices, 32,768 vertices
    ref_chain = regular(chain, chain.pairs)
    ref_mail = regular(mail, mail.pairs)
    # first call: the small FP64 chain from device memory; second call: a
    # larger FP32 sheet from host memory, reusing the same static array
    first = noalloc(chain, chain.pairs, on_device=True)
    second = noalloc(mail, mail.pairs, on_device=False)
    check_same(first, ref_chain)
    check_same(second, ref_mail)
    # and the chain again after the sheet left its contents behind
    third = noalloc(chain, chain.pairs[::-1].copy(), on_device=False)
    check_same(third, tuple(x[::-1] for x in ref_chain))


def test_noalloc_rejects_sizes_beyond_its_limits():
    g = W.chainmail(seed=9, rows=32, cols=64)                # 524,288 vertices > 262,144
    with pytest.raises(lk.LkError) as ei:
        noalloc(g, g.pairs[:10], on_device=False)
    assert ei.value.status == lk.LK_ERR_ARG
    assert "limit" in str(ei.value)


def stacked_rings(n_rings=1024, nseg=256, dr=0.01, dz=0.003):
    """Coaxial rings of radii 1 + k dr at heights k dz: no two link (lk = 0),
    and each ring lies within a few segment lengths of its ten nearest
    neighbours along its whole length, so most of each neighbour pair's
    32-row chunks are near enough for the careful pass."""
    loops = [W.circle([0.0, 0.0, k * dz], [1, 0, 0], [0, 1, 0], nseg, radius=1.0 + k * dr) for k in range(n_rings)]
    pairs = [(a, b) for a in range(n_rings) for b in range(a + 1, min(n_rings, a + 12))]
    return W.from_loops(loops, dtype=np.float32, pairs=pairs)


def test_noalloc_allocates_nothing_past_the_chunk_list():
    """A (2,3) torus link of 2 x 65,536 segments: 131,072 work items and about
    10^6 32-row chunks, far more than the 65,536 entries of the static chunk
    list.  The call must size its lists to the static array (before this was
    fixed it asked for a larger list and reallocated it), match the closed
    form -6 and lk_verify, and leave the device's free memory unchanged."""
    g = W.torus_link(2, 3, 65_536, dtype=np.float32)
    ref = regular(g, g.pairs)
    first = noalloc(g, g.pairs, on_device=False)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    second = noalloc(g, g.pairs, on_device=False)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for out in (first, second):
        check_same(out, ref)
        assert out[2][0] == lk.LK_OK and out[0][0] == -6
        assert abs(out[1][0] + 6.0) <= RAW_TOL


def test_noalloc_chunk_list_overflow_hands_whole_items_over():
    """Near chunks beyond the static chunk list: the call hands whole work
    items to the careful pass instead.  Every pair of coaxial rings has lk = 0;
    the raw sums match lk_verify (whose list is large enough) and a seeded
    sample of them the FP64 oracle."""
    from oracle import oracle as O

    g = stacked_rings()
    assert g.pairs.shape[0] <= 16_384 and g.vertices.shape[0] <= 262_144
    ref = regular(g, g.pairs)
    out = noalloc(g, g.pairs, on_device=False)
    check_same(out, ref)
    assert np.all(out[2] == lk.LK_OK) and np.all(out[0] == 0)
    assert np.max(np.abs(out[1])) <= RAW_TOL
    pick = np.random.default_rng(4).choice(g.pairs.shape[0], 64, replace=False)
    want = O.link_pairs(g.vertices, g.offsets, g.pairs[pick])
    assert np.max(np.abs(out[1][pick] - want)) <= RAW_TOL
