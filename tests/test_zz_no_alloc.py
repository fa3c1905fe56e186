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
