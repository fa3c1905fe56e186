"""Pins of the oracle's potential link search (Sec. 3.2, Algorithm 2): the
plain all-pairs box-overlap definition in oracle/lk_oracle.c.

Pinned against what the paper and geometry fix: every pair of loops with a
nonzero linking number (by the direct-sum oracle) must be a candidate; boxes
that touch on a face, edge or corner overlap (closed boxes) and boxes one ulp
apart on any single axis do not; an independent sweep-and-prune over sorted
intervals gives the same set; relabelling the loops relabels the pairs.
Planted mistakes in the C source must each fail one of these pins.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_12655_gb300 import workloads as W


def tri(lo, hi):
    """A closed 3-vertex loop whose bounding box is exactly [lo, hi]."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    return np.array([lo, [hi[0], lo[1], hi[2]], hi])


def as_geometry(loops):
    return W.from_loops(loops, dtype=np.float64)


def pairs_set(p):
    return {(int(a), int(b)) for a, b in np.asarray(p).reshape(-1, 2)}


def sweep_and_prune(vertices, offsets):
    """Independent method: sort boxes by low x, sweep an active list."""
    v = np.asarray(vertices, float)
    L = len(offsets) - 1
    lo = np.array([v[offsets[i]:offsets[i + 1]].min(0) for i in range(L)])
    hi = np.array([v[offsets[i]:offsets[i + 1]].max(0) for i in range(L)])
    order = sorted(range(L), key=lambda i: (lo[i, 0], i))
    active, out = [], set()
    for i in order:
        active = [j for j in active if hi[j, 0] >= lo[i, 0]]
        for j in active:
            if all(lo[i, a] <= hi[j, a] and lo[j, a] <= hi[i, a] for a in (1, 2)):
                out.add((min(i, j), max(i, j)))
        active.append(i)
    return out


# ----------------------------------------------------------------------------- pins
# Each pin takes the oracle library and returns (ok, detail).

def pin_linked_pairs_are_candidates(lib):
    g = W.chainmail(rows=4, cols=5, nseg=48, sigma=0.02, dtype=np.float64)
    all_pairs = np.array(list(itertools.combinations(range(g.n_loops), 2)), np.int32)
    raw = O.link_pairs(g.vertices, g.offsets, all_pairs)
    linked = {tuple(p) for p, r in zip(all_pairs.tolist(), raw) if abs(round(r)) > 0}
    cand = pairs_set(O.candidates(g.vertices, g.offsets, lib=lib))
    return len(linked) > 10 and linked <= cand, (len(linked), len(linked - cand))


def pin_touching_and_separated_boxes(lib):
    base = ([0.0, 0.0, 0.0], [1.0, 1.0, 1.0])
    ok = True
    detail = []
    for axis in range(3):
        for case in ("face", "gap"):
            lo2, hi2 = np.array([0.2, 0.2, 0.2]), np.array([0.8, 0.8, 0.8])
            lo2[axis], hi2[axis] = 1.0, 2.0                  # touches box 1 at its upper face
            if case == "gap":
                lo2[axis] = np.nextafter(1.0, 2.0)           # one ulp apart on this axis only
            for swap in (False, True):
                loops = [tri(*base), tri(lo2, hi2)]
                if swap:
                    loops = loops[::-1]
                g = as_geometry(loops)
                got = pairs_set(O.candidates(g.vertices, g.offsets, lib=lib))
                want = {(0, 1)} if case == "face" else set()
                ok &= got == want
                detail.append((axis, case, swap, got == want))
    # edge and corner contact
    for lo2 in ([1.0, 1.0, 0.3], [1.0, 1.0, 1.0]):
        g = as_geometry([tri(*base), tri(lo2, [2.0, 2.0, 2.0])])
        ok &= pairs_set(O.candidates(g.vertices, g.offsets, lib=lib)) == {(0, 1)}
    return ok, detail


def pin_sweep_and_prune_agrees(lib):
    rng = np.random.default_rng(3)
    loops = []
    for _ in range(60):
        lo = rng.integers(0, 8, size=3).astype(float) / 4.0   # coarse grid: many exact ties
        hi = lo + rng.integers(0, 4, size=3).astype(float) / 4.0
        loops.append(tri(lo, hi))
    g = as_geometry(loops)
    got = O.candidates(g.vertices, g.offsets, lib=lib)
    ordered = all(tuple(a) < tuple(b) for a, b in zip(got[:-1], got[1:])) and bool(np.all(got[:, 0] < got[:, 1]))
    return pairs_set(got) == sweep_and_prune(g.vertices, g.offsets) and ordered, len(got)


def pin_relabelling(lib):
    g = W.chainmail(rows=3, cols=5, nseg=32, dtype=np.float64)
    L = g.n_loops
    perm = np.random.default_rng(4).permutation(L)
    loops = [g.vertices[g.offsets[i]:g.offsets[i + 1]] for i in range(L)]
    h = as_geometry([loops[p] for p in perm])                # new loop k is old loop perm[k]
    a = pairs_set(O.candidates(g.vertices, g.offsets, lib=lib))
    b = {tuple(sorted((int(perm[i]), int(perm[j])))) for i, j in pairs_set(O.candidates(h.vertices, h.offsets, lib=lib))}
    return a == b and len(a) > 0, len(a)


PINS = [pin_linked_pairs_are_candidates, pin_touching_and_separated_boxes, pin_sweep_and_prune_agrees,
        pin_relabelling]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_oracle_candidates_pins(pin):
    ok, detail = pin(O._load())
    assert ok, detail


def test_degenerate_inputs():
    g = as_geometry([tri([0, 0, 0], [1, 1, 1])])
    assert O.candidates(g.vertices, g.offsets).shape == (0, 2)
    # identical boxes overlap; a loop is never paired with itself
    g = as_geometry([tri([0, 0, 0], [1, 1, 1])] * 3)
    assert pairs_set(O.candidates(g.vertices, g.offsets)) == {(0, 1), (0, 2), (1, 2)}


PLS_MUTATIONS = {
    "strict_overlap_test": ("bi[a] <= bj[3 + a] && bj[a] <= bi[3 + a]", "bi[a] < bj[3 + a] && bj[a] < bi[3 + a]"),
    "z_axis_dropped": ("for (int a = 0; a < 3; ++a)\n                if (!(bi[a]", "for (int a = 0; a < 2; ++a)\n                if (!(bi[a]"),
    "one_sided_test": ("bi[a] <= bj[3 + a] && bj[a] <= bi[3 + a]", "bi[a] <= bj[3 + a]"),
    "low_end_from_first_vertex_only": ("if (v[3 * q + a] < lo[a]) lo[a] = v[3 * q + a];", "if (q == offsets[l]) lo[a] = v[3 * q + a];"),
    "last_loop_skipped": ("for (int64_t j = i + 1; j < nloops; ++j)", "for (int64_t j = i + 1; j < nloops - 1; ++j)"),
}


@pytest.mark.parametrize("name", sorted(PLS_MUTATIONS))
def test_pls_pins_catch_planted_mistakes(name, tmp_path):
    old, new = PLS_MUTATIONS[name]
    src = O.source_text()
    assert src.count(old) == 1, name
    lib = O.load_library(O.compile_source(src.replace(old, new), str(tmp_path / ("p_%s.so" % name))))
    failures = [p.__name__ for p in PINS if not p(lib)[0]]
    assert failures, "no pin caught the planted mistake %r" % name
