"""Pins for the FP64 direct-sum oracle against facts fixed outside it.

Each pin is independent of the oracle's own formula: Gauss-Legendre quadrature
of Eq. 1 over one segment pair, exact integer crossing counts (Sec. 2.1,
"Counting Crossings"), the paper's printed linking numbers and textbook closed
forms, symmetries of Eq. 1, integrality of the polyline sum (Eq. 3) and
convergence of the midpoint rule (Eq. 2).  ``test_pins_catch_planted_mistakes``
recompiles the oracle with typical mistakes planted in its source and checks
that at least one pin fails for each.
"""
import json
import os

import numpy as np
import pytest

from crossings import linking_number_exact
from oracle import oracle as O
from paper_2106_12655_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
FOUR_PI = 4.0 * np.pi


# ----------------------------------------------------------------------------- independent references

def gauss_legendre_term(lj, lj1, ki, ki1, n=24):
    """(1/4pi) double integral of Eq. 1 over two straight segments, tensor GL rule."""
    x, w = np.polynomial.legendre.leggauss(n)
    s = 0.5 * (x + 1.0)
    w = 0.5 * w
    sj = lj1 - lj
    si = ki1 - ki
    r1 = lj[None, :] + s[:, None] * sj[None, :]
    r2 = ki[None, :] + s[:, None] * si[None, :]
    diff = r1[:, None, :] - r2[None, :, :]
    num = diff @ np.cross(sj, si)
    den = np.linalg.norm(diff, axis=2) ** 3
    return float(np.einsum("a,b,ab->", w, w, num / den) / FOUR_PI)


def midpoint_sum(l, k, m):
    """Eq. 2 on the polylines with every segment split into m equal pieces."""
    def refine(x):
        nxt = np.roll(x, -1, 0)
        f = (np.arange(m) / m)[None, :, None]
        return (x[:, None, :] + f * (nxt - x)[:, None, :]).reshape(-1, 3)

    a, b = refine(l), refine(k)
    ra = 0.5 * (a + np.roll(a, -1, 0))
    sa = np.roll(a, -1, 0) - a
    rb = 0.5 * (b + np.roll(b, -1, 0))
    sb = np.roll(b, -1, 0) - b
    total = 0.0
    for c0 in range(0, ra.shape[0], 256):
        d = ra[c0:c0 + 256, None, :] - rb[None, :, :]
        cr = np.cross(sa[c0:c0 + 256, None, :], sb[None, :, :])
        total += np.sum(np.einsum("abk,abk->ab", d, cr) / np.linalg.norm(d, axis=2) ** 3)
    return total / FOUR_PI


def separated_segment_pairs(rng, n):
    out = []
    while len(out) < n:
        lj = rng.normal(size=3)
        lj1 = lj + rng.normal(size=3)
        direction = rng.normal(size=3)
        direction /= np.linalg.norm(direction)
        ki = lj + direction * rng.uniform(3.0, 6.0)
        ki1 = ki + rng.normal(size=3)
        out.append((lj, lj1, ki, ki1))
    return out


def random_integer_polygons(rng, n_cases, lo=4, hi=30, box=40):
    cases = []
    for _ in range(n_cases):
        n1, n2 = rng.integers(lo, hi, 2)
        cases.append((rng.integers(-box, box + 1, (n1, 3)), rng.integers(-box, box + 1, (n2, 3))))
    return cases


# ----------------------------------------------------------------------------- pins (take a library)

def pin_quadrature(lib, n=120, seed=11):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for lj, lj1, ki, ki1 in separated_segment_pairs(rng, n):
        worst = max(worst, abs(O.term(lj, lj1, ki, ki1, lib=lib) - gauss_legendre_term(lj, lj1, ki, ki1)))
    return worst <= 1e-12, worst


def pin_exact_crossings(lib, n=150, seed=5):
    rng = np.random.default_rng(seed)
    bad = []
    for l, k in random_integer_polygons(rng, n):
        try:
            cc = linking_number_exact(l, k, rng)
        except Exception:
            continue
        raw = O.link(l.astype(np.float64), k.astype(np.float64), threads=1, lib=lib)
        if not (abs(raw - cc) < 1e-8):
            bad.append((cc, raw))
    return not bad, bad[:3]


def pin_closed_forms(lib):
    with open(os.path.join(HERE, "golden", "closed_forms.json")) as f:
        cases = json.load(f)["cases"]
    bad = []
    for c in cases:
        g = getattr(W, c["fn"])(*c["args"])
        a, b = c.get("pair", [0, 1])
        raw = O.link(g.loop(a), g.loop(b), lib=lib)
        if abs(abs(raw) - c["abs_lk"]) > 1e-8:
            bad.append((c["name"], raw))
    return not bad, bad


PINS = [pin_quadrature, pin_exact_crossings, pin_closed_forms]


# ----------------------------------------------------------------------------- tests of the shipped oracle

def test_term_matches_gauss_legendre_quadrature_of_eq1():
    ok, worst = pin_quadrature(None, n=300)
    assert ok, worst


def test_random_polygons_match_exact_crossing_count():
    ok, bad = pin_exact_crossings(None, n=400)
    assert ok, bad


def test_closed_forms_golden():
    ok, bad = pin_closed_forms(None)
    assert ok, bad


def test_closed_form_signs_match_crossing_count():
    rng = np.random.default_rng(1)
    for g in [W.hopf(24, 30), W.torus_link(2, 3, 150), W.double_helix_ribbon(4, 160), W.torus_periods(2, 3, 90, 90),
              W.whitehead(50, 70), W.woundball(6, 300)]:
        cc = linking_number_exact(g.loop(0), g.loop(1), rng)
        raw = O.link(g.loop(0), g.loop(1))
        assert abs(raw - cc) < 1e-9, (g.name, raw, cc)


def test_square_links_exactly_the_cross_family_pairs_link():
    """Thick square links (Fig. "Large-Input Stress Tests"): every pair of
    rectangles from different families links once, with one sign, and no two
    of one family link; the exact crossing count fixes each value."""
    rng = np.random.default_rng(2)
    g = W.square_links(3, 40)
    for a in range(g.n_loops):
        for b in range(a + 1, g.n_loops):
            cc = linking_number_exact(g.loop(a), g.loop(b), rng)
            raw = O.link(g.loop(a), g.loop(b))
            assert abs(raw - cc) < 1e-9, (a, b, raw, cc)
            assert cc == (1 if (a < 3) != (b < 3) else 0), (a, b, cc)
    # the boxes of one family are disjoint, so the box search keeps exactly the linked pairs
    assert np.array_equal(W.aabb_candidates(g.vertices, g.offsets), g.pairs)


def test_term_bounds_and_segment_reversal_antisymmetry():
    rng = np.random.default_rng(3)
    for _ in range(500):
        lj, lj1, ki, ki1 = (rng.normal(size=3) for _ in range(4))
        t = O.term(lj, lj1, ki, ki1)
        assert abs(t) <= 0.5 + 1e-15
        assert abs(O.term(lj1, lj, ki, ki1) + t) <= 1e-14
        assert abs(O.term(lj, lj1, ki1, ki) + t) <= 1e-14
        # exchanging the roles of the two segments leaves Eq. 1 unchanged
        assert abs(O.term(ki, ki1, lj, lj1) - t) <= 1e-14


def test_polyline_sum_is_an_integer():
    rng = np.random.default_rng(8)
    worst = 0.0
    for l, k in random_integer_polygons(rng, 200, lo=20, hi=60):
        raw = O.link(l.astype(float) * 0.37, k.astype(float) * 0.37)
        worst = max(worst, abs(raw - np.round(raw)))
    assert worst < 1e-9, worst


def test_invariants():
    rng = np.random.default_rng(4)
    g = W.torus_link(3, 4, 700, n2=650)
    l, k = g.loop(0), g.loop(1)
    base = O.link(l, k)
    assert abs(abs(base) - 12) < 1e-9
    assert abs(O.link(l[::-1], k) + base) < 1e-9                       # orientation reversal
    assert abs(O.link(l, k[::-1]) + base) < 1e-9
    mir = np.array([1.0, 1.0, -1.0])
    assert abs(O.link(l * mir, k * mir) + base) < 1e-9                # mirror image
    assert abs(O.link(k, l) - base) < 1e-9                             # role swap
    R = W.random_rotation(rng)
    t = rng.normal(size=3) * 10
    assert abs(O.link(l @ R.T + t, k @ R.T + t) - base) < 1e-9         # rigid motion
    assert abs(O.link(l * 1e3, k * 1e3) - base) < 1e-9                 # uniform scale
    assert abs(O.link(np.roll(l, 17, 0), np.roll(k, -5, 0)) - base) < 1e-9   # start vertex
    mid = 0.5 * (l + np.roll(l, -1, 0))
    sub = np.empty((2 * l.shape[0], 3))
    sub[0::2], sub[1::2] = l, mid
    assert abs(O.link(sub, k) - base) < 1e-9                           # vertex insertion


def test_ring_chain_neighbours_link_once_others_zero():
    g = W.ring_chain()
    raw = O.link_pairs(g.vertices, g.offsets, g.pairs)
    lk = O.round_lk(raw)
    for (a, b), v in zip(g.pairs, lk):
        assert abs(v) == (1 if b == a + 1 else 0), (a, b, v)
    assert np.max(np.abs(raw - lk)) < 1e-9


def test_midpoint_rule_eq2_converges_to_direct_sum():
    g = W.torus_link(2, 3, 120)
    exact = O.link(g.loop(0), g.loop(1))
    errs = [abs(midpoint_sum(g.loop(0), g.loop(1), m) - exact) for m in (1, 2, 4, 8)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0] / 20.0, errs


def test_fixed_order_sum_is_thread_count_independent():
    g = W.torus_link(2, 3, 2000, n2=1900)
    ref = O.link(g.loop(0), g.loop(1), threads=1)
    for th in (2, 3, 8):
        assert O.link(g.loop(0), g.loop(1), threads=th) == ref
    two = W.from_loops([g.loop(0), g.loop(1)])
    assert O.link_pairs(two.vertices, two.offsets, [[0, 1]], threads=4)[0] == ref


def test_blocks_and_rows_partition_the_double_sum():
    g = W.torus_link(2, 3, 300, n2=257)
    l, k = g.loop(0), g.loop(1)
    whole = O.link(l, k)
    parts = sum(O.block(l, k, j0, min(j0 + 100, 300), i0, min(i0 + 64, 257))
                for j0 in range(0, 300, 100) for i0 in range(0, 257, 64))
    assert abs(parts - whole) < 1e-12
    rows = O.link_rows(l, k, np.arange(257))
    assert abs(rows.sum() - whole) < 1e-12


def test_invalid_arguments_raise():
    with pytest.raises(ValueError):
        O.link(np.zeros((2, 3)), np.ones((5, 3)))
    g = W.hopf()
    with pytest.raises(ValueError):
        O.link_pairs(g.vertices, g.offsets, [[0, 0]])
    with pytest.raises(ValueError):
        O.link_pairs(g.vertices, g.offsets, [[0, 2]])


MUTATIONS = {
    "dropped_term_in_first_denominator": ("+ dot3(b, c) * na;", ";"),
    "wrong_sign_second_triple_product": ("double p2 = dot3(c, t);", "double p2 = -dot3(c, t);"),
    "wrong_vertex_index_for_b": ("sub3(lj, ki1, b);", "sub3(lj, ki, b);"),
    "transposed_cross_operands": ("cross3(b, c, t);", "cross3(c, b, t);"),
    "wrong_norm_in_second_denominator": ("dot3(a, c) * nd", "dot3(a, c) * nb"),
    "closing_segment_dropped": ("k + 3 * ((i + 1) % nk)", "k + 3 * (i + 1 < nk ? i + 1 : i)"),
    "half_normalisation": ("/ LKO_TWO_PI;", "/ (2.0 * LKO_TWO_PI);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(name, tmp_path):
    old, new = MUTATIONS[name]
    src = O.source_text()
    assert src.count(old) >= 1, name
    lib = O.load_library(O.compile_source(src.replace(old, new), str(tmp_path / ("m_%s.so" % name))))
    failures = [p.__name__ for p in PINS if not p(lib)[0]]
    assert failures, "no pin caught the planted mistake %r" % name
