"""Exact projected-crossing count of the linking number (test helper).

An independent way to the linking number (Qu & James 2021, Sec. 2.1,
"Counting Crossings"): project both closed polylines along a direction v,
find the proper crossings of their projections, and add the crossing signs.
Everything here is exact integer / rational arithmetic, so on tiny inputs this
is a brute-force pin for the FP64 direct-sum oracle.

Sign convention, derived from Eq. 1 (degree of the Gauss map, not from the
direct-sum formula): with sigma = sign(v . (t1 x t2)) at a crossing of segment
directions t1 (loop 1) and t2 (loop 2),

    lk = sum over crossings where loop 1 lies above loop 2 along v of sigma
       = - sum over crossings where loop 2 lies above loop 1 of sigma,

and the two one-sided counts must agree (checked here on every call).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


class Degenerate(Exception):
    """The projection is not regular (retry with another direction)."""


class Intersecting(Exception):
    """The two loops intersect in 3-D: the linking number is undefined."""


def to_integer_coords(*loops):
    """Scale float64 loops by one power of two so that every coordinate is an integer
    (exact: float64 values are dyadic rationals)."""
    arrs = [np.asarray(x, dtype=np.float64) for x in loops]
    max_exp = 0
    for a in arrs:
        for v in a.ravel():
            if v != 0.0:
                m, e = np.frexp(v)
                max_exp = max(max_exp, 53 - int(e))
    scale = 1 << max_exp
    out = []
    for a in arrs:
        out.append([[int(Fraction(float(c)) * scale) for c in row] for row in a])
    return out


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _orient(p, q, r):
    return (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0])


def _sgn(x):
    return (x > 0) - (x < 0)


def _boxes_touch(p1, p2, q1, q2):
    return not (max(p1[0], p2[0]) < min(q1[0], q2[0]) or max(q1[0], q2[0]) < min(p1[0], p2[0]) or
                max(p1[1], p2[1]) < min(q1[1], q2[1]) or max(q1[1], q2[1]) < min(p1[1], p2[1]))


def crossing_count(l, k, v):
    """Linking number of integer polylines l, k by crossings of the projection along
    the integer direction v.  Raises Degenerate or Intersecting."""
    v = tuple(int(x) for x in v)
    w = (1, 0, 0) if abs(v[0]) <= max(abs(v[1]), abs(v[2])) else (0, 1, 0)
    e1 = _cross(v, w)
    e2 = _cross(v, e1)
    if e1 == (0, 0, 0):
        raise Degenerate("bad direction")

    def proj(pts):
        return [(_dot(p, e1), _dot(p, e2), _dot(p, v)) for p in pts]

    L, K = proj(l), proj(k)
    nl, nk = len(l), len(k)
    over1 = over2 = 0
    for j in range(nl):
        P1, P2 = L[j], L[(j + 1) % nl]
        t1 = tuple(l[(j + 1) % nl][c] - l[j][c] for c in range(3))
        for i in range(nk):
            Q1, Q2 = K[i], K[(i + 1) % nk]
            o1, o2 = _orient(P1, P2, Q1), _orient(P1, P2, Q2)
            o3, o4 = _orient(Q1, Q2, P1), _orient(Q1, Q2, P2)
            if 0 in (o1, o2, o3, o4):
                if _boxes_touch(P1, P2, Q1, Q2):
                    raise Degenerate("vertex on a projected segment")
                continue
            if _sgn(o1) == _sgn(o2) or _sgn(o3) == _sgn(o4):
                continue
            t = Fraction(o3, o3 - o4)
            u = Fraction(o1, o1 - o2)
            h1 = P1[2] + t * (P2[2] - P1[2])
            h2 = Q1[2] + u * (Q2[2] - Q1[2])
            if h1 == h2:
                raise Intersecting("segments %d and %d meet" % (j, i))
            t2 = tuple(k[(i + 1) % nk][c] - k[i][c] for c in range(3))
            sigma = _sgn(_dot(v, _cross(t1, t2)))
            if sigma == 0:
                raise Degenerate("parallel crossing")
            if h1 > h2:
                over1 += sigma
            else:
                over2 += sigma
    if over1 != -over2:
        raise AssertionError("one-sided crossing counts disagree: %d vs %d" % (over1, -over2))
    return over1


def linking_number_exact(l, k, rng=None, tries=20):
    """Exact linking number of two float or integer polylines (retries degenerate
    projections with fresh random integer directions)."""
    rng = np.random.default_rng(0) if rng is None else rng
    la = np.asarray(l)
    ka = np.asarray(k)
    if np.issubdtype(la.dtype, np.integer) and np.issubdtype(ka.dtype, np.integer):
        li = [[int(c) for c in row] for row in la]
        ki = [[int(c) for c in row] for row in ka]
    else:
        li, ki = to_integer_coords(la, ka)
    for _ in range(tries):
        v = rng.integers(-7, 8, size=3)
        if not v.any():
            continue
        try:
            return crossing_count(li, ki, v)
        except Degenerate:
            continue
    raise Degenerate("no regular projection found")
