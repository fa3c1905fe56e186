"""The identities behind the fast sweep's one-step cell angle, checked in FP64.

A cell of the direct sum (Eq. 4) is the parallelogram of vertex differences
a = l_j - k_i, b = a - s_i, c = a - s_i + s_j, d = a + s_j (a + c = b + d), and
its two triangle angles theta_1 = atan2(p, d_1), theta_2 = atan2(p, d_2) share
p = a.(s_j x s_i).  With the edge terms H_uv = |u||v| + u.v:

* for any triangle, D^2 + p^2 = 2 H_ab H_bc H_ca (D its Eq. 4 denominator);
* for the parallelogram, d_1 + d_2 = H_ac (|a| + |b| + |c| + |d|);

so |(d_1 + i p)(d_2 + i p)|^2 = 4 H_ab H_bc H_cd H_da H_ac^2 and
tan(theta_1 + theta_2) = (p S / 2) / sqrt(H_ab H_bc H_cd H_da - (p S / 2)^2)
with S = |a| + |b| + |c| + |d|, wherever d_1 d_2 > p^2.  The GPU's fast variant
sums that angle; these checks pin the algebra, independently of the oracle.
"""
import numpy as np


def H(u, v):
    return np.linalg.norm(u) * np.linalg.norm(v) + u @ v


def triangle_denominator(a, b, c):
    na, nb, nc = (np.linalg.norm(x) for x in (a, b, c))
    return na * nb * nc + (a @ b) * nc + (a @ c) * nb + (b @ c) * na


def test_triangle_identity():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a, b, c = rng.normal(size=(3, 3)) * rng.uniform(0.1, 10, size=(3, 1))
        p = a @ np.cross(b, c)
        D = triangle_denominator(a, b, c)
        rhs = 2 * H(a, b) * H(b, c) * H(c, a)
        assert abs(D * D + p * p - rhs) <= 1e-11 * rhs


def test_edge_terms_from_distances():
    """Law of cosines: for corners u, v joined by e = v - u,
    2 H_uv = (|u| + |v|)^2 - |e|^2 (the fast sweep forms every edge term so)."""
    rng = np.random.default_rng(4)
    for _ in range(2000):
        u, v = rng.normal(size=(2, 3)) * rng.uniform(0.1, 10, size=(2, 1))
        lhs = 2 * H(u, v)
        rhs = (np.linalg.norm(u) + np.linalg.norm(v)) ** 2 - np.linalg.norm(v - u) ** 2
        assert abs(lhs - rhs) <= 1e-12 * (np.linalg.norm(u) + np.linalg.norm(v)) ** 2


def test_parallelogram_cell_angle():
    rng = np.random.default_rng(2)
    checked = 0
    for _ in range(4000):
        a = rng.normal(size=3) * rng.uniform(0.2, 5)
        si = rng.normal(size=3) * rng.uniform(0.01, 1)
        sj = rng.normal(size=3) * rng.uniform(0.01, 1)
        b, c, d = a - si, a - si + sj, a + sj
        p = a @ np.cross(sj, si)
        d1 = triangle_denominator(a, b, c)
        d2 = triangle_denominator(c, d, a)
        S = sum(np.linalg.norm(x) for x in (a, b, c, d))
        assert abs((d1 + d2) - H(a, c) * S) <= 1e-12 * abs(d1 + d2) + 1e-15
        if d1 * d2 - p * p <= 0:
            continue
        P = H(a, b) * H(b, c) * H(c, d) * H(d, a)
        w = 0.5 * p * S
        angle = np.arctan(w / np.sqrt(P - w * w))
        assert abs(angle - (np.arctan2(p, d1) + np.arctan2(p, d2))) <= 1e-11
        checked += 1
    assert checked > 3000


def test_far_cells_always_qualify():
    """Every cell whose corners are all at least 4.5 segment lengths away (the
    bulk sweep's cells) has d_1 d_2 > p^2, i.e. a half solid angle below pi/2."""
    rng = np.random.default_rng(3)
    for _ in range(4000):
        L = 1.0
        si = rng.normal(size=3)
        si *= rng.uniform(0.01, L) / np.linalg.norm(si)
        sj = rng.normal(size=3)
        sj *= rng.uniform(0.01, L) / np.linalg.norm(sj)
        direction = rng.normal(size=3)
        a = direction / np.linalg.norm(direction) * rng.uniform(4.5 * L + 2 * L, 20 * L)
        b, c, d = a - si, a - si + sj, a + sj
        if min(np.linalg.norm(x) for x in (a, b, c, d)) < 4.5 * L:
            continue
        p = a @ np.cross(sj, si)
        assert triangle_denominator(a, b, c) * triangle_denominator(c, d, a) > p * p
