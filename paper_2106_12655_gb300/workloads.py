"""Seeded synthetic loop geometries and the host-side candidate-pair search.

This module draws inputs only; it holds none of the linking-number arithmetic
and is shared by the tests, the benchmark and the oracle-side checks.

Every generator returns a :class:`Geometry` in CSR form: ``vertices`` is an
``[N, 3]`` array (float32 or float64), ``offsets`` is ``int64[L+1]`` with loop
``l`` owning ``vertices[offsets[l]:offsets[l+1]]``.  Loops close implicitly:
the last vertex joins back to the first (Qu & James 2021, Sec. 3.4.2,
Algorithm 5 indexes ``l_{j+1}`` with wrap-around), so no vertex is repeated.

Shapes follow the paper's workloads (Sec. 4, Table 1 and Fig. "Large-Input
Stress Tests"): rings and chainmail sheets, knit-like stitch loops, torus links
and double-helix ribbons.  The paper's own models are not available; these
stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Geometry:
    vertices: np.ndarray
    offsets: np.ndarray
    pairs: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_loops(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def loop(self, i: int) -> np.ndarray:
        return self.vertices[self.offsets[i]:self.offsets[i + 1]]

    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)

    def segment_pairs(self, pairs=None) -> int:
        pr = self.pairs if pairs is None else np.asarray(pairs).reshape(-1, 2)
        n = self.sizes().astype(np.int64)
        return int(np.sum(n[pr[:, 0]] * n[pr[:, 1]]))


def from_loops(loops, dtype=np.float64, name="", pairs=None, meta=None) -> Geometry:
    sizes = [int(np.asarray(x).shape[0]) for x in loops]
    off = np.zeros(len(loops) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    v = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in loops], 0).astype(dtype))
    pr = np.zeros((0, 2), np.int32) if pairs is None else np.asarray(pairs, np.int32).reshape(-1, 2)
    return Geometry(v, off, pr, name, dict(meta or {}))


# ----------------------------------------------------------------------------- primitives

def circle(center, e1, e2, n, radius=1.0, phase=0.0) -> np.ndarray:
    t = phase + np.arange(n) * (2.0 * np.pi / n)
    c = np.asarray(center, np.float64)
    return c[None, :] + radius * (np.cos(t)[:, None] * np.asarray(e1, np.float64)[None, :]
                                  + np.sin(t)[:, None] * np.asarray(e2, np.float64)[None, :])


def _rot(axis: str, ang: float) -> np.ndarray:
    c, s = np.cos(ang), np.sin(ang)
    if axis == "x":
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    if axis == "y":
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


# ----------------------------------------------------------------------------- small closed forms

def hopf(n1=64, n2=64) -> Geometry:
    """Two unit circles threading each other (Hopf link, |lk| = 1)."""
    a = circle([0, 0, 0], [1, 0, 0], [0, 1, 0], n1)
    b = circle([1, 0, 0], [1, 0, 0], [0, 0, 1], n2)
    return from_loops([a, b], name="hopf", pairs=[[0, 1]])


def torus_knot_component(p, q, m, n, R=3.0, r=1.0) -> np.ndarray:
    """Component m (0 or 1) of the (2p,2q) torus link: longitude angle p*t + m*pi/q,
    meridian angle q*t, t in [0, 2pi) sampled at n points."""
    t = np.arange(n) * (2.0 * np.pi / n)
    ph = p * t + m * np.pi / q
    th = q * t
    rad = R + r * np.cos(th)
    return np.stack([rad * np.cos(ph), rad * np.sin(ph), r * np.sin(th)], 1)


def torus_link(p, q, n, R=3.0, r=1.0, dtype=np.float64, n2=None) -> Geometry:
    """(2p,2q) torus link: two (p,q) torus-knot components, |lk| = p*q."""
    a = torus_knot_component(p, q, 0, n, R, r)
    b = torus_knot_component(p, q, 1, n if n2 is None else n2, R, r)
    return from_loops([a, b], dtype=dtype, name=f"torus_link_{p}_{q}_{n}", pairs=[[0, 1]],
                      meta={"p": p, "q": q, "abs_lk": p * q})


def torus_periods(T, P, n1, n2, R=3.0, r_inner=0.4, r_outer=1.0) -> Geometry:
    """The paper's torus stress test shape (Fig. "Large-Input Stress Tests"): loop 1
    winds T times around the torus axis on an inner tube, loop 2 winds P times
    around the tube on an outer tube; |lk| = T*P."""
    t = np.arange(n1) * (2.0 * np.pi / n1)
    ph, th = T * t, t
    rad = R + r_inner * np.cos(th)
    a = np.stack([rad * np.cos(ph), rad * np.sin(ph), r_inner * np.sin(th)], 1)
    t = np.arange(n2) * (2.0 * np.pi / n2)
    ph, th = t, P * t
    rad = R + r_outer * np.cos(th)
    b = np.stack([rad * np.cos(ph), rad * np.sin(ph), r_outer * np.sin(th)], 1)
    return from_loops([a, b], name=f"torus_periods_{T}_{P}", pairs=[[0, 1]], meta={"abs_lk": T * P})


def double_helix_ribbon(twists, n, R=4.0, w=0.3) -> Geometry:
    """DNA-like double-helix ribbon (Fig. "Large-Input Stress Tests"): the two edges of
    a ribbon whose core is a planar circle of radius R, the edges rotating
    ``twists`` full turns about the core; |lk| = twists."""
    t = np.arange(n) * (2.0 * np.pi / n)
    core = np.stack([R * np.cos(t), R * np.sin(t), 0 * t], 1)
    nrm = np.stack([np.cos(t), np.sin(t), 0 * t], 1)
    bin_ = np.tile(np.array([0.0, 0.0, 1.0]), (n, 1))
    loops = []
    for m in range(2):
        ang = twists * t + m * np.pi
        loops.append(core + w * (np.cos(ang)[:, None] * nrm + np.sin(ang)[:, None] * bin_))
    return from_loops(loops, name=f"ribbon_{twists}", pairs=[[0, 1]], meta={"abs_lk": twists})


def _spherical_winding(nu, n, radius, tilt, R3) -> np.ndarray:
    """One woundball curve: a great circle of the given radius, tilted by ``tilt``
    off the polar axis so that it misses the poles, and turned one full
    revolution about the polar axis over ``nu`` passes.  It passes near the
    north pole ``nu`` times and closes after the last pass; the whole curve is
    then rotated by ``R3``."""
    t = np.arange(n) * (2.0 * np.pi * nu / n)
    g = np.stack([np.sin(t), -np.cos(t) * np.sin(tilt), np.cos(t) * np.cos(tilt)], 1)
    a = t / nu
    c, s = np.cos(a), np.sin(a)
    p = np.stack([c * g[:, 0] - s * g[:, 1], s * g[:, 0] + c * g[:, 1], g[:, 2]], 1)
    return radius * p @ R3.T


def woundball(nu, n, n2=None, R=1.0, ratio=0.5, seed=5) -> Geometry:
    """The paper's woundball stress test (Fig. "Large-Input Stress Tests"): two
    similar spherical curves on concentric spheres of radii R and ratio*R, each
    passing near the north pole ``nu`` times.  The inner curve lies in a ball
    that the outer sphere does not meet, so it can be shrunk to a point
    without crossing the outer curve: lk = 0, reached by a sum of many terms
    that cancel."""
    rng = np.random.default_rng(seed)
    a = _spherical_winding(nu, n, R, 0.05, np.eye(3))
    b = _spherical_winding(nu, n if n2 is None else n2, ratio * R, 0.08, random_rotation(rng))
    return from_loops([a, b], name=f"woundball_{nu}", pairs=[[0, 1]], meta={"abs_lk": 0})


def _rectangle(corners, nseg) -> np.ndarray:
    """Closed polyline through the four corners, ``nseg`` segments shared among
    the sides in proportion to their lengths (every corner is a vertex)."""
    corners = np.asarray(corners, np.float64)
    side = np.linalg.norm(np.roll(corners, -1, 0) - corners, axis=1)
    per = np.maximum(1, np.round(nseg * side / side.sum()).astype(int))
    per[np.argmax(per)] += nseg - per.sum()
    pts = []
    for k in range(4):
        u = np.arange(per[k])[:, None] / per[k]
        pts.append(corners[k] + u * (corners[(k + 1) % 4] - corners[k]))
    return np.concatenate(pts, 0)


def square_links(n, nseg, w=0.25, gap=1.0, sigma=1e-3, seed=6, dtype=np.float64) -> Geometry:
    """The paper's thick square link stress test (Fig. "Large-Input Stress
    Tests"): L = 2n long flat rectangles, n in the planes y = a*gap and n in the
    planes x = b*gap, woven so that every rectangle of one family threads every
    rectangle of the other exactly once: L^2/4 linked pairs, each |lk| = 1,
    all of one sign, and no linked pair within a family.  Rectangle a spans
    z in [-w, w]; rectangle b spans z in [0, 2w], so only its lower long side
    passes through rectangle a.  Loops are ordered a = 0..n-1, then b; the
    closest approach of two loops is w.  Seeded jitter (sigma*w) keeps the
    vertices in general position."""
    rng = np.random.default_rng(seed)
    lo, hi = -gap, n * gap
    loops = []
    for a in range(n):
        y = a * gap
        loops.append(_rectangle([[lo, y, -w], [hi, y, -w], [hi, y, w], [lo, y, w]], nseg))
    for b in range(n):
        x = b * gap + 0.5 * gap
        loops.append(_rectangle([[x, lo, 0.0], [x, lo, 2 * w], [x, hi, 2 * w], [x, hi, 0.0]], nseg))
    loops = [x + rng.normal(scale=sigma * w, size=x.shape) for x in loops]
    aa, bb = np.meshgrid(np.arange(n), np.arange(n, 2 * n), indexing="ij")
    pairs = np.stack([aa.ravel(), bb.ravel()], 1)
    return from_loops(loops, dtype=dtype, name=f"square_links_{n}", pairs=pairs, meta={"abs_lk": 1})


def whitehead(n1=200, n2=400, h=0.5, lift=0.3) -> Geometry:
    """Whitehead link as a reduced alternating 5-crossing diagram: loop 2 is a
    lemniscate (figure-eight) in the xy-plane whose self-crossing is lifted by
    +-``lift``; loop 1 is the unit circle, undulating as z = h*sin(2s) so that
    it passes alternately over and under the lemniscate at its four crossings.
    The two lobes are threaded in opposite senses, so lk = 0."""
    s = np.arange(n1) * (2.0 * np.pi / n1)
    a = np.stack([np.cos(s), np.sin(s), h * np.sin(2.0 * s)], 1)
    t = np.arange(n2) * (2.0 * np.pi / n2)
    b = np.stack([2.0 * np.sin(t), np.sin(2.0 * t), lift * np.cos(t)], 1)
    return from_loops([a, b], name="whitehead", pairs=[[0, 1]], meta={"abs_lk": 0})


# ----------------------------------------------------------------------------- paper-shaped workloads

def ring_chain(seed=1, n_rings=16, nseg=128, sigma=1e-3) -> Geometry:
    """16 unit rings of 128 segments centred at (1.5 i, 0, 0); odd rings rotated 90
    degrees about x so neighbours interlink; Gaussian jitter; FP64; all pairs."""
    rng = np.random.default_rng(seed)
    loops = []
    for i in range(n_rings):
        e1 = np.array([1.0, 0.0, 0.0])
        e2 = np.array([0.0, 1.0, 0.0]) if i % 2 == 0 else np.array([0.0, 0.0, 1.0])
        ring = circle([1.5 * i, 0.0, 0.0], e1, e2, nseg)
        loops.append(ring + rng.normal(scale=sigma, size=ring.shape))
    pairs = np.array([[a, b] for a in range(n_rings) for b in range(a + 1, n_rings)], np.int32)
    return from_loops(loops, np.float64, "ring_chain", pairs, {"seed": seed})


def _mail_frame(row, beta, gamma):
    """Ring axes of a 4-in-1 sheet: e1 along the wale (tilted by gamma out of the
    sheet), e2 along the course, tilted by +-beta on alternate rows."""
    s = 1.0 if row % 2 == 0 else -1.0
    e1 = np.array([0.0, np.cos(gamma), np.sin(gamma)])
    e2 = np.array([np.cos(beta), 0.0, s * np.sin(beta)])
    e2 = e2 - e1 * np.dot(e1, e2)
    return e1, e2 / np.linalg.norm(e2)


def chainmail(seed=2, rows=32, cols=64, nseg=256, sigma=0.02, dtype=np.float32,
              pitch=(1.5, 0.8), beta_deg=35.0, gamma_deg=20.0, nseg_per_ring=None) -> Geometry:
    """European 4-in-1 chainmail sheet: unit rings on a staggered rows x cols grid,
    alternate rows tilted +-beta, each interior ring linked with its four diagonal
    neighbours.  Centres and ring orientations are perturbed with N(0, sigma).
    Candidate pairs come from loop AABB overlap."""
    rng = np.random.default_rng(seed)
    P, Q = pitch
    beta, gamma = np.deg2rad(beta_deg), np.deg2rad(gamma_deg)
    loops = []
    for r in range(rows):
        e1, e2 = _mail_frame(r, beta, gamma)
        for c in range(cols):
            ctr = np.array([c * P + (r % 2) * P / 2.0, r * Q, 0.0]) + rng.normal(scale=sigma, size=3)
            rot = _rot("x", rng.normal(scale=sigma)) @ _rot("y", rng.normal(scale=sigma)) @ \
                _rot("z", rng.normal(scale=sigma))
            n = nseg if nseg_per_ring is None else int(nseg_per_ring[r * cols + c])
            loops.append(circle(ctr, rot @ e1, rot @ e2, n, phase=rng.uniform(0, 2 * np.pi)))
    g = from_loops(loops, dtype, "chainmail", None, {"seed": seed, "rows": rows, "cols": cols})
    g.pairs = aabb_candidates(g.vertices, g.offsets)
    return g


def knit_yarn(seed=3, rows=30, cols=20, min_seg=1000, max_seg=20000, dtype=np.float32,
              turns=24, helix=0.05, wave=0.04) -> Geometry:
    """Knit-yarn-like sheet: 600 closed stitch loops on a course/wale lattice.  Each
    loop is a tilted unit ring (the 4-in-1 lattice, so it interlocks with its row
    neighbours) carrying a helix of ``turns`` coils around the core plus a
    sinusoidal undulation out of its plane; each loop is sampled at a segment
    count drawn log-uniformly in [min_seg, max_seg]."""
    rng = np.random.default_rng(seed)
    P, Q = 1.5, 0.8
    beta, gamma = np.deg2rad(35.0), np.deg2rad(20.0)
    loops = []
    for r in range(rows):
        e1, e2 = _mail_frame(r, beta, gamma)
        nrm = np.cross(e1, e2)
        for c in range(cols):
            n = int(np.exp(rng.uniform(np.log(min_seg), np.log(max_seg))))
            ctr = np.array([c * P + (r % 2) * P / 2.0, r * Q, 0.0]) + rng.normal(scale=0.01, size=3)
            t = rng.uniform(0, 2 * np.pi) + np.arange(n) * (2.0 * np.pi / n)
            radial = np.cos(t)[:, None] * e1[None, :] + np.sin(t)[:, None] * e2[None, :]
            core = ctr[None, :] + radial
            coil = turns * t
            off = helix * (np.cos(coil)[:, None] * radial + np.sin(coil)[:, None] * nrm[None, :])
            off += wave * np.sin(6.0 * t)[:, None] * nrm[None, :]
            loops.append(core + off)
    g = from_loops(loops, dtype, "knit_yarn", None, {"seed": seed})
    g.pairs = aabb_candidates(g.vertices, g.offsets)
    return g


def serving_pile(seed, min_rings=500, max_rings=14000, min_seg=64, max_seg=256,
                 dtype=np.float32) -> Geometry:
    """One serving request: a jittered 4-in-1 chainmail pile whose ring count is drawn
    log-uniformly in [min_rings, max_rings] and whose per-ring segment counts are
    drawn uniformly in [min_seg, max_seg]."""
    rng = np.random.default_rng(seed)
    n_rings = int(np.exp(rng.uniform(np.log(min_rings), np.log(max_rings))))
    cols = max(4, int(np.sqrt(n_rings * 2)))
    rows = max(2, n_rings // cols)
    nseg = rng.integers(min_seg, max_seg + 1, size=rows * cols)
    g = chainmail(seed=int(rng.integers(1 << 30)), rows=rows, cols=cols, nseg=None, dtype=dtype,
                  nseg_per_ring=nseg)
    g.name = "serving_pile"
    return g


# ----------------------------------------------------------------------------- candidate search

def loop_aabbs(vertices, offsets):
    v = np.asarray(vertices, np.float64)
    off = np.asarray(offsets, np.int64)
    lo = np.minimum.reduceat(v, off[:-1], axis=0)
    hi = np.maximum.reduceat(v, off[:-1], axis=0)
    return lo, hi


def aabb_candidates(vertices, offsets, pad=0.0) -> np.ndarray:
    """All loop pairs (a < b) whose axis-aligned boxes overlap (the paper's potential
    link search, Sec. 3.2, done here as a sort-and-sweep on x on the host)."""
    lo, hi = loop_aabbs(vertices, offsets)
    lo = lo - pad
    hi = hi + pad
    order = np.argsort(lo[:, 0], kind="stable")
    out = []
    for pos, a in enumerate(order):
        xa = hi[a, 0]
        k = pos + 1
        cand = []
        while k < len(order) and lo[order[k], 0] <= xa:
            cand.append(order[k])
            k += 1
        if not cand:
            continue
        cand = np.asarray(cand)
        ok = np.all((lo[cand] <= hi[a]) & (hi[cand] >= lo[a]), axis=1)
        for b in cand[ok]:
            out.append((min(a, b), max(a, b)))
    if not out:
        return np.zeros((0, 2), np.int32)
    pr = np.unique(np.asarray(out, np.int64), axis=0)
    return pr.astype(np.int32)


def min_pair_distance(g: Geometry, pairs=None) -> np.ndarray:
    """Minimum vertex-vertex distance of each candidate pair (generator guard)."""
    from scipy.spatial import cKDTree

    pr = g.pairs if pairs is None else np.asarray(pairs).reshape(-1, 2)
    trees = {}
    out = np.zeros(pr.shape[0])
    for idx, (a, b) in enumerate(pr):
        if b not in trees:
            trees[b] = cKDTree(np.asarray(g.loop(b), np.float64))
        d, _ = trees[b].query(np.asarray(g.loop(a), np.float64))
        out[idx] = d.min()
    return out


def max_segment_length(g: Geometry) -> np.ndarray:
    v = np.asarray(g.vertices, np.float64)
    out = np.zeros(g.n_loops)
    for i in range(g.n_loops):
        x = g.loop(i).astype(np.float64)
        out[i] = np.linalg.norm(np.roll(x, -1, 0) - x, axis=1).max()
    return out
