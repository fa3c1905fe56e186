/*
 * Oracle for the linking-number direct sum — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU evaluation of the Gauss linking number of two closed
 * polylines by direct summation of the closed-form segment-pair term
 * (Qu & James 2021, Sec. 2.1 "Direct Summation Methods", Eq. 3 and Eq. 4;
 * Sec. 3.4.2, Algorithm 5).  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file; the product
 * path (the CUDA library) never calls it and shares no code with it.
 *
 * Conventions (readings of the paper, Sec. 3.4.2 / Algorithm 5):
 *   - loop 1 has vertices l_j, j = 0..Nl-1; loop 2 has vertices k_i,
 *     i = 0..Nk-1; indices wrap (l_Nl = l_0, k_Nk = k_0): vertex lists do not
 *     repeat their first vertex.
 *   - a = l_j - k_i, b = l_j - k_{i+1}, c = l_{j+1} - k_{i+1},
 *     d = l_{j+1} - k_i (Eq. 4).
 *   - both triple products a.(b x c) and c.(d x a) are formed as written in
 *     Eq. 4 (the paper notes they are equal in exact arithmetic, Sec. 3.4.2);
 *     the two arctangents are std atan2 calls (Eq. 4: atan(y/x) = atan2(y,x)).
 *   - the double sum is taken in a fixed order: i outer, j inner, Neumaier
 *     compensated, in fixed blocks of LKO_ROWS_PER_BLOCK values of i whose
 *     compensated block sums are then combined in block order.  The result is
 *     therefore independent of the thread count.
 *
 * Parity: pinned by tests/test_oracle_pins.py (Gauss-Legendre quadrature of
 * Eq. 1 per segment pair, exact integer crossing counts, closed forms,
 * invariants, integrality of the polyline sum, midpoint convergence of Eq. 2).
 * The potential link search (lko_candidates) is pinned by
 * tests/test_oracle_pls.py (linked pairs are candidates, touching and
 * one-ulp-separated boxes on each axis, an independent sweep-and-prune,
 * permutation covariance).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LKO_ROWS_PER_BLOCK 64

static const double LKO_TWO_PI = 6.283185307179586476925286766559;

typedef struct { double s, c; } lko_acc; /* Neumaier running sum */

static void acc_add(lko_acc* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double acc_value(const lko_acc* a) { return a->s + a->c; }

static void sub3(const double* p, const double* q, double* r) {
    r[0] = p[0] - q[0]; r[1] = p[1] - q[1]; r[2] = p[2] - q[2];
}
static double dot3(const double* p, const double* q) {
    return p[0] * q[0] + p[1] * q[1] + p[2] * q[2];
}
static void cross3(const double* p, const double* q, double* r) {
    r[0] = p[1] * q[2] - p[2] * q[1];
    r[1] = p[2] * q[0] - p[0] * q[2];
    r[2] = p[0] * q[1] - p[1] * q[0];
}
static double norm3(const double* p) { return sqrt(dot3(p, p)); }

/* Eq. 4: the contribution lambda_ji of segment j of loop 1 (l_j -> l_{j+1})
 * and segment i of loop 2 (k_i -> k_{i+1}). */
double lko_term(const double* lj, const double* lj1, const double* ki, const double* ki1) {
    double a[3], b[3], c[3], d[3], t[3];
    sub3(lj, ki, a);
    sub3(lj, ki1, b);
    sub3(lj1, ki1, c);
    sub3(lj1, ki, d);
    double na = norm3(a), nb = norm3(b), nc = norm3(c), nd = norm3(d);
    cross3(b, c, t);
    double p1 = dot3(a, t);                           /* a . (b x c) */
    cross3(d, a, t);
    double p2 = dot3(c, t);                           /* c . (d x a) */
    double den1 = na * nb * nc + dot3(a, b) * nc + dot3(c, a) * nb + dot3(b, c) * na;
    double den2 = nc * nd * na + dot3(c, d) * na + dot3(a, c) * nd + dot3(d, a) * nc;
    return (atan2(p1, den1) + atan2(p2, den2)) / LKO_TWO_PI;
}

/* Sum over j of lambda_ji for one row i, j in [j0, j1). */
static void row_sum(const double* l, int64_t nl, const double* k, int64_t nk, int64_t i,
                    int64_t j0, int64_t j1, lko_acc* acc) {
    const double* ki = k + 3 * i;
    const double* ki1 = k + 3 * ((i + 1) % nk);
    for (int64_t j = j0; j < j1; ++j) {
        const double* lj = l + 3 * j;
        const double* lj1 = l + 3 * ((j + 1) % nl);
        acc_add(acc, lko_term(lj, lj1, ki, ki1));
    }
}

static int valid_loop(int64_t n) { return n >= 3; }

/* Sum of lambda_ji over j in [j0,j1) and i in [i0,i1): a sub-rectangle of the
 * double sum of Sec. 3.4.2 (the whole pair when the ranges are complete). */
int lko_block(const double* l, int64_t nl, const double* k, int64_t nk, int64_t j0, int64_t j1,
              int64_t i0, int64_t i1, int nthreads, double* out) {
    if (!l || !k || !out || !valid_loop(nl) || !valid_loop(nk)) return 1;
    if (j0 < 0 || j1 > nl || j0 > j1 || i0 < 0 || i1 > nk || i0 > i1) return 1;
    int64_t nrows = i1 - i0;
    int64_t nblocks = (nrows + LKO_ROWS_PER_BLOCK - 1) / LKO_ROWS_PER_BLOCK;
    lko_acc* blocks = (lko_acc*)calloc((size_t)(nblocks > 0 ? nblocks : 1), sizeof(lko_acc));
    if (!blocks) return 2;
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t bidx = 0; bidx < nblocks; ++bidx) {
        lko_acc acc = {0.0, 0.0};
        int64_t r0 = i0 + bidx * LKO_ROWS_PER_BLOCK;
        int64_t r1 = r0 + LKO_ROWS_PER_BLOCK < i1 ? r0 + LKO_ROWS_PER_BLOCK : i1;
        for (int64_t i = r0; i < r1; ++i) row_sum(l, nl, k, nk, i, j0, j1, &acc);
        blocks[bidx] = acc;
    }
    lko_acc total = {0.0, 0.0};
    for (int64_t bidx = 0; bidx < nblocks; ++bidx) {
        acc_add(&total, blocks[bidx].s);
        acc_add(&total, blocks[bidx].c);
    }
    *out = acc_value(&total);
    free(blocks);
    return 0;
}

/* lambda(gamma1, gamma2) = sum_i sum_j lambda_ji (Eq. 3, Sec. 3.4.2). */
int lko_link(const double* l, int64_t nl, const double* k, int64_t nk, int nthreads, double* raw) {
    return lko_block(l, nl, k, nk, 0, nl, 0, nk, nthreads, raw);
}

/* Per-row sums: out[r] = sum_j lambda_{j, rows[r]} (used to sample huge pairs). */
int lko_link_rows(const double* l, int64_t nl, const double* k, int64_t nk, const int64_t* rows,
                  int64_t nrows, int nthreads, double* out) {
    if (!l || !k || !rows || !out || !valid_loop(nl) || !valid_loop(nk)) return 1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= nk) return 1;
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t r = 0; r < nrows; ++r) {
        lko_acc acc = {0.0, 0.0};
        row_sum(l, nl, k, nk, rows[r], 0, nl, &acc);
        out[r] = acc_value(&acc);
    }
    return 0;
}

/* Linking numbers of many loop pairs of one CSR geometry (Algorithm 1: loop
 * over the candidate pairs; each pair is summed serially in the fixed order
 * above, pairs run in parallel).  pairs[2p] is gamma1 (l), pairs[2p+1] is
 * gamma2 (k).  Returns 0 on success, 1 on a bad argument. */
int lko_link_pairs(const double* v, const int64_t* offsets, int64_t nloops, const int32_t* pairs,
                   int64_t npairs, int nthreads, double* raw) {
    if (!v || !offsets || !pairs || !raw || nloops <= 0) return 1;
    for (int64_t p = 0; p < npairs; ++p) {
        int32_t a = pairs[2 * p], b = pairs[2 * p + 1];
        if (a < 0 || b < 0 || a >= nloops || b >= nloops || a == b) return 1;
        if (!valid_loop(offsets[a + 1] - offsets[a]) || !valid_loop(offsets[b + 1] - offsets[b]))
            return 1;
    }
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t p = 0; p < npairs; ++p) {
        int32_t a = pairs[2 * p], b = pairs[2 * p + 1];
        const double* l = v + 3 * offsets[a];
        const double* k = v + 3 * offsets[b];
        int64_t nl = offsets[a + 1] - offsets[a], nk = offsets[b + 1] - offsets[b];
        lko_acc acc = {0.0, 0.0};
        lko_acc blk = {0.0, 0.0};
        for (int64_t i = 0; i < nk; ++i) {
            row_sum(l, nl, k, nk, i, 0, nl, &blk);
            if ((i + 1) % LKO_ROWS_PER_BLOCK == 0 || i + 1 == nk) {
                acc_add(&acc, blk.s);
                acc_add(&acc, blk.c);
                blk.s = blk.c = 0.0;
            }
        }
        raw[p] = acc_value(&acc);
    }
    return 0;
}

/* Potential link search (Sec. 3.2, Algorithm 2) as its plain definition: the
 * pairs (i, j), i < j, of loops whose axis-aligned bounding boxes overlap.
 * A loop's box is the componentwise min and max of its vertices; two closed
 * boxes overlap when, on each of the three axes, each box's low end is at
 * most the other's high end.  Pairs are listed in (i, j) order; the first
 * min(n, capacity) are written to pairs_out and n is returned in *n_out. */
int lko_candidates(const double* v, const int64_t* offsets, int64_t nloops, int32_t* pairs_out,
                   int64_t capacity, int64_t* n_out) {
    if (!v || !offsets || !n_out || nloops < 0 || capacity < 0 || (capacity > 0 && !pairs_out)) return 1;
    double* box = (double*)malloc((size_t)(nloops > 0 ? nloops : 1) * 6 * sizeof(double));
    if (!box) return 2;
    for (int64_t l = 0; l < nloops; ++l) {
        double* lo = box + 6 * l;
        double* hi = lo + 3;
        for (int a = 0; a < 3; ++a) {
            lo[a] = INFINITY;
            hi[a] = -INFINITY;
        }
        for (int64_t q = offsets[l]; q < offsets[l + 1]; ++q)
            for (int a = 0; a < 3; ++a) {
                if (v[3 * q + a] < lo[a]) lo[a] = v[3 * q + a];
                if (v[3 * q + a] > hi[a]) hi[a] = v[3 * q + a];
            }
    }
    int64_t n = 0;
    for (int64_t i = 0; i < nloops; ++i) {
        for (int64_t j = i + 1; j < nloops; ++j) {
            const double* bi = box + 6 * i;
            const double* bj = box + 6 * j;
            int overlap = 1;
            for (int a = 0; a < 3; ++a)
                if (!(bi[a] <= bj[3 + a] && bj[a] <= bi[3 + a])) overlap = 0;
            if (!overlap) continue;
            if (n < capacity) {
                pairs_out[2 * n] = (int32_t)i;
                pairs_out[2 * n + 1] = (int32_t)j;
            }
            ++n;
        }
    }
    free(box);
    *n_out = n;
    return 0;
}

int lko_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
