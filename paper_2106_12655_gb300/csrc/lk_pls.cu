// Potential link search on the device (Sec. 3.2, Algorithm 2): the loop
// pairs (i, j), i < j, whose axis-aligned bounding boxes overlap.  Two loops
// with a nonzero linking number have overlapping convex hulls, so every other
// pair has linking number 0 and needs no direct sum.
//
// Boxes overlap when their closed intervals intersect on all three axes.  The
// FP64 box bounds are compared exactly, as order-preserving int64 keys (the
// FP64 pipe of this GPU is a small fraction of its integer pipe): for a finite
// double x with bits b (after mapping -0 to +0), key = b for x >= 0 and
// key = b ^ 0x7fff...f for x < 0, so key(x) <= key(y) exactly when x <= y.
//
// Up to 2^27 box pairs the search tests every pair (tiled through shared
// memory: one warp per row i, eight rows per block sharing each staged tile
// of 256 boxes; a count pass, then a write pass at each row's offset, so the
// list is in (i, j) order), which is faster than the sorts' launches there.
//
// Above that, sort and sweep on one axis (Algorithm 2 builds a bounding-volume
// hierarchy; a sorted sweep finds the same set, with work proportional to the
// pairs that overlap in x rather than to L^2): the loops are sorted by the
// upper 32 bits of their lower x key (ties by loop index), and each loop
// scans forward in that order while the next loop's key is at most the upper
// 32 bits of its own upper x key -- every box whose lower x bound lies within
// its x extent, so each overlapping pair is met exactly once, from the one
// that comes first -- and tests all three axes exactly.  A count pass and a
// write pass (after an exclusive scan of the counts) produce the pairs as
// 64-bit keys (i << 32 | j), which a final sort puts in (i, j) order, so the
// list does not depend on scheduling.  Both sorts are bitonic networks over
// 64-bit keys: a block sorts 2048 keys in shared memory, longer merges run
// one global pass per step above that size.
#include "lk_internal.h"

namespace lk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPlsRows = 8;      // rows (warps) per block
constexpr int kPlsTile = 256;    // boxes staged per shared-memory tile

__device__ __forceinline__ long long order_key(double x) {
    const long long b = __double_as_longlong(x + 0.0);   // -0 becomes +0
    return b < 0 ? (b ^ 0x7fffffffffffffffll) : b;
}

// keys[a * L + l], a = 0..5: lo.x, lo.y, lo.z, hi.x, hi.y, hi.z of loop l.
__global__ void pls_keys_kernel(const double* __restrict__ aabb, int64_t L, long long* __restrict__ keys) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
#pragma unroll
    for (int a = 0; a < 6; ++a) keys[a * L + l] = order_key(aabb[6 * l + a]);
}

template <bool WRITE>
__global__ void __launch_bounds__(32 * kPlsRows) pls_kernel(const long long* __restrict__ keys, int64_t L,
                                                             int32_t* __restrict__ counts,
                                                             const int64_t* __restrict__ offsets,
                                                             int32_t* __restrict__ pairs, int64_t capacity) {
    __shared__ long long tile[6][kPlsTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * kPlsRows;
    const int64_t i = row0 + warp;
    const bool live = i < L;                       // warp-uniform
    long long me[6] = {0, 0, 0, 0, 0, 0};
    if (live) {
#pragma unroll
        for (int a = 0; a < 6; ++a) me[a] = keys[a * L + i];
    }
    int64_t out = (WRITE && live) ? offsets[i] : 0;
    int64_t cnt = 0;
    const unsigned below = (1u << lane) - 1u;
    for (int64_t j0 = row0 + 1; j0 < L; j0 += kPlsTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < 6 * kPlsTile; k += blockDim.x) {
            const int a = k / kPlsTile, c = k % kPlsTile;
            const int64_t j = j0 + c;
            tile[a][c] = j < L ? keys[a * L + j] : 0;
        }
        __syncthreads();
        if (!live) continue;
        for (int c = 0; c < kPlsTile; c += 32) {
            const int64_t j = j0 + c + lane;
            const int cl = c + lane;
            const bool hit = j > i && j < L && me[0] <= tile[3][cl] && tile[0][cl] <= me[3] &&
                             me[1] <= tile[4][cl] && tile[1][cl] <= me[4] && me[2] <= tile[5][cl] &&
                             tile[2][cl] <= me[5];
            const unsigned m = __ballot_sync(kFull, hit);
            if (WRITE && hit) {
                const int64_t slot = out + __popc(m & below);
                if (slot < capacity) {
                    pairs[2 * slot] = (int32_t)i;
                    pairs[2 * slot + 1] = (int32_t)j;
                }
            }
            out += __popc(m);
            cnt += __popc(m);
        }
    }
    if (!WRITE && live && lane == 0) counts[i] = (int32_t)cnt;
}

constexpr int kSortBlock = 2048;       // keys per block of the shared-memory bitonic stages

// One compare-exchange step of the bitonic network: element i against i ^ j,
// ascending where (i & k) == 0.
__device__ __forceinline__ void bitonic_step(unsigned long long* a, unsigned i, unsigned j, unsigned k) {
    const unsigned p = i ^ j;
    if (p > i) {
        const unsigned long long x = a[i], y = a[p];
        if (((i & k) == 0) == (x > y)) {
            a[i] = y;
            a[p] = x;
        }
    }
}

// Stages k = 2 .. kSortBlock of the network on each block's 2048 keys.
__global__ void __launch_bounds__(kSortBlock / 2) bitonic_block_kernel(unsigned long long* __restrict__ a) {
    __shared__ unsigned long long s[kSortBlock];
    const unsigned base = blockIdx.x * kSortBlock;
    for (unsigned t = threadIdx.x; t < kSortBlock; t += blockDim.x) s[t] = a[base + t];
    __syncthreads();
    for (unsigned k = 2; k <= kSortBlock; k <<= 1)
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned t = threadIdx.x; t < kSortBlock; t += blockDim.x) {
                const unsigned i = t, p = i ^ j;
                if (p > i) {
                    const unsigned long long x = s[i], y = s[p];
                    if ((((base + i) & k) == 0) == (x > y)) {
                        s[i] = y;
                        s[p] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (unsigned t = threadIdx.x; t < kSortBlock; t += blockDim.x) a[base + t] = s[t];
}

// One global step j >= kSortBlock of stage k.
__global__ void bitonic_global_kernel(unsigned long long* __restrict__ a, unsigned n, unsigned j, unsigned k) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) bitonic_step(a, i, j, k);
}

// Steps j = kSortBlock/2 .. 1 of stage k on each block's keys.
__global__ void __launch_bounds__(kSortBlock / 2) bitonic_tail_kernel(unsigned long long* __restrict__ a,
                                                                     unsigned k) {
    __shared__ unsigned long long s[kSortBlock];
    const unsigned base = blockIdx.x * kSortBlock;
    for (unsigned t = threadIdx.x; t < kSortBlock; t += blockDim.x) s[t] = a[base + t];
    __syncthreads();
    for (unsigned j = kSortBlock >> 1; j > 0; j >>= 1) {
        for (unsigned t = threadIdx.x; t < kSortBlock; t += blockDim.x) {
            const unsigned i = t, p = i ^ j;
            if (p > i) {
                const unsigned long long x = s[i], y = s[p];
                if ((((base + i) & k) == 0) == (x > y)) {
                    s[i] = y;
                    s[p] = x;
                }
            }
        }
        __syncthreads();
    }
    for (unsigned t = threadIdx.x; t < kSortBlock; t += blockDim.x) a[base + t] = s[t];
}

// Upper 32 bits of a key as an unsigned order (the sign bit flipped).
__device__ __forceinline__ unsigned long long key_hi32(long long key) {
    return ((unsigned long long)key ^ 0x8000000000000000ull) >> 32;
}

// a[l] = (hi32(lower x key of l) << 32) | l for l < L; the padding n > L with
// the largest key.
__global__ void pls_sort_keys_kernel(const long long* __restrict__ keys, int64_t L, unsigned n,
                                     unsigned long long* __restrict__ a) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    a[i] = (int64_t)i < L ? (key_hi32(keys[i]) << 32) | i : ~0ull;
}

// Sweep: sorted position r against the positions after it, while their lower
// x key is within r's upper x key (see the head of this file).
template <bool WRITE>
__global__ void pls_sweep_kernel(const long long* __restrict__ keys, int64_t L, const unsigned long long* __restrict__ a,
                                 int32_t* __restrict__ counts, const int64_t* __restrict__ offsets,
                                 unsigned long long* __restrict__ pairs, int64_t capacity) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= L) return;
    const unsigned l = (unsigned)(a[r] & 0xffffffffu);
    long long me[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) me[k] = keys[k * L + l];
    const unsigned long long hx = key_hi32(me[3]);
    int64_t out = WRITE ? offsets[r] : 0;
    int32_t cnt = 0;
    for (int64_t s = r + 1; s < L; ++s) {
        const unsigned long long e = a[s];
        if ((e >> 32) > hx) break;
        const unsigned m = (unsigned)(e & 0xffffffffu);
        if (me[0] <= keys[3 * L + m] && keys[m] <= me[3] && me[1] <= keys[4 * L + m] &&
            keys[L + m] <= me[4] && me[2] <= keys[5 * L + m] && keys[2 * L + m] <= me[5]) {
            if (WRITE && out < capacity)
                pairs[out] = l < m ? ((unsigned long long)l << 32) | m : ((unsigned long long)m << 32) | l;
            ++out;
            ++cnt;
        }
    }
    if (!WRITE) counts[r] = cnt;
}

// (i << 32 | j) keys to int32 pairs.
__global__ void pls_unpack_kernel(const unsigned long long* __restrict__ keys, int64_t n, int32_t* __restrict__ pairs) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    pairs[2 * k] = (int32_t)(keys[k] >> 32);
    pairs[2 * k + 1] = (int32_t)(keys[k] & 0xffffffffu);
}

}  // namespace

unsigned pls_sort_size(int64_t n) {
    unsigned p = kSortBlock;
    while ((int64_t)p < n) p <<= 1;
    return p;
}

void launch_bitonic_sort(unsigned long long* a, unsigned n, cudaStream_t s) {
    // n: a power of two, at least kSortBlock
    bitonic_block_kernel<<<n / kSortBlock, kSortBlock / 2, 0, s>>>(a);
    for (unsigned k = 2 * kSortBlock; k <= n; k <<= 1) {
        for (unsigned j = k >> 1; j >= (unsigned)kSortBlock; j >>= 1)
            bitonic_global_kernel<<<(n + 255) / 256, 256, 0, s>>>(a, n, j, k);
        bitonic_tail_kernel<<<n / kSortBlock, kSortBlock / 2, 0, s>>>(a, k);
    }
}

void launch_pls_sort(const long long* keys, int64_t n_loops, unsigned long long* order, unsigned n, cudaStream_t s) {
    pls_sort_keys_kernel<<<(n + 255) / 256, 256, 0, s>>>(keys, n_loops, n, order);
    launch_bitonic_sort(order, n, s);
}

void launch_pls_sweep_count(const long long* keys, int64_t n_loops, const unsigned long long* order,
                            int32_t* counts, cudaStream_t s) {
    if (n_loops <= 0) return;
    pls_sweep_kernel<false><<<(unsigned)((n_loops + 127) / 128), 128, 0, s>>>(keys, n_loops, order, counts, nullptr,
                                                                          nullptr, 0);
}

void launch_pls_sweep_write(const long long* keys, int64_t n_loops, const unsigned long long* order,
                            const int64_t* offsets, unsigned long long* pairs, int64_t capacity, cudaStream_t s) {
    if (n_loops <= 0) return;
    pls_sweep_kernel<true><<<(unsigned)((n_loops + 127) / 128), 128, 0, s>>>(keys, n_loops, order, nullptr, offsets,
                                                                         pairs, capacity);
}

void launch_pls_unpack(const unsigned long long* keys, int64_t n, int32_t* pairs, cudaStream_t s) {
    if (n <= 0) return;
    pls_unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, pairs);
}

void launch_pls_keys(const double* aabb, int64_t n_loops, long long* keys, cudaStream_t s) {
    if (n_loops <= 0) return;
    pls_keys_kernel<<<(unsigned)((n_loops + 255) / 256), 256, 0, s>>>(aabb, n_loops, keys);
}

void launch_pls_count(const long long* keys, int64_t n_loops, int32_t* counts, cudaStream_t s) {
    if (n_loops <= 0) return;
    const int64_t blocks = (n_loops + kPlsRows - 1) / kPlsRows;
    pls_kernel<false><<<(unsigned)blocks, 32 * kPlsRows, 0, s>>>(keys, n_loops, counts, nullptr, nullptr, 0);
}

void launch_pls_write(const long long* keys, int64_t n_loops, const int64_t* offsets, int32_t* pairs,
                      int64_t capacity, cudaStream_t s) {
    if (n_loops <= 0 || capacity <= 0) return;
    const int64_t blocks = (n_loops + kPlsRows - 1) / kPlsRows;
    pls_kernel<true><<<(unsigned)blocks, 32 * kPlsRows, 0, s>>>(keys, n_loops, nullptr, offsets, pairs, capacity);
}

}  // namespace lk
