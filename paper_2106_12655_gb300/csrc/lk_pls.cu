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
// The search is a brute-force test of all L(L-1)/2 box pairs, tiled through
// shared memory: one warp per row i, eight rows per block sharing each staged
// tile of 256 boxes.  A count pass gives each row its number of candidates; a
// write pass, after the host's exclusive scan of those counts, writes row i's
// pairs in increasing j at its offset, so the list is sorted by (i, j) and
// independent of scheduling.
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

}  // namespace

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
