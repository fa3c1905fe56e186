// Device-side work packing of a pair list that lives on the device: the
// candidates of a geometry-only serving request (the potential link search,
// Sec. 3.2, Algorithm 2, run on the device), or a served pair list uploaded
// as it is, laid out as work items without the host packer.
//
// Each pair's tiling is the host packer's (it depends only on the pair's two
// loop sizes and the tune table), so each pair's result is the same; the
// tasks are ordered accurate-variant pairs first, then fast-variant ones,
// each in list order (the host packer also puts the largest items first
// within a variant, which only balances the persistent grid's tail and is
// left out here to spare the sort):
//   1. per pair its shape and counts (variant, items, 32-row chunks, segment
//      pairs);
//   2. an exclusive scan of the counts: each pair's rank and first item
//      within its variant, the totals last;
//   3. per pair its PairTask at its place, and item_begin;
//   4. per work item its task, by binary search in item_begin.
// The scans here sum 64-bit integers in a fixed order: one block for up to
// 2^16 elements, else three passes (block totals, one block over the
// totals, block-local scan plus the block's offset).
#include <algorithm>

#include "lk.h"
#include "lk_internal.h"

namespace lk {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanBlock = kScanThreads * kScanPer;   // elements per block

__device__ __forceinline__ PackSums operator+(const PackSums& x, const PackSums& y) {
    return PackSums{x.acc_n + y.acc_n, x.acc_items + y.acc_items, x.fast_n + y.fast_n,
                    x.fast_items + y.fast_items, x.chunks + y.chunks, x.segment_pairs + y.segment_pairs};
}
__device__ __forceinline__ void zero(long long& v) { v = 0; }
__device__ __forceinline__ void zero(PackSums& v) { v = PackSums{0, 0, 0, 0, 0, 0}; }
__device__ __forceinline__ long long load(const int32_t* in, int64_t i) { return (long long)in[i]; }
__device__ __forceinline__ PackSums load(const PackSums* in, int64_t i) { return in[i]; }

// Exclusive scan of the block's thread sums in shared memory; returns the
// block's total.
template <class T>
__device__ T block_exclusive(T& v, T* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int d = 1; d < kScanThreads; d <<= 1) {
        T add;
        zero(add);
        if (t >= d) add = sh[t - d];
        __syncthreads();
        if (t >= d) sh[t] = sh[t] + add;
        __syncthreads();
    }
    const T total = sh[kScanThreads - 1];
    T ex;
    zero(ex);
    if (t > 0) ex = sh[t - 1];
    __syncthreads();
    v = ex;
    return total;
}

template <class T, class In>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const In* __restrict__ in, int64_t n,
                                                                   T* __restrict__ block_sums) {
    __shared__ T sh[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
    T v;
    zero(v);
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < n) v = v + load(in, base + k);
    const T total = block_exclusive(v, sh);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// One block: exclusive scan of the block totals in place, the grand total at [nb].
template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(T* __restrict__ block_sums, int64_t nb) {
    __shared__ T sh[kScanThreads];
    T carry;
    zero(carry);
    for (int64_t b0 = 0; b0 < nb; b0 += kScanBlock) {
        const int64_t base = b0 + (int64_t)threadIdx.x * kScanPer;
        T loc[kScanPer];
        T v;
        zero(v);
        for (int k = 0; k < kScanPer; ++k) {
            zero(loc[k]);
            if (base + k < nb) loc[k] = block_sums[base + k];
            v = v + loc[k];
        }
        const T total = block_exclusive(v, sh);
        T run = carry + v;
        for (int k = 0; k < kScanPer; ++k) {
            if (base + k < nb) block_sums[base + k] = run;
            run = run + loc[k];
        }
        carry = carry + total;
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[nb] = carry;
}

template <class T, class In>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const In* __restrict__ in, int64_t n,
                                                                  const T* __restrict__ block_sums,
                                                                  int64_t nb, T* __restrict__ out) {
    __shared__ T sh[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
    T loc[kScanPer];
    T v;
    zero(v);
    for (int k = 0; k < kScanPer; ++k) {
        zero(loc[k]);
        if (base + k < n) loc[k] = load(in, base + k);
        v = v + loc[k];
    }
    block_exclusive(v, sh);
    T run = block_sums[blockIdx.x] + v;
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) out[base + k] = run;
        run = run + loc[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = block_sums[nb];
}

// One block of 512 threads for lists of up to 2^14 elements (a served
// request's pairs): rounds of 512 coalesced elements, each scanned by warp
// shuffles and a scan of the 16 warp totals, with a carry from round to
// round; the same sums in the same fixed order every time.
constexpr int kScanSingleThreads = 512;
constexpr int64_t kScanSingleMax = (int64_t)1 << 14;

__device__ __forceinline__ long long minus(long long a, long long b) { return a - b; }
__device__ __forceinline__ PackSums minus(const PackSums& a, const PackSums& b) {
    return PackSums{a.acc_n - b.acc_n, a.acc_items - b.acc_items, a.fast_n - b.fast_n,
                    a.fast_items - b.fast_items, a.chunks - b.chunks, a.segment_pairs - b.segment_pairs};
}
__device__ __forceinline__ long long shfl_up(long long v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ PackSums shfl_up(const PackSums& v, int d) {
    return PackSums{shfl_up(v.acc_n, d), shfl_up(v.acc_items, d), shfl_up(v.fast_n, d),
                    shfl_up(v.fast_items, d), shfl_up(v.chunks, d), shfl_up(v.segment_pairs, d)};
}

template <class T, class In>
__global__ void __launch_bounds__(kScanSingleThreads) scan_single_kernel(const In* __restrict__ in, int64_t n,
                                                                         T* __restrict__ out) {
    __shared__ T warp_sum[kScanSingleThreads / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    T carry;
    zero(carry);
    T next;                                   // the next round's element, loaded a round ahead
    zero(next);
    if (t < n) next = load(in, t);
    for (int64_t base = 0; base < n; base += kScanSingleThreads) {
        const int64_t i = base + t;
        const T v = next;
        zero(next);
        if (i + kScanSingleThreads < n) next = load(in, i + kScanSingleThreads);
        T x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T y = shfl_up(x, d);
            if (lane >= d) x = x + y;
        }
        if (lane == 31) warp_sum[w] = x;
        __syncthreads();
        if (w == 0) {
            T z;
            zero(z);
            if (lane < kScanSingleThreads / 32) z = warp_sum[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const T y = shfl_up(z, d);
                if (lane >= d) z = z + y;
            }
            if (lane < kScanSingleThreads / 32) warp_sum[lane] = z;
        }
        __syncthreads();
        T before;
        zero(before);
        if (w > 0) before = warp_sum[w - 1];
        // exclusive: the inclusive sum less this element (integer sums: exact)
        if (i < n) out[i] = carry + before + minus(x, v);
        carry = carry + warp_sum[kScanSingleThreads / 32 - 1];
        __syncthreads();
    }
    if (t == 0) out[n] = carry;
}

template <class T, class In>
void scan(const In* in, int64_t n, T* out, T* scratch, cudaStream_t s) {
    if (n <= kScanSingleMax) {
        scan_single_kernel<T, In><<<1, kScanSingleThreads, 0, s>>>(in, n, out);
        return;
    }
    const int64_t nb = std::max<int64_t>(1, (n + kScanBlock - 1) / kScanBlock);
    scan_reduce_kernel<T, In><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, scratch);
    scan_blocks_kernel<T><<<1, kScanThreads, 0, s>>>(scratch, nb);
    scan_apply_kernel<T, In><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, scratch, nb, out);
}

struct Shape {
    int32_t row_loop, col_loop, n_rows, n_cols, tile_rows, col_tiles, accurate, status;
    int64_t items, chunks;
    uint32_t key;
};

__device__ __forceinline__ uint32_t ceil_log2(int64_t v) {
    uint32_t b = 0;
    while (((int64_t)1 << b) < v) ++b;
    return b;
}

// The shape of pair (a, b), as the host packer computes it.
__device__ Shape pair_shape(const PackParams& P, int32_t a, int32_t b) {
    Shape t{};
    if (a < 0 || b < 0 || a >= P.n_loops || b >= P.n_loops || a == b) {
        t.status = LK_ERR_ARG;              // no items; sorted after every valid pair
        t.key = 0xffffffffu;
        return t;
    }
    t.status = LK_OK;
    const int64_t tc = kTileCols;
    const int64_t na = P.offsets[a + 1] - P.offsets[a];
    const int64_t nb = P.offsets[b + 1] - P.offsets[b];
    // the orientation that sweeps fewer cells including the last column
    // tile's padding; on a tie the longer loop is the row loop
    const int64_t cells_a_rows = na * ((nb + tc - 1) / tc);
    const int64_t cells_b_rows = nb * ((na + tc - 1) / tc);
    const bool a_rows = cells_a_rows != cells_b_rows ? cells_a_rows < cells_b_rows : na >= nb;
    t.row_loop = a_rows ? a : b;
    t.col_loop = a_rows ? b : a;
    const int64_t nr = a_rows ? na : nb, ncl = a_rows ? nb : na;
    t.n_rows = (int32_t)nr;
    t.n_cols = (int32_t)ncl;
    int64_t rows = P.user_rows;
    if (rows <= 0 && P.tune) {
        const uint32_t rc = ceil_log2(nr), cc = ceil_log2(ncl);
        if (rc < kTuneClasses && cc < kTuneClasses) rows = P.tune[rc * kTuneClasses + cc];
    }
    if (rows <= 0) {
        const int64_t col_tiles = (ncl + tc - 1) / tc;
        int64_t row_tiles = (nr + 255) / 256;
        const int64_t max_items = 1 << 16;
        if (col_tiles * row_tiles > max_items) row_tiles = max_items / col_tiles > 1 ? max_items / col_tiles : 1;
        rows = (nr + row_tiles - 1) / row_tiles;
        rows = (rows + kChunkRows - 1) / kChunkRows * kChunkRows;
        if (rows > (int64_t)INT32_MAX) rows = INT32_MAX;
    }
    t.tile_rows = (int32_t)rows;
    t.col_tiles = (int32_t)((ncl + tc - 1) / tc);
    t.items = (int64_t)t.col_tiles * ((nr + rows - 1) / rows);
    t.accurate = nr * ncl >= P.accurate_threshold ? 1 : 0;
    const int64_t cost = (rows < nr ? rows : nr) * (tc < ncl ? tc : ncl);
    const uint32_t c = (uint32_t)(cost < 0x7ffffffe ? cost : 0x7ffffffe);
    t.key = (t.accurate ? 0u : 0x80000000u) | (0x7ffffffeu - c);
    const int64_t full = nr / rows, last = nr - full * rows;
    const int64_t per_col = full * ((rows + kChunkRows - 1) / kChunkRows) +
                            (last > 0 ? (last + kChunkRows - 1) / kChunkRows : 0);
    t.chunks = per_col * t.col_tiles;
    return t;
}

// Per pair, in list order, its variant and counts: the scan input.  An
// invalid pair counts as a fast-variant pair with no items.
__global__ void pack_count_kernel(const int32_t* __restrict__ pairs, int64_t n, PackParams P,
                                  PackSums* __restrict__ vals) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const Shape t = pair_shape(P, pairs[2 * p], pairs[2 * p + 1]);
    if (t.status != LK_OK) {
        vals[p] = PackSums{0, 0, 1, 0, 0, 0};
        return;
    }
    const long long sp = (long long)t.n_rows * t.n_cols;
    vals[p] = t.accurate ? PackSums{1, t.items, 0, 0, t.chunks, sp} : PackSums{0, 0, 1, t.items, t.chunks, sp};
}

// Per pair its task, at its rank within its variant (accurate-variant pairs
// first, list order within each), and its first item.
__global__ void pack_place_kernel(const int32_t* __restrict__ pairs, int64_t n, PackParams P,
                                  const PackSums* __restrict__ scan, PairTask* __restrict__ tasks,
                                  int64_t* __restrict__ item_begin) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const PackSums e = scan[p], tot = scan[n];
    if (p == 0) item_begin[n] = tot.acc_items + tot.fast_items;
    const Shape t = pair_shape(P, pairs[2 * p], pairs[2 * p + 1]);
    const bool acc = t.status == LK_OK && t.accurate;
    const int64_t k = acc ? e.acc_n : tot.acc_n + e.fast_n;
    item_begin[k] = acc ? e.acc_items : tot.acc_items + e.fast_items;
    PairTask q{};
    q.out_index = (int32_t)p;
    q.scale = 1.0f;
    if (t.status != LK_OK) {
        q.status = t.status;
        tasks[k] = q;
        return;
    }
    q.V = P.V;
    q.R = P.R;
    q.row_loop = t.row_loop;
    q.col_loop = t.col_loop;
    q.row_base = P.offsets[t.row_loop];
    q.col_base = P.offsets[t.col_loop];
    q.n_rows = t.n_rows;
    q.n_cols = t.n_cols;
    q.tile_rows = t.tile_rows;
    q.col_tiles = t.col_tiles;
    q.status = 0;
    q.accurate = t.accurate;
    tasks[k] = q;
}

// item_task[i] = the task k with item_begin[k] <= i < item_begin[k + 1].
__global__ void pack_item_task_kernel(const int64_t* __restrict__ item_begin, int64_t n_tasks, int64_t n_items,
                                      int32_t* __restrict__ item_task) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    int64_t lo = 0, hi = n_tasks - 1;   // the last k with item_begin[k] <= i
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (item_begin[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    item_task[i] = (int32_t)lo;
}

}  // namespace

size_t scan_scratch_count(int64_t n) { return (size_t)std::max<int64_t>(1, (n + kScanBlock - 1) / kScanBlock) + 1; }

void launch_scan_counts(const int32_t* counts, int64_t n, int64_t* offsets, long long* scratch, cudaStream_t s) {
    scan<long long, int32_t>(counts, n, reinterpret_cast<long long*>(offsets), scratch, s);
}

void launch_pack(const int32_t* pairs, int64_t n, const PackParams& P, PairTask* tasks, PackSums* vals,
                 PackSums* scan_out, PackSums* scratch, int64_t* item_begin, cudaStream_t s) {
    if (n <= 0) return;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    pack_count_kernel<<<blocks, 256, 0, s>>>(pairs, n, P, vals);
    scan<PackSums, PackSums>(vals, n, scan_out, scratch, s);
    pack_place_kernel<<<blocks, 256, 0, s>>>(pairs, n, P, scan_out, tasks, item_begin);
}

void launch_pack_item_task(const int64_t* item_begin, int64_t n_tasks, int64_t n_items, int32_t* item_task,
                           cudaStream_t s) {
    if (n_items <= 0 || n_tasks <= 0) return;
    pack_item_task_kernel<<<(unsigned)((n_items + 255) / 256), 256, 0, s>>>(item_begin, n_tasks, n_items, item_task);
}

}  // namespace lk
