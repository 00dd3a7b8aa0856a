// Line sums s_l = sum_{k in line l} val_k g[idx_k] over the lines of a
// compressed view (the rows of A by row_ptr / col / values, or its columns by
// col_ptr / csc_row / column-ordered values), the common core of the update
// (eq. phys-inter-ELLAM), the scalings (eq. volAdj) and the minimisation's
// matrix products.
//
// Lines hold a few to a few tens of entries, so one thread or one warp per
// line reads memory in short dependent chains and leaves HBM idle.  Instead,
// the entries are cut into tiles of about kTileEntries consecutive entries at
// line boundaries (tile k holds the lines whose first entry lies in
// [k T, (k + 1) T), found once per step by binary search on the pointers).  A
// block streams a tile's indices and values into shared memory with
// coalesced loads, then each thread sums whole lines from shared memory,
// gathering g (resident in L2) by index, while the next tile streams into a
// second buffer (cp.async).  A tile whose last line overhangs the shared
// arrays (a line of more than kTileSlack entries) is summed from global
// memory by one warp per line instead.  Every line is summed by one thread or
// one warp in entry order, and the grid is fixed, so each sum's order is fixed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bchar {

constexpr int kTileEntries = 1536;
constexpr int kTileSlack = 512;
constexpr int kTileCap = kTileEntries + kTileSlack;
constexpr int kTileThreads = 256;
constexpr int kTileBlocks = 152 * 4;  // persistent grid: 4 blocks of 2 x 24 KB shared memory per SM
// dynamic shared memory of a tile kernel: two buffers of kTileCap indices and values
constexpr size_t kTileSmem = 2 * static_cast<size_t>(kTileCap) * (sizeof(int32_t) + sizeof(double));

struct LineView {
    int64_t n;             // lines
    const int64_t *ptr;    // n + 1 line pointers
    const int32_t *idx;    // gathered index of every entry
    const double *val;     // value of every entry
    const int32_t *tile;   // ntile + 1: first line of each tile
    int64_t ntile;
};

// tile[k] = the first line l with ptr[l] >= k T (k < ntile), tile[ntile] = n.
__global__ void k_tile_bounds(int64_t n, const int64_t *ptr, int64_t ntile, int32_t *tile);

inline int64_t tile_count(int64_t nnz) { return (nnz + kTileEntries - 1) / kTileEntries; }

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

struct TileBufs {
    int32_t *idx[2];
    double *val[2];
    __device__ explicit TileBufs(unsigned char *smem) {
        val[0] = reinterpret_cast<double *>(smem);
        val[1] = val[0] + kTileCap;
        idx[0] = reinterpret_cast<int32_t *>(val[1] + kTileCap);
        idx[1] = idx[0] + kTileCap;
    }
};

// Starts the asynchronous copy of tile k of V into buffer b (nothing when the
// tile is empty or too wide for the buffers) and commits it as one group.
__device__ __forceinline__ void tile_prefetch(const LineView &V, int64_t k, TileBufs &B, int b) {
    const int64_t l0 = V.tile[k], l1 = V.tile[k + 1];
    if (l0 < l1) {
        const int64_t e0 = V.ptr[l0], ne = V.ptr[l1] - e0;
        if (ne <= kTileCap)
            for (int64_t t = threadIdx.x; t < ne; t += blockDim.x) {
                cp_async4(&B.idx[b][t], V.idx + e0 + t);
                cp_async8(&B.val[b][t], V.val + e0 + t);
            }
    }
    cp_async_commit();
}

// Sums the lines of tile k of V from buffer b (already landed): epi(l, s)
// once per line, from one thread (or lane 0 of one warp for a tile too wide
// for the buffers, summed from global memory).
template <class G, class Epi>
__device__ __forceinline__ void tile_compute(const LineView &V, int64_t k, const G *g, Epi &epi, TileBufs &B, int b) {
    const int64_t l0 = V.tile[k], l1 = V.tile[k + 1];
    if (l0 >= l1) return;  // block-uniform: a line spanning several tiles leaves some empty
    const int64_t e0 = V.ptr[l0], ne = V.ptr[l1] - e0;
    if (ne <= kTileCap) {
        const int32_t *sidx = B.idx[b];
        const double *sval = B.val[b];
        for (int64_t l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
            const int64_t a = V.ptr[l] - e0, c = V.ptr[l + 1] - e0;
            double s = 0.0;
            for (int64_t e = a; e < c; ++e) s += sval[e] * static_cast<double>(g[sidx[e]]);
            epi(l, s);
        }
    } else {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        for (int64_t l = l0 + warp; l < l1; l += nwarps) {  // warp-uniform
            double s = 0.0;
            for (int64_t e = V.ptr[l] + lane; e < V.ptr[l + 1]; e += 32)
                s += V.val[e] * static_cast<double>(g[V.idx[e]]);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) epi(l, s);
        }
    }
}

// The persistent tile loop over the tiles of view A, then those of view B
// (B.ntile may be 0), k = blockIdx.x, blockIdx.x + gridDim.x, ...: tile k + grid
// streams into the other buffer while tile k is summed.  Every thread of the
// block must call it.
template <class GA, class EA, class GB, class EB>
__device__ __forceinline__ void tile_loop(const LineView &A, const GA *ga, EA &ea, const LineView &Bv, const GB *gb,
                                          EB &eb, unsigned char *smem) {
    TileBufs B(smem);
    const int64_t total = A.ntile + Bv.ntile;
    const int64_t step = gridDim.x;
    int64_t k = blockIdx.x;
    if (k >= total) return;  // block-uniform
    if (k < A.ntile) tile_prefetch(A, k, B, 0);
    else tile_prefetch(Bv, k - A.ntile, B, 0);
    int b = 0;
    for (; k < total; k += step) {
        const int64_t kn = k + step;
        if (kn < total) {
            if (kn < A.ntile) tile_prefetch(A, kn, B, b ^ 1);
            else tile_prefetch(Bv, kn - A.ntile, B, b ^ 1);
        } else {
            cp_async_commit();  // an empty group keeps the count: wait_group 1 then means "tile k landed"
        }
        cp_async_wait_one();
        __syncthreads();
        if (k < A.ntile) tile_compute(A, k, ga, ea, B, b);
        else tile_compute(Bv, k - A.ntile, gb, eb, B, b);
        __syncthreads();  // buffer b is refilled by the next iteration's prefetch
        b ^= 1;
    }
}

}  // namespace bchar
