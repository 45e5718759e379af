// tile_sort.cuh -- per-tile depth sort, run by the forward kernel's block before it
// composites the tile.
//
// Eqs. 2-4 composite the Gaussians of a pixel front to back, so every tile needs its
// entries in ascending camera depth; ties are broken by Gaussian index (the order the
// oracle uses), which the record index already encodes (records are numbered in
// (view, Gaussian) order).  k_emit leaves each tile's 64-bit keys (depth bits << 32 |
// record) in arrival order inside the tile's own slice of the key array, so the sort is
// segmented by construction: the block of a tile sorts only its slice.  Up to
// kSortSmemKeys keys: each warp sorts runs of 32 keys in registers (a bitonic network
// over the lanes, exchanging by shuffles), then runs are merged pairwise in shared
// memory, each key moving to its position in its run plus the number of smaller keys in
// the partner run (a binary search; keys are unique): one barrier per doubling of the
// run length instead of one per bitonic stage.  Longer slices: a bitonic network in
// place in global memory (padding is virtual: a missing partner is +inf).  The record
// ids, in order, are written to `sorted` for the compositors.
#pragma once

#include "gs_internal.cuh"

namespace gsk {

constexpr int kSortSmemKeys = 1024;

__device__ __forceinline__ void cmp_swap(unsigned long long *k, int lo, int hi) {
    const unsigned long long a = k[lo], b = k[hi];
    if (a > b) {
        k[lo] = b;
        k[hi] = a;
    }
}

// Ascending bitonic sort of k[0, n) by all threads of the block.  Each merge of size
// `size` starts with a mirrored comparison (lo, size-1-lo) followed by half-cleaners, so
// every compare-exchange puts the smaller key at the lower index and entries >= n can
// be treated as +inf without being stored.
__device__ inline void bitonic_sort(unsigned long long *k, int n) {
    int P = 1;
    while (P < n) P <<= 1;
    const int pairs = P >> 1;
    for (int size = 2; size <= P; size <<= 1) {
        const int half = size >> 1;
        for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
            const int blk = p / half, off = p - blk * half;
            const int lo = blk * size + off, hi = blk * size + size - 1 - off;
            if (hi < n) cmp_swap(k, lo, hi);
        }
        __syncthreads();
        for (int j = half >> 1; j > 0; j >>= 1) {
            for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
                const int lo = (p / j) * 2 * j + (p % j), hi = lo + j;
                if (hi < n) cmp_swap(k, lo, hi);
            }
            __syncthreads();
        }
    }
}

// Ascending bitonic sort of 32 keys, one per lane of the warp.
__device__ __forceinline__ unsigned long long warp_sort32(unsigned long long key, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, j);
            const bool up = (lane & k) == 0, low = (lane & j) == 0;
            key = (low == up) ? (other < key ? other : key) : (other > key ? other : key);
        }
    }
    return key;
}

// Sort the tile's keys [start, start + n) and write the record ids to sorted[start ..).
// sk: 2 kSortSmemKeys keys of shared memory.  Ends with a barrier.
__device__ inline void sort_tile(const WsPtrs &ws, uint32_t start, int n, unsigned long long *sk) {
    if (n <= 0) {
        __syncthreads();
        return;
    }
    if (n > kSortSmemKeys) {
        unsigned long long *k = ws.keys + start;
        bitonic_sort(k, n);
        for (int i = threadIdx.x; i < n; i += blockDim.x) ws.sorted[start + i] = (uint32_t)k[i];
        __syncthreads();
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (int)(blockDim.x >> 5);
    unsigned long long *A = sk, *B = sk + kSortSmemKeys;
    // runs of 32 sorted in registers; a short run's missing keys are +inf and sort last
    for (int c = warp; (c << 5) < n; c += nwarps) {
        const int i = (c << 5) + lane;
        const unsigned long long key = warp_sort32(i < n ? ws.keys[start + i] : ~0ull, lane);
        if (i < n) A[i] = key;
    }
    __syncthreads();
    // pairwise merges: a key of run c lands at (pair start) + (its place in run c) + (keys
    // of the partner run smaller than it)
    for (int m = 32; m < n; m <<= 1) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long key = A[i];
            const int c = i / m, p = i - c * m;
            const int o0 = (c ^ 1) * m, o1 = min(o0 + m, n);
            int lo = o0, hi = o1 > o0 ? o1 : o0;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (A[mid] < key) lo = mid + 1; else hi = mid;
            }
            B[(c & ~1) * m + p + (lo - o0)] = key;
        }
        __syncthreads();
        unsigned long long *t = A;
        A = B;
        B = t;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) ws.sorted[start + i] = (uint32_t)A[i];
    __syncthreads();
}

}  // namespace gsk
