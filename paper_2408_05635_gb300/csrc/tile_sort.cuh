// tile_sort.cuh -- per-tile depth sort, run by the forward kernel's block before it
// composites the tile.
//
// Eqs. 2-4 composite the Gaussians of a pixel front to back, so every tile needs its
// entries in ascending camera depth; ties are broken by Gaussian index (the order the
// oracle uses), which the record index already encodes (records are numbered in
// (view, Gaussian) order).  k_emit leaves each tile's 64-bit keys (depth bits << 32 |
// record) in arrival order inside the tile's own slice of the key array, so the sort is
// segmented by construction: the block of a tile sorts only its slice.  Up to
// kRankSortMax keys: each thread ranks its keys by counting the smaller ones (keys are
// unique) and scatters them, no barrier between steps; up to kSortSmemKeys keys: a
// bitonic network in shared memory; longer slices: the same network in place in global
// memory (padding is virtual: a missing partner is +inf).  The record ids, in order,
// are written to `sorted` for the compositors.
#pragma once

#include "gs_internal.cuh"

namespace gsk {

constexpr int kRankSortMax = 128;
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

// Sort the tile's keys [start, start + n) and write the record ids to sorted[start ..).
// sk: kSortSmemKeys keys of shared memory.  Ends with a barrier.
__device__ inline void sort_tile(const WsPtrs &ws, uint32_t start, int n, unsigned long long *sk) {
    if (n <= 0) {
        __syncthreads();
        return;
    }
    if (n <= kRankSortMax) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = ws.keys[start + i];
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long key = sk[i];
            int rank = 0;
            for (int j = 0; j < n; ++j) rank += sk[j] < key;
            ws.sorted[start + rank] = (uint32_t)key;
        }
    } else {
        unsigned long long *k = ws.keys + start;
        if (n <= kSortSmemKeys) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = ws.keys[start + i];
            __syncthreads();
            k = sk;
        }
        bitonic_sort(k, n);
        for (int i = threadIdx.x; i < n; i += blockDim.x) ws.sorted[start + i] = (uint32_t)k[i];
    }
    __syncthreads();
}

}  // namespace gsk
