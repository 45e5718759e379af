// sort.cu -- per-tile depth sort.
//
// Eqs. 2-4 composite the Gaussians of a pixel front to back, so every tile needs its
// entries in ascending camera depth; ties are broken by Gaussian index (the order the
// oracle uses).  k_emit leaves each tile's 64-bit keys (depth bits << 32 | record) in
// arrival order inside the tile's own slice of the key array, so the sort is segmented
// by construction: one block per tile sorts only its slice.  Slices of up to
// kSortSmemCap keys are sorted in shared memory, longer ones in place in global memory,
// both with the same bitonic network (padding is virtual: a missing partner is +inf).
#include "gs_internal.cuh"

namespace gsk {

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
__device__ void bitonic_sort(unsigned long long *k, int n) {
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

// Keys with equal depth bits came out ordered by record; reorder each such run by
// Gaussian index (one thread; runs are rare and short).
__device__ void fix_ties(unsigned long long *k, int n, const Rec *rec) {
    int tie = 0;
    for (int i = threadIdx.x; i + 1 < n; i += blockDim.x)
        if ((k[i] >> 32) == (k[i + 1] >> 32)) tie = 1;
    if (!__syncthreads_or(tie)) return;
    if (threadIdx.x == 0) {
        for (int i = 1; i < n; ++i) {
            int j = i;
            while (j > 0 && (k[j - 1] >> 32) == (k[j] >> 32) &&
                   __float_as_uint(rec[(uint32_t)k[j - 1]].c.w) > __float_as_uint(rec[(uint32_t)k[j]].c.w)) {
                const unsigned long long t = k[j - 1];
                k[j - 1] = k[j];
                k[j] = t;
                --j;
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kTilePix) k_tile_sort(WsPtrs ws, Dims d) {
    __shared__ unsigned long long sk[kSortSmemCap];
    const uint32_t tile = blockIdx.x;
    uint32_t start;
    const int n = (int)tile_entries(ws, d, tile, start);
    if (n == 0) return;
    unsigned long long *k;
    if (n <= kSortSmemCap) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = ws.keys[start + i];
        __syncthreads();
        k = sk;
    } else {
        k = ws.keys + start;
    }
    bitonic_sort(k, n);
    fix_ties(k, n, ws.rec);
    for (int i = threadIdx.x; i < n; i += blockDim.x) ws.sorted[start + i] = (uint32_t)k[i];
}

cudaError_t launch_tile_sort(const WsPtrs &ws, const Dims &d, cudaStream_t st) {
    if (d.T == 0) return cudaSuccess;
    k_tile_sort<<<d.T, kTilePix, 0, st>>>(ws, d);
    return cudaGetLastError();
}

}  // namespace gsk
