// sort.cu -- per-tile depth sort.
//
// Eqs. 2-4 composite the Gaussians of a pixel front to back, so every tile needs its
// entries in ascending camera depth; ties are broken by Gaussian index (the order the
// oracle uses), which the record index already encodes (records are numbered in
// (view, Gaussian) order).  k_emit leaves each tile's 64-bit keys (depth bits << 32 | record) in
// arrival order inside the tile's own slice of the key array, so the sort is segmented
// by construction: one block per tile sorts only its slice.  Slices of up to
// kRankSortMax keys are sorted by ranking (no barriers), up to kSortSmemCap keys by a
// bitonic network in shared memory, longer ones by the same network in place in global
// memory (padding is virtual: a missing partner is +inf).
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

// Short lists (the common case): each thread ranks its keys by counting the smaller
// ones (keys are unique: the low word is the record) and scatters them; no barrier
// between steps, O(n^2 / threads) compares.
constexpr int kRankSortMax = 512;

__global__ void __launch_bounds__(kTilePix) k_tile_sort(WsPtrs ws, Dims d) {
    __shared__ __align__(16) unsigned long long sk[kSortSmemCap];
    __shared__ unsigned long long so[kRankSortMax];
    const uint32_t tile = blockIdx.x;
    uint32_t start;
    const int n = (int)tile_entries(ws, d, tile, start);
    if (n == 0) return;
    unsigned long long *k;
    if (n <= kRankSortMax) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = ws.keys[start + i];
        if (threadIdx.x == 0 && (n & 1)) sk[n] = ~0ull;  // pad to pairs: compares as largest
        __syncthreads();
        const ulonglong2 *sk2 = reinterpret_cast<const ulonglong2 *>(sk);
        const int n2 = (n + 1) >> 1;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long key = sk[i];
            int rank = 0;
            for (int j = 0; j < n2; ++j) {
                const ulonglong2 p = sk2[j];
                rank += (p.x < key) + (p.y < key);
            }
            so[rank] = key;
        }
        __syncthreads();
        k = so;
    } else if (n <= kSortSmemCap) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = ws.keys[start + i];
        __syncthreads();
        bitonic_sort(sk, n);
        k = sk;
    } else {
        k = ws.keys + start;
        bitonic_sort(k, n);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) ws.sorted[start + i] = (uint32_t)k[i];
}

cudaError_t launch_tile_sort(const WsPtrs &ws, const Dims &d, cudaStream_t st) {
    if (d.T == 0) return cudaSuccess;
    k_tile_sort<<<d.T, kTilePix, 0, st>>>(ws, d);
    return cudaGetLastError();
}

}  // namespace gsk
