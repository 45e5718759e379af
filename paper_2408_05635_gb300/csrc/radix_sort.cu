// radix_sort.cu -- the front-to-back order of Eqs. 2-4 as one device-wide LSD radix sort
// of every (Gaussian, tile) pair on the key (tile, depth), the alternative to the per-tile
// sort inside the forward (tile_sort.cuh), picked by the launch schedule (GS_SCHED_RADIX).
//
// k_emit (in this mode) writes each pair as the 64-bit key tile << 32 | bits(depth) (the
// depth is positive, so its IEEE bits order as unsigned integers) with the record as the
// value.  Eight-bit digits are sorted least significant first, each pass stable:
//   k_radix_hist     per block of 1,024 or 4,096 keys, the count of each digit value;
//   k_radix_scan     per digit value, the exclusive prefix of its counts over the blocks
//                    and its total;
//   k_radix_scatter  per block, every key's destination: the keys of smaller digit values
//                    (prefix of the totals), those of the same value in earlier blocks
//                    (the scanned counts) and in earlier positions of this block (a stable
//                    rank: rounds of 256 keys in index order, ranked inside a warp with
//                    __match_any_sync and across the block's warps through shared counts).
// Passes cover the 32 depth bits and then the tile bits.  Equal (tile, depth) keys keep
// the order k_emit left them in, which its atomics make arbitrary, so k_radix_ties puts
// each run of equal keys in record order: the result is the (tile, depth, record) order
// of the per-tile sort, and each tile's pairs occupy the same range as before the sort
// (the range the scan of the tile counts gave it).  The number of pairs is read on the
// device (the grids cover the pair capacity; blocks past the last pair only count zeros).
#include "gs_internal.cuh"

namespace gsk {

namespace {

constexpr int kRxThreads = 256;
constexpr int kRxDigits = 256;
// Keys per thread per pass: 4 while that leaves at most kRxSmallBlocks blocks (small
// problems then still spread over the GPU), 16 above.
constexpr int kRxSmallBlocks = 4096;

__device__ __forceinline__ uint32_t pair_count(const DevHeader *hdr, uint32_t cap) {
    const unsigned long long n = hdr->n_pairs;
    return n < (unsigned long long)cap ? (uint32_t)n : cap;
}

// Exclusive scan of one value per thread over a block of kRxThreads; `total` gets the sum.
__device__ __forceinline__ uint32_t block_scan256(uint32_t x, uint32_t *warp_sum, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    uint32_t w = lane < kRxThreads / 32 ? warp_sum[lane] : 0u;
#pragma unroll
    for (int off = 1; off < kRxThreads / 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += v;
    }
    const uint32_t before = warp > 0 ? __shfl_sync(0xffffffffu, w, warp - 1) : 0u;
    total = __shfl_sync(0xffffffffu, w, kRxThreads / 32 - 1);
    __syncthreads();
    return before + incl - x;
}

template <int ITEMS>
__global__ void __launch_bounds__(kRxThreads) k_radix_hist(const unsigned long long *keys, const DevHeader *hdr,
                                                           uint32_t cap, int shift, uint32_t *hist, uint32_t nblk) {
    __shared__ uint32_t h[kRxDigits];
    const int tid = threadIdx.x;
    const uint32_t n = pair_count(hdr, cap);
    h[tid] = 0u;
    __syncthreads();
    const uint32_t base = blockIdx.x * (uint32_t)(kRxThreads * ITEMS);
#pragma unroll 4
    for (int r = 0; r < ITEMS; ++r) {
        const uint32_t i = base + (uint32_t)(r * kRxThreads + tid);
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[(size_t)tid * nblk + blockIdx.x] = h[tid];
}

// One block per digit value: its counts over the blocks become exclusive prefixes.
__global__ void __launch_bounds__(kRxThreads) k_radix_scan(uint32_t *hist, uint32_t nblk, uint32_t *total_out) {
    __shared__ uint32_t warp_sum[kRxThreads / 32];
    uint32_t *row = hist + (size_t)blockIdx.x * nblk;
    uint32_t run = 0;
    for (uint32_t b = 0; b < nblk; b += kRxThreads) {
        const uint32_t j = b + threadIdx.x;
        const uint32_t x = j < nblk ? row[j] : 0u;
        uint32_t total;
        const uint32_t excl = block_scan256(x, warp_sum, total);
        if (j < nblk) row[j] = run + excl;
        run += total;
    }
    if (threadIdx.x == 0) total_out[blockIdx.x] = run;
}

template <int ITEMS>
__global__ void __launch_bounds__(kRxThreads) k_radix_scatter(const unsigned long long *src_k, const uint32_t *src_v,
                                                              unsigned long long *dst_k, uint32_t *dst_v,
                                                              const DevHeader *hdr, uint32_t cap, int shift,
                                                              const uint32_t *hist, const uint32_t *total,
                                                              uint32_t nblk) {
    __shared__ uint32_t warp_sum[kRxThreads / 32];
    __shared__ uint32_t s_base[kRxDigits];               // destination of the next key of each value
    __shared__ uint32_t s_cnt[kRxThreads / 32][kRxDigits];  // per-warp counts of the current round
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = pair_count(hdr, cap);
    const uint32_t base = blockIdx.x * (uint32_t)(kRxThreads * ITEMS);
    if (base >= n) return;  // block-uniform
    {
        uint32_t all;
        const uint32_t before = block_scan256(total[tid], warp_sum, all);
        s_base[tid] = before + hist[(size_t)tid * nblk + blockIdx.x];
    }
    const unsigned int lt = (1u << lane) - 1u;
    for (int r = 0; r < ITEMS; ++r) {
        if (base + (uint32_t)(r * kRxThreads) >= n) break;  // block-uniform
#pragma unroll
        for (int w = 0; w < kRxThreads / 32; ++w) s_cnt[w][tid] = 0u;
        const uint32_t i = base + (uint32_t)(r * kRxThreads + tid);
        const bool live = i < n;
        unsigned long long key = 0ull;
        uint32_t val = 0u, dig = kRxDigits;  // kRxDigits: no key
        if (live) {
            key = src_k[i];
            val = src_v[i];
            dig = (uint32_t)(key >> shift) & 0xffu;
        }
        const unsigned int peers = __match_any_sync(0xffffffffu, dig);
        const uint32_t rank = (uint32_t)__popc(peers & lt);
        __syncthreads();  // s_cnt zeroed, s_base of the previous round settled
        if (live && rank == 0) s_cnt[warp][dig] = (uint32_t)__popc(peers);
        __syncthreads();
        if (live) {
            uint32_t off = s_base[dig] + rank;
            for (int w = 0; w < warp; ++w) off += s_cnt[w][dig];
            dst_k[off] = key;
            dst_v[off] = val;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < kRxThreads / 32; ++w) add += s_cnt[w][tid];
        s_base[tid] += add;
    }
}

// Runs of equal (tile, depth) keys put in record order; writes every value to `sorted`.
__global__ void __launch_bounds__(kRxThreads) k_radix_ties(const unsigned long long *keys, const uint32_t *vals,
                                                           uint32_t *sorted, const DevHeader *hdr, uint32_t cap) {
    const uint32_t n = pair_count(hdr, cap);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = keys[i];
    if (i > 0 && keys[i - 1] == k) return;  // inside a run: its first entry's thread writes it
    uint32_t end = i + 1;
    while (end < n && keys[end] == k) ++end;
    if (end == i + 1) {
        sorted[i] = vals[i];
        return;
    }
    // insertion sort of the run's records (runs are a few entries: duplicated depths)
    for (uint32_t a = i; a < end; ++a) {
        const uint32_t v = vals[a];
        uint32_t b = a;
        while (b > i && sorted[b - 1] > v) {
            sorted[b] = sorted[b - 1];
            --b;
        }
        sorted[b] = v;
    }
}

}  // namespace

int radix_items(uint32_t pair_cap) {
    return (pair_cap + 4u * kRxThreads - 1) / (4u * kRxThreads) <= (uint32_t)kRxSmallBlocks ? 4 : 16;
}

uint32_t radix_blocks(uint32_t pair_cap) {
    const uint32_t tile = (uint32_t)(kRxThreads * radix_items(pair_cap));
    return (pair_cap + tile - 1) / tile;
}

int radix_passes(uint32_t tiles) {
    int tile_bits = 0;
    while (tile_bits < 32 && (1ull << tile_bits) < (unsigned long long)tiles) ++tile_bits;
    return 4 + (tile_bits + 7) / 8;
}

cudaError_t launch_radix_sort(const RadixLaunch &L, cudaStream_t st) {
    const uint32_t nblk = radix_blocks(L.d.pair_cap);
    if (nblk == 0) return cudaSuccess;
    const int passes = radix_passes(L.d.T);
    const bool small = radix_items(L.d.pair_cap) == 4;
    unsigned long long *k[2] = {L.ws.keys, L.ws.rkeys};
    uint32_t *v[2] = {L.ws.sorted, L.ws.rvals};
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        const int s = p & 1, t = s ^ 1;
        if (small) k_radix_hist<4><<<nblk, kRxThreads, 0, st>>>(k[s], L.ws.hdr, L.d.pair_cap, shift, L.ws.rhist, nblk);
        else k_radix_hist<16><<<nblk, kRxThreads, 0, st>>>(k[s], L.ws.hdr, L.d.pair_cap, shift, L.ws.rhist, nblk);
        k_radix_scan<<<kRxDigits, kRxThreads, 0, st>>>(L.ws.rhist, nblk, L.ws.rtotal);
        if (small)
            k_radix_scatter<4><<<nblk, kRxThreads, 0, st>>>(k[s], v[s], k[t], v[t], L.ws.hdr, L.d.pair_cap, shift,
                                                            L.ws.rhist, L.ws.rtotal, nblk);
        else
            k_radix_scatter<16><<<nblk, kRxThreads, 0, st>>>(k[s], v[s], k[t], v[t], L.ws.hdr, L.d.pair_cap, shift,
                                                             L.ws.rhist, L.ws.rtotal, nblk);
    }
    const int f = passes & 1;
    k_radix_ties<<<(L.d.pair_cap + kRxThreads - 1) / kRxThreads, kRxThreads, 0, st>>>(k[f], v[f], L.ws.sorted,
                                                                                      L.ws.hdr, L.d.pair_cap);
    return cudaGetLastError();
}

}  // namespace gsk
