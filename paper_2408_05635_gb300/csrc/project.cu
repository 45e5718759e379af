// project.cu -- projection of every (Gaussian, view) pair, tile counting and key emission.
//
// k_project follows the projection of the paper: camera-frame mean R x + t (Sec. II-A),
// Sigma = Rg diag(s^2) Rg^T and Sigma' = J W Sigma W^T J^T (covariance formulas written
// in the source of Sec. I), mu' = pi_m(x_c) (Sec. II-A) and the 2-D footprint of Eq. 1.
// The support of a Gaussian is opacity-aware: o exp(-d^2/2) >= alpha_min holds exactly
// for Mahalanobis d^2 <= 2 ln(o / alpha_min), so tiles outside that ellipse can be
// skipped without changing a single pixel.
#include "gs_internal.cuh"

namespace gsk {

// Tile rectangle of a record's support ellipse.  The pixel box is derived from the
// stored conic (Sigma'_xx = c / det, Sigma'_yy = a / det of the conic); the one-pixel
// margin of tile_rect absorbs the error of the fast reciprocal and square root.  Both
// k_project (counting) and k_emit (writing) call exactly this code on the same floats,
// so they enumerate the same tiles.  Returns false when the box misses the image.
__device__ __forceinline__ bool record_rect(const ViewInfo &vi, float4 A, float4 B, int &tx0, int &tx1, int &ty0,
                                            int &ty1) {
    const float detc = diff_of_products(B.x, B.z, B.y, B.y);
    if (!(detc > 0.f)) return false;
    float hx = INFINITY, hy = INFINITY;
    if (B.w < INFINITY) {
        const float idet = __fdividef(1.f, detc);
        const float qx = __fmul_rn(B.w, __fmul_rn(B.z, idet)), qy = __fmul_rn(B.w, __fmul_rn(B.x, idet));
        hx = qx > 0.f ? __fmul_rn(qx, rsqrtf(qx)) : 0.f;
        hy = qy > 0.f ? __fmul_rn(qy, rsqrtf(qy)) : 0.f;
    }
    tile_rect(vi, A.x, A.y, hx, hy, tx0, tx1, ty0, ty1);
    return tx0 <= tx1 && ty0 <= ty1;
}

__device__ __forceinline__ bool tile_hit(const ViewInfo &vi, float4 A, float4 B, float ia, float ic, int tx, int ty) {
    float x0, x1, y0, y1;
    tile_bounds(vi, tx, ty, x0, x1, y0, y1);
    return ellipse_meets_rect(A.x, A.y, B.x, B.y, B.z, ia, ic, B.w, x0, x1, y0, y1);
}

// Tiles met by each lane's own record (mine = the lane has one).  A lane whose tile
// rectangle has at most kSoloTiles candidates tests them alone; larger rectangles (a
// Gaussian close to the camera can span thousands of tiles) are split over the 32 lanes
// of the warp, so one of them never holds the rest of the grid.  body(src lane, tile,
// record's A, record's tag) runs once for every tile the support meets.
constexpr int kSoloTiles = 24;

template <bool SOLO = true, class Body>
__device__ __forceinline__ void record_tiles(bool mine, const ViewInfo &vi, float4 A, float4 B, uint32_t tag, int lane,
                                             Body &&body) {
    int tx0 = 1, tx1 = 0, ty0 = 1, ty1 = 0;
    const bool has = mine && record_rect(vi, A, B, tx0, tx1, ty0, ty1);
    const int rw = tx1 - tx0 + 1;
    const int count = has ? rw * (ty1 - ty0 + 1) : 0;
    if (SOLO && has && count <= kSoloTiles) {
        const RowSpan span = row_span_setup(A.x, A.y, B.x, B.y, B.z, B.w);
        for (int ty = ty0; ty <= ty1; ++ty) {
            int a0, a1;
            row_span(vi, span, ty, tx0, tx1, a0, a1);
            for (int tx = a0; tx <= a1; ++tx) body(lane, vi.tile_base + (uint32_t)(ty * vi.tiles_x + tx), A, tag);
        }
    }
    uint32_t big = __ballot_sync(0xffffffffu, count > kSoloTiles);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        float4 As, Bs;
        As.x = __shfl_sync(0xffffffffu, A.x, src);
        As.y = __shfl_sync(0xffffffffu, A.y, src);
        As.z = __shfl_sync(0xffffffffu, A.z, src);
        As.w = __shfl_sync(0xffffffffu, A.w, src);
        Bs.x = __shfl_sync(0xffffffffu, B.x, src);
        Bs.y = __shfl_sync(0xffffffffu, B.y, src);
        Bs.z = __shfl_sync(0xffffffffu, B.z, src);
        Bs.w = __shfl_sync(0xffffffffu, B.w, src);
        const uint32_t tg = __shfl_sync(0xffffffffu, tag, src);
        const int sx0 = __shfl_sync(0xffffffffu, tx0, src), sy0 = __shfl_sync(0xffffffffu, ty0, src);
        const int srw = __shfl_sync(0xffffffffu, rw, src), scount = __shfl_sync(0xffffffffu, count, src);
        const float ia = __fdividef(1.f, Bs.x), ic = __fdividef(1.f, Bs.z);
        for (int t = lane; t < scount; t += 32) {
            const int ty = sy0 + t / srw, tx = sx0 + t % srw;
            if (tile_hit(vi, As, Bs, ia, ic, tx, ty)) body(src, vi.tile_base + (uint32_t)(ty * vi.tiles_x + tx), As, tg);
        }
    }
}

struct ViewChunk {
    ViewInfo v[32];
};

// Copies up to 32 views into the device table (block 0) and zeroes `zero_words` 32-bit
// words at `zero` (all blocks, grid-stride): the per-call reset of the flag word, the
// header and the tile counters, folded into the same launch.
__global__ void k_copy_views(ViewInfo *dst, int count, ViewChunk chunk, uint32_t *zero, size_t zero_words) {
    // the projection may be scheduled now: it waits (griddep_wait) for this grid to end
    // before it touches the workspace
    griddep_launch_dependents();
    if (blockIdx.x == 0 && threadIdx.x < count) dst[threadIdx.x] = chunk.v[threadIdx.x];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < zero_words; i += (size_t)gridDim.x * blockDim.x)
        zero[i] = 0u;
}

cudaError_t launch_upload_views(const ViewInfo *host_views, int V, ViewInfo *dev, void *zero, size_t zero_bytes,
                                cudaStream_t st) {
    constexpr int kThreads = 256;
    for (int base = 0; base < V || (base == 0 && zero_bytes); base += 32) {
        ViewChunk c;
        const int cnt = V - base < 32 ? (V - base > 0 ? V - base : 0) : 32;
        for (int k = 0; k < cnt; ++k) c.v[k] = host_views[base + k];
        const size_t words = base == 0 ? zero_bytes / 4 : 0;
        size_t blocks = (words + 4 * kThreads - 1) / (4 * kThreads);
        blocks = blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks);
        k_copy_views<<<(unsigned)blocks, kThreads, 0, st>>>(dev + base, cnt, c, static_cast<uint32_t *>(zero), words);
    }
    return cudaGetLastError();
}

// Exclusive scan of the per-(tile, sub-bucket) counts into list offsets, by one block of
// kScanThreads.  Each pass loads kScanPer contiguous counters per thread in one round
// (and zeroes them for the next projection), scans the per-thread totals across the
// block and writes the offsets.  Since S divides kScanPer, a tile's S counters sit in
// one thread, which also counts the tile's list length into the buckets of the
// longest-first launch order; the lengths stay in registers when one pass covers all
// counters.  Also: the total pair count, the longest list and the number of records.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kOrderBuckets = kScanThreads;  // list lengths >= kOrderBuckets - 1 share the first bucket

__device__ __forceinline__ uint32_t order_bucket(uint32_t len) {
    return kOrderBuckets - 1 - min(len, (uint32_t)kOrderBuckets - 1);
}

// Exclusive block-wide scan of one value per thread; `total` gets the block sum.  Uses
// warp_sum (kScanThreads / 32 words) and ends with a barrier.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *warp_sum, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    uint32_t wi = lane < kScanThreads / 32 ? warp_sum[lane] : 0u;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, wi, off);
        if (lane >= off) wi += v;
    }
    const uint32_t prev = __shfl_sync(0xffffffffu, wi, (warp + 31) & 31);
    total = __shfl_sync(0xffffffffu, wi, kScanThreads / 32 - 1);
    __syncthreads();
    return (warp > 0 ? prev : 0u) + incl - x;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(WsPtrs ws, Dims d) {
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    __shared__ uint32_t warp_sum[kScanThreads / 32];
    __shared__ uint32_t s_bucket[kOrderBuckets];
    __shared__ uint32_t s_max;
    __shared__ unsigned long long s_recs;
    const uint32_t TS = d.T * d.S, S = d.S, smask = d.S - 1, sshift = __ffs(d.S) - 1;  // S: 1, 2 or 4
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        s_max = 0;
        s_recs = 0;
    }
    s_bucket[tid] = 0;
    // record counts of the first cells, fetched now so their latency overlaps the scan
    const uint32_t ncell = (uint32_t)d.V * (uint32_t)d.nblk;
    uint32_t cc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t c = (uint32_t)tid + (uint32_t)k * kScanThreads;
        cc[k] = c < ncell ? ws.cell_cnt[c] : 0u;
    }
    __syncthreads();
    const bool one_pass = TS <= (uint32_t)kScanThreads * kScanPer;
    uint32_t len[kScanPer];  // length of the tile whose first counter is j (j % S == 0)
    unsigned long long carry = 0;  // identical in every thread
    uint32_t max_tile = 0;
    for (uint32_t base = 0; base < TS; base += (uint32_t)kScanThreads * kScanPer) {
        const uint32_t i0 = base + (uint32_t)tid * kScanPer;
        uint32_t c[kScanPer];
        if (i0 + kScanPer <= TS) {
            uint4 *q = reinterpret_cast<uint4 *>(ws.tile_cnt + i0);
            const uint4 a = q[0], b = q[1];
            c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
            c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
            q[0] = make_uint4(0u, 0u, 0u, 0u);
            q[1] = make_uint4(0u, 0u, 0u, 0u);
        } else {
#pragma unroll
            for (int k = 0; k < kScanPer; ++k) {
                c[k] = i0 + k < TS ? ws.tile_cnt[i0 + k] : 0u;
                if (i0 + k < TS) ws.tile_cnt[i0 + k] = 0u;
            }
        }
        uint32_t mine = 0;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) mine += c[k];
        uint32_t total;
        const uint32_t excl = block_exclusive_scan(mine, warp_sum, total);
        unsigned long long run = carry + excl;
        uint32_t o[kScanPer];
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            o[k] = (uint32_t)min(run, (unsigned long long)0xffffffffu);
            run += c[k];
        }
        if (i0 + kScanPer <= TS) {  // whole 32-byte rows: two vector stores per array
            const uint4 a = make_uint4(o[0], o[1], o[2], o[3]), b = make_uint4(o[4], o[5], o[6], o[7]);
            reinterpret_cast<uint4 *>(ws.tile_start + i0)[0] = a;
            reinterpret_cast<uint4 *>(ws.tile_start + i0)[1] = b;
            reinterpret_cast<uint4 *>(ws.cursor + i0)[0] = a;
            reinterpret_cast<uint4 *>(ws.cursor + i0)[1] = b;
        } else {
#pragma unroll
            for (int k = 0; k < kScanPer; ++k)
                if (i0 + k < TS) {
                    ws.tile_start[i0 + k] = o[k];
                    ws.cursor[i0 + k] = o[k];
                }
        }
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            len[j] = 0;
            if ((j & smask) == 0 && i0 + j < TS) {
                uint32_t l = c[j];
                if (S > 1) l += c[(j + 1) % kScanPer];
                if (S > 2) l += c[(j + 2) % kScanPer] + c[(j + 3) % kScanPer];
                len[j] = l;
                max_tile = max(max_tile, l);
                atomicAdd(&s_bucket[order_bucket(l)], 1u);
            }
        }
        carry += total;
    }
    if (tid == 0) {
        ws.tile_start[TS] = (uint32_t)min(carry, (unsigned long long)0xffffffffu);
        ws.hdr->n_big = ws.tile_cnt[TS];  // the large records k_project listed, zeroed for the next pass
        ws.tile_cnt[TS] = 0u;
    }
    __syncthreads();
    {  // exclusive scan of the buckets, one bucket per thread
        uint32_t total;
        const uint32_t c = s_bucket[tid];
        const uint32_t excl = block_exclusive_scan(c, warp_sum, total);
        s_bucket[tid] = excl;
    }
    __syncthreads();
    if (one_pass) {
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const uint32_t i = (uint32_t)tid * kScanPer + (uint32_t)j;
            if ((j & smask) == 0 && i < TS) ws.tile_order[atomicAdd(&s_bucket[order_bucket(len[j])], 1u)] = i >> sshift;
        }
    } else {
        for (uint32_t t = tid; t < d.T; t += kScanThreads) {
            const uint32_t l = ws.tile_start[(t + 1) * S] - ws.tile_start[t * S];
            ws.tile_order[atomicAdd(&s_bucket[order_bucket(l)], 1u)] = t;
        }
    }
    unsigned long long recs = (unsigned long long)cc[0] + cc[1] + cc[2] + cc[3];
    for (uint32_t c = (uint32_t)tid + 4u * kScanThreads; c < ncell; c += kScanThreads) recs += ws.cell_cnt[c];
    max_tile = __reduce_max_sync(0xffffffffu, max_tile);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) recs += __shfl_xor_sync(0xffffffffu, recs, off);
    if (lane == 0) {
        atomicMax(&s_max, max_tile);
        atomicAdd(&s_recs, recs);
    }
    __syncthreads();
    if (tid == 0) {
        ws.hdr->max_tile = s_max;
        ws.hdr->n_rec = s_recs;
        ws.hdr->n_pairs = carry;
        if (carry > d.pair_cap) atomicOr(ws.err, (uint32_t)kErrPairs);
    }
}

// ------------------------------------------------------------ multi-block form of the scan
// For problems with more counters than one block covers in one pass (many views or small
// tiles), three kernels: (1) each block of kMBThreads sums a chunk of kMBChunk counters,
// counts its tiles into kMBuckets launch-order buckets (list length / 16, the longest
// first), and sums a slice of the cells' record counts; (2) one block turns the chunk sums
// and the bucket counts (bucket-major, so a bucket's blocks are consecutive) into
// exclusive offsets, and writes the totals to the header; (3) each block scans its chunk
// again from its offset, writes the list offsets and cursors, zeroes the counters, and
// places its tiles in the launch order from its buckets' offsets.  The per-block arrays
// live in ws.scan_part: sums, longest lists, record counts (NB each), then the bucket
// counts (kMBuckets x NB).

__device__ __forceinline__ uint32_t mb_bucket(uint32_t len) {
    return kMBuckets - 1 - min(len >> 4, (uint32_t)kMBuckets - 1);
}

// Exclusive scan of one value per thread over a block of NT threads (NT / 32 <= 32 warps);
// `total` gets the block sum.  Ends with a barrier.
template <int NT, class T>
__device__ __forceinline__ T block_scan_excl(T x, T *warp_sum, T &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    T wi = lane < NT / 32 ? warp_sum[lane] : T(0);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T v = __shfl_up_sync(0xffffffffu, wi, off);
        if (lane >= off) wi += v;
    }
    const T prev = __shfl_sync(0xffffffffu, wi, (warp + 31) & 31);
    total = __shfl_sync(0xffffffffu, wi, NT / 32 - 1);
    __syncthreads();
    return (warp > 0 ? prev : T(0)) + incl - x;
}

// This thread's kMBPer counters of chunk position i0 (vector loads where the run is whole).
__device__ __forceinline__ void load_counts(const uint32_t *cnt, uint32_t i0, uint32_t TS, uint32_t (&c)[kMBPer]) {
    if (i0 + kMBPer <= TS) {
        const uint4 *q = reinterpret_cast<const uint4 *>(cnt + i0);
        const uint4 a = q[0], b = q[1];
        c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
        c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < kMBPer; ++k) c[k] = i0 + k < TS ? cnt[i0 + k] : 0u;
    }
}

__global__ void __launch_bounds__(kMBThreads) k_scan_part(WsPtrs ws, Dims d) {
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    __shared__ uint32_t s_hist[kMBuckets], s_sum, s_max, s_rec;
    const uint32_t TS = d.T * d.S, smask = d.S - 1, NB = gridDim.x, b = blockIdx.x;
    const int tid = threadIdx.x;
    if (tid < kMBuckets) s_hist[tid] = 0u;
    if (tid == 0) s_sum = s_max = s_rec = 0u;
    __syncthreads();
    uint32_t c[kMBPer];
    const uint32_t i0 = b * kMBChunk + (uint32_t)tid * kMBPer;
    load_counts(ws.tile_cnt, i0, TS, c);
    uint32_t mine = 0, mx = 0;
#pragma unroll
    for (int j = 0; j < kMBPer; ++j) {
        mine += c[j];
        if ((j & smask) == 0 && i0 + j < TS) {  // the S counters of a tile sit in one thread
            uint32_t l = c[j];
            if (d.S > 1) l += c[(j + 1) % kMBPer];
            if (d.S > 2) l += c[(j + 2) % kMBPer] + c[(j + 3) % kMBPer];
            mx = max(mx, l);
            atomicAdd(&s_hist[mb_bucket(l)], 1u);
        }
    }
    const uint32_t ncell = (uint32_t)d.V * (uint32_t)d.nblk, cpb = (ncell + NB - 1) / NB;
    uint32_t rec = 0;
    for (uint32_t k = b * cpb + (uint32_t)tid; k < min(ncell, (b + 1) * cpb); k += kMBThreads) rec += ws.cell_cnt[k];
    mine = __reduce_add_sync(0xffffffffu, mine);
    mx = __reduce_max_sync(0xffffffffu, mx);
    rec = __reduce_add_sync(0xffffffffu, rec);
    if ((tid & 31) == 0) {
        atomicAdd(&s_sum, mine);
        atomicMax(&s_max, mx);
        atomicAdd(&s_rec, rec);
    }
    __syncthreads();
    uint32_t *part = ws.scan_part;
    if (tid == 0) {
        part[b] = s_sum;
        part[NB + b] = s_max;
        part[2 * NB + b] = s_rec;
    }
    if (tid < kMBuckets) part[3 * NB + (uint32_t)tid * NB + b] = s_hist[tid];
}

// In-place exclusive scan of a[0, n) by one block of kScanThreads (each thread a
// contiguous run); returns the total to every thread.  Sums saturate at 2^32 - 1 where
// they are stored.
__device__ __forceinline__ unsigned long long block_scan_array(uint32_t *a, uint32_t n,
                                                               unsigned long long *warp_sum) {
    const uint32_t per = (n + kScanThreads - 1) / kScanThreads, lo = min(n, (uint32_t)threadIdx.x * per),
                   hi = min(n, lo + per);
    unsigned long long sum = 0;
    for (uint32_t i = lo; i < hi; ++i) sum += a[i];
    unsigned long long total;
    unsigned long long run = block_scan_excl<kScanThreads>(sum, warp_sum, total);
    for (uint32_t i = lo; i < hi; ++i) {
        const uint32_t v = a[i];
        a[i] = (uint32_t)min(run, (unsigned long long)0xffffffffu);
        run += v;
    }
    return total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(WsPtrs ws, Dims d) {
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    __shared__ unsigned long long warp_sum[kScanThreads / 32];
    __shared__ uint32_t s_max;
    __shared__ unsigned long long s_rec;
    const uint32_t TS = d.T * d.S, NB = (TS + kMBChunk - 1) / kMBChunk;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_max = 0u;
        s_rec = 0ull;
    }
    uint32_t *part = ws.scan_part;
    const unsigned long long total = block_scan_array(part, NB, warp_sum);  // chunk offsets
    block_scan_array(part + 3 * NB, kMBuckets * NB, warp_sum);              // launch-order offsets
    uint32_t mx = 0;
    unsigned long long rec = 0;
    for (uint32_t i = (uint32_t)tid; i < NB; i += kScanThreads) {
        mx = max(mx, part[NB + i]);
        rec += part[2 * NB + i];
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rec += __shfl_xor_sync(0xffffffffu, rec, off);
    if ((tid & 31) == 0) {
        atomicMax(&s_max, mx);
        atomicAdd(&s_rec, rec);
    }
    __syncthreads();
    if (tid == 0) {
        ws.tile_start[TS] = (uint32_t)min(total, (unsigned long long)0xffffffffu);
        ws.hdr->n_big = ws.tile_cnt[TS];  // the large records k_project listed, zeroed for the next pass
        ws.tile_cnt[TS] = 0u;
        ws.hdr->max_tile = s_max;
        ws.hdr->n_rec = s_rec;
        ws.hdr->n_pairs = total;
        if (total > d.pair_cap) atomicOr(ws.err, (uint32_t)kErrPairs);
    }
}

__global__ void __launch_bounds__(kMBThreads) k_scan_write(WsPtrs ws, Dims d) {
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    __shared__ uint32_t warp_sum[kMBThreads / 32], s_pos[kMBuckets];
    const uint32_t TS = d.T * d.S, smask = d.S - 1, sshift = __ffs(d.S) - 1, NB = gridDim.x, b = blockIdx.x;
    const int tid = threadIdx.x;
    const uint32_t *part = ws.scan_part;
    if (tid < kMBuckets) s_pos[tid] = part[3 * NB + (uint32_t)tid * NB + b];
    uint32_t c[kMBPer];
    const uint32_t i0 = b * kMBChunk + (uint32_t)tid * kMBPer;
    load_counts(ws.tile_cnt, i0, TS, c);
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < kMBPer; ++k) mine += c[k];
    uint32_t total;
    const uint32_t excl = block_scan_excl<kMBThreads>(mine, warp_sum, total);  // (ends with a barrier)
    unsigned long long run = (unsigned long long)part[b] + excl;
    uint32_t o[kMBPer];
#pragma unroll
    for (int k = 0; k < kMBPer; ++k) {
        o[k] = (uint32_t)min(run, (unsigned long long)0xffffffffu);
        run += c[k];
    }
    if (i0 + kMBPer <= TS) {  // whole 32-byte rows: two vector stores per array
        const uint4 a = make_uint4(o[0], o[1], o[2], o[3]), e = make_uint4(o[4], o[5], o[6], o[7]);
        reinterpret_cast<uint4 *>(ws.tile_start + i0)[0] = a;
        reinterpret_cast<uint4 *>(ws.tile_start + i0)[1] = e;
        reinterpret_cast<uint4 *>(ws.cursor + i0)[0] = a;
        reinterpret_cast<uint4 *>(ws.cursor + i0)[1] = e;
        reinterpret_cast<uint4 *>(ws.tile_cnt + i0)[0] = make_uint4(0u, 0u, 0u, 0u);
        reinterpret_cast<uint4 *>(ws.tile_cnt + i0)[1] = make_uint4(0u, 0u, 0u, 0u);
    } else {
#pragma unroll
        for (int k = 0; k < kMBPer; ++k)
            if (i0 + k < TS) {
                ws.tile_start[i0 + k] = o[k];
                ws.cursor[i0 + k] = o[k];
                ws.tile_cnt[i0 + k] = 0u;
            }
    }
#pragma unroll
    for (int j = 0; j < kMBPer; ++j) {
        if ((j & smask) == 0 && i0 + j < TS) {
            uint32_t l = c[j];
            if (d.S > 1) l += c[(j + 1) % kMBPer];
            if (d.S > 2) l += c[(j + 2) % kMBPer] + c[(j + 3) % kMBPer];
            ws.tile_order[atomicAdd(&s_pos[mb_bucket(l)], 1u)] = (i0 + (uint32_t)j) >> sshift;
        }
    }
}

// Up to four passes of the one-block scan take less than the three launches of the
// multi-block form.
constexpr uint64_t kMultiBlockScanFrom = 4ull * kScanThreads * kScanPer;

cudaError_t launch_scan_tiles(const WsPtrs &ws, const Dims &d, cudaStream_t st) {
    const uint64_t TS = (uint64_t)d.T * d.S;
    if (TS <= kMultiBlockScanFrom || !ws.scan_part)
        return launch_dep(k_scan_tiles, dim3(1), dim3(kScanThreads), st, ws, d);
    const uint32_t NB = scan_blocks(TS);
    cudaError_t e = launch_dep(k_scan_part, dim3(NB), dim3(kMBThreads), st, ws, d);
    if (e == cudaSuccess) e = launch_dep(k_scan_top, dim3(1), dim3(kScanThreads), st, ws, d);
    if (e == cudaSuccess) e = launch_dep(k_scan_write, dim3(NB), dim3(kMBThreads), st, ws, d);
    return e;
}

// A block's large records (more than kSoloTiles candidate tiles) are counted by all its
// threads at once, each taking (record, tile) pairs of their concatenated rectangles,
// instead of one record after the other by the warp that holds it; kBigPerBlock of them,
// a further one by its warp.
constexpr int kBigPerBlock = 64;

template <int DT, bool ISO>
__global__ void __launch_bounds__(kBlock, 6) k_project(ProjectLaunch L) {
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    const int v = blockIdx.y, b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    __shared__ float sRt[12];
    __shared__ ViewInfo sv;
    __shared__ uint32_t warp_off[kWarps];
    __shared__ float4 sbA[kBigPerBlock], sbB[kBigPerBlock];
    __shared__ int4 sbR[kBigPerBlock];         // first tile column and row, columns, candidates
    __shared__ uint32_t sbPre[kBigPerBlock + 1], sbSub[kBigPerBlock], s_nbig;
    const uint32_t cell = (uint32_t)v * (uint32_t)L.d.nblk + (uint32_t)b;
    if (tid == 0) {
        load_pose(L.poses + 7 * v, sRt);
        sv = L.ws.views[v];
        s_nbig = 0u;
    }
    __syncthreads();
    if (b == 0 && tid < 12) L.ws.view_rt[12 * v + tid] = sRt[tid];
    // per-iteration counters start at zero (nothing else touches the header before the scan)
    if (b == 0 && v == 0 && tid < (int)(sizeof(DevHeader) / 8))
        reinterpret_cast<unsigned long long *>(L.ws.hdr)[tid] = 0ull;
    const ViewInfo vi = sv;
    const int64_t i = (int64_t)b * kBlock + tid;
    const Settings &S = L.s;
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A, C = A;
    bool vis = false, big = false;
    int4 rect = make_int4(0, 0, 0, 0);
    if (i < L.d.n) {
        const float mx = __ldg(L.g.means + 3 * i), my = __ldg(L.g.means + 3 * i + 1), mz = __ldg(L.g.means + 3 * i + 2);
        const float x = cam_coord(sRt, 0, mx, my, mz);
        const float y = cam_coord(sRt, 1, mx, my, mz);
        const float z = cam_coord(sRt, 2, mx, my, mz);
        bool reach = z > S.z_near;
        if (reach && S.alpha_min > 0.f) {
            // Early reject of a Gaussian whose support cannot reach the image, before the
            // covariance (it pays off when a warp's Gaussians are spatial neighbours, as in a
            // map built frame by frame): Sigma'_xx = |J0 M|^2 + e <= |J0|^2 s_max^2 + e
            // (M = W Rg diag(s), W and Rg orthonormal; J0 the first row of the clamped
            // Jacobian) and the support radius^2 is at most 2 ln(1 / alpha_min).  Widened by
            // 1 % and 3 px, so a Gaussian dropped here would also fail record_rect's box test.
            float lsm;
            if constexpr (ISO) {
                lsm = ld_attr<DT>(L.g.log_scales, i);
            } else {
                lsm = fmaxf(fmaxf(ld_attr<DT>(L.g.log_scales, 3 * i), ld_attr<DT>(L.g.log_scales, 3 * i + 1)),
                            ld_attr<DT>(L.g.log_scales, 3 * i + 2));
            }
            const float sm2 = __expf(2.f * lsm);
            const float iz = __fdividef(1.f, z);
            const float tx = fminf(fmaxf(x * iz, -vi.tan_lim_x), vi.tan_lim_x);
            const float ty = fminf(fmaxf(y * iz, -vi.tan_lim_y), vi.tan_lim_y);
            const float r2 = -2.f * __logf(S.alpha_min);
            const float hx = 1.01f * sqrtf(r2 * (vi.fx * vi.fx * iz * iz * (1.f + tx * tx) * sm2 + S.dilation)) + 3.f;
            const float hy = 1.01f * sqrtf(r2 * (vi.fy * vi.fy * iz * iz * (1.f + ty * ty) * sm2 + S.dilation)) + 3.f;
            const float mu_x = vi.fx * x * iz + vi.cx, mu_y = vi.fy * y * iz + vi.cy;
            reach = mu_x + hx >= 0.f && mu_x - hx <= (float)(vi.width - 1) && mu_y + hy >= 0.f &&
                    mu_y - hy <= (float)(vi.height - 1);
        }
        if (reach) {
            // M = W Rg diag(s): Sigma_c = M M^T (isotropic: M = s W)
            float M[9];
            if constexpr (ISO) {
                const float sc = __expf(ld_attr<DT>(L.g.log_scales, i));
#pragma unroll
                for (int k = 0; k < 9; ++k) M[k] = sRt[k] * sc;
            } else {
                float qw = ld_attr<DT>(L.g.quats, 4 * i), qx = ld_attr<DT>(L.g.quats, 4 * i + 1);
                float qy = ld_attr<DT>(L.g.quats, 4 * i + 2), qz = ld_attr<DT>(L.g.quats, 4 * i + 3);
                const float qq = qw * qw + qx * qx + qy * qy + qz * qz;
                const float qi = qq > 0.f ? rsqrtf(qq) : 0.f;
                qw *= qi; qx *= qi; qy *= qi; qz *= qi;
                float Rg[9];
                quat_to_rot(qw, qx, qy, qz, Rg);
                const float s0 = __expf(ld_attr<DT>(L.g.log_scales, 3 * i));
                const float s1 = __expf(ld_attr<DT>(L.g.log_scales, 3 * i + 1));
                const float s2 = __expf(ld_attr<DT>(L.g.log_scales, 3 * i + 2));
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    M[3 * r + 0] = (sRt[3 * r] * Rg[0] + sRt[3 * r + 1] * Rg[3] + sRt[3 * r + 2] * Rg[6]) * s0;
                    M[3 * r + 1] = (sRt[3 * r] * Rg[1] + sRt[3 * r + 1] * Rg[4] + sRt[3 * r + 2] * Rg[7]) * s1;
                    M[3 * r + 2] = (sRt[3 * r] * Rg[2] + sRt[3 * r + 1] * Rg[5] + sRt[3 * r + 2] * Rg[8]) * s2;
                }
            }
            const float iz = __fdividef(1.f, z);
            // J at the mean's image-plane tangent, clamped to the view's limits
            const float tx = fminf(fmaxf(x * iz, -vi.tan_lim_x), vi.tan_lim_x);
            const float ty = fminf(fmaxf(y * iz, -vi.tan_lim_y), vi.tan_lim_y);
            const float J00 = vi.fx * iz, J02 = -vi.fx * tx * iz;
            const float J11 = vi.fy * iz, J12 = -vi.fy * ty * iz;
            // N = J M, Sigma' = N N^T + dilation I
            float N0[3], N1[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                N0[c] = J00 * M[c] + J02 * M[6 + c];
                N1[c] = J11 * M[3 + c] + J12 * M[6 + c];
            }
            const float S00 = N0[0] * N0[0] + N0[1] * N0[1] + N0[2] * N0[2] + S.dilation;
            const float S01 = N0[0] * N1[0] + N0[1] * N1[1] + N0[2] * N1[2];
            const float S11 = N1[0] * N1[0] + N1[1] * N1[1] + N1[2] * N1[2] + S.dilation;
            // det(N N^T + e I) = |N0 x N1|^2 + e (S00 + S11) - e^2 (Cauchy-Binet): a sum of
            // squares, where S00 S11 - S01^2 cancels catastrophically once the footprint is
            // thin (N0, N1 nearly parallel: a Gaussian seen edge-on or close to the camera)
            const float cx = diff_of_products(N0[1], N1[2], N0[2], N1[1]);
            const float cy = diff_of_products(N0[2], N1[0], N0[0], N1[2]);
            const float cz = diff_of_products(N0[0], N1[1], N0[1], N1[0]);
            const float det = cx * cx + cy * cy + cz * cz + S.dilation * (S00 + S11 - S.dilation);
            if (det > 0.f) {
                const float idet = __fdividef(1.f, det);
                const float o = __fdividef(1.f, 1.f + __expf(-ld_attr<DT>(L.g.logits, i)));
                float dmax2;
                if (S.alpha_min > 0.f)
                    dmax2 = o >= S.alpha_min ? 2.f * __logf(__fdividef(o, S.alpha_min)) : -1.f;
                else
                    dmax2 = INFINITY;
                if (dmax2 >= 0.f) {
                    A = make_float4(vi.fx * x * iz + vi.cx, vi.fy * y * iz + vi.cy, z, o);
                    B = make_float4(S11 * idet, -S01 * idet, S00 * idet, dmax2);
                    C = make_float4(ld_attr<DT>(L.g.rgb, 3 * i), ld_attr<DT>(L.g.rgb, 3 * i + 1),
                                    ld_attr<DT>(L.g.rgb, 3 * i + 2),
                                    __uint_as_float((uint32_t)((int64_t)v * L.d.n + i)));
                    int tx0, tx1, ty0, ty1;
                    vis = record_rect(vi, A, B, tx0, tx1, ty0, ty1);
                    big = vis && (tx1 - tx0 + 1) * (ty1 - ty0 + 1) > kSoloTiles;
                    rect = make_int4(tx0, ty0, tx1 - tx0 + 1, (tx1 - tx0 + 1) * (ty1 - ty0 + 1));
                }
            }
        }
    }
    // compaction into this block's cell: visible Gaussians take the first slots, in order
    const uint32_t ballot = __ballot_sync(0xffffffffu, vis);
    if (lane == 0) warp_off[warp] = __popc(ballot);
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = warp_off[w];
            warp_off[w] = run;
            run += c;
        }
        L.ws.cell_cnt[cell] = run;
    }
    // the block's large records, for the block-wide count below
    const uint32_t nsub = L.d.S;
    bool mine_solo = vis;
    if (big) {
        const uint32_t k = atomicAdd(&s_nbig, 1u);
        if (k < (uint32_t)kBigPerBlock) {
            sbA[k] = A;
            sbB[k] = B;
            sbR[k] = rect;
            sbSub[k] = (uint32_t)i & (nsub - 1);
            mine_solo = false;
        }
    }
    __syncthreads();
    if (vis) {
        const uint32_t rec = cell * kCell + warp_off[warp] + __popc(ballot & ((1u << lane) - 1u));
        Rec r;
        r.a = A; r.b = B; r.c = C;
        L.ws.rec[rec] = r;
        RecGrad z;
        z.g0 = z.g1 = z.g2 = make_float4(0.f, 0.f, 0.f, 0.f);
        L.ws.rec_grad[rec] = z;
        // the large records of a cell that holds kBigCell or more: listed for k_emit's extra
        // blocks while the list has room (the cell's warps emit the others)
        uint8_t listed = 0;
        if (big && s_nbig >= (uint32_t)kBigCell) {
            const uint32_t k = atomicAdd(L.ws.tile_cnt + L.d.T * L.d.S, 1u);
            if (k < (uint32_t)kBigListCap) {
                L.ws.big[k] = rec;
                listed = 1;
            }
        }
        L.ws.big_listed[rec] = listed;
    }
    // per-(tile, sub-bucket) pair counts: the block's listed large records by all threads,
    // every other visible record by its own lane (or, above kSoloTiles, its warp)
    uint32_t *cnt = L.ws.tile_cnt;
    const uint32_t nbig = min(s_nbig, (uint32_t)kBigPerBlock);  // block-uniform
    if (nbig) {
        if (warp == 0) {  // exclusive prefix of the rectangles' candidate counts
            uint32_t run = 0;
            for (uint32_t base = 0; base < nbig; base += 32) {
                const uint32_t e = base + (uint32_t)lane;
                const uint32_t c = e < nbig ? (uint32_t)sbR[e].w : 0u;
                uint32_t incl = c;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += y;
                }
                if (e < nbig) sbPre[e] = run + incl - c;
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) sbPre[nbig] = run;
        }
        __syncthreads();
        const uint32_t total = sbPre[nbig];
        for (uint32_t f = (uint32_t)tid; f < total; f += kBlock) {
            int lo = 0, hi = (int)nbig - 1;  // the last entry whose prefix is at most f
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sbPre[mid] <= f) lo = mid; else hi = mid - 1;
            }
            const int4 R = sbR[lo];
            const int t = (int)(f - sbPre[lo]);
            const int ty = R.y + t / R.z, tx = R.x + t % R.z;
            const float4 Ab = sbA[lo], Bb = sbB[lo];
            if (tile_hit(vi, Ab, Bb, __fdividef(1.f, Bb.x), __fdividef(1.f, Bb.z), tx, ty))
                red_add(cnt + (vi.tile_base + (uint32_t)(ty * vi.tiles_x + tx)) * nsub + sbSub[lo], 1u);
        }
    }
    record_tiles(mine_solo, vi, A, B, (uint32_t)i & (nsub - 1), lane, [&](int, uint32_t tile, float4, uint32_t sub) {
        red_add(cnt + tile * nsub + sub, 1u);
    });
}

cudaError_t launch_project(const ProjectLaunch &L, cudaStream_t st) {
    dim3 grid(L.d.nblk, L.d.V);
    const bool iso = L.g.quats == nullptr;  // isotropic Gaussians: one log-radius, no rotation
    cudaError_t e;
    switch (L.dtype) {
        case GS_F32:
            if (iso) e = launch_dep(k_project<GS_F32, true>, grid, dim3(kBlock), st, L);
            else e = launch_dep(k_project<GS_F32, false>, grid, dim3(kBlock), st, L);
            break;
        case GS_BF16:
            if (iso) e = launch_dep(k_project<GS_BF16, true>, grid, dim3(kBlock), st, L);
            else e = launch_dep(k_project<GS_BF16, false>, grid, dim3(kBlock), st, L);
            break;
        case GS_F16:
            if (iso) e = launch_dep(k_project<GS_F16, true>, grid, dim3(kBlock), st, L);
            else e = launch_dep(k_project<GS_F16, false>, grid, dim3(kBlock), st, L);
            break;
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Write one (record, tile) pair at its slot: for the per-tile sort the key depth bits << 32 |
// record; for the device-wide radix sort (GS_SCHED_RADIX) the key tile << 32 | depth bits
// with the record as the value.  Depths are positive, so their bits order as unsigned.
__device__ __forceinline__ void put_pair(const WsPtrs &ws, bool radix, uint32_t slot, uint32_t tile, uint32_t depth_bits,
                                         uint32_t rec) {
    if (radix) {
        ws.keys[slot] = ((unsigned long long)tile << 32) | depth_bits;
        ws.sorted[slot] = rec;
    } else {
        ws.keys[slot] = ((unsigned long long)depth_bits << 32) | rec;
    }
}

// The emission runs kEmitThreads threads per block, kCell / kEmitThreads blocks per cell,
// compiled for kEmitMinBlocks resident blocks per SM (64 registers a thread).
constexpr int kEmitThreads = 64;
constexpr int kEmitMinBlocks = 16;
static_assert(kCell % kEmitThreads == 0 && kEmitThreads % 32 == 0, "emission blocks split cells into warps");

// One key per (record, tile met): depth bits (positive floats sort as unsigned ints) in
// the high word, the record in the low word, stored at the next free slot of the tile's
// sub-bucket.  One block per cell, one thread per record (record_tiles).
// Blocks of k_emit after the cells' blocks: each warp emits the pairs of the large records
// k_project listed (those of cells crowded with them, ws.big), a record at a time with one
// tile of its rectangle per lane, so the records close to the camera are spread over many
// warps instead of lengthening the few warps of the cells that hold them.
constexpr int kBigBlocks = 256;

__device__ __forceinline__ void emit_big(const WsPtrs &ws, const Dims &d, uint32_t gwarp, int lane) {
    const uint32_t nbig = min(ws.hdr->n_big, (uint32_t)kBigListCap);
    const uint32_t slots = rec_slots(d);
    const bool radix = (d.flags & GS_SCHED_RADIX) != 0;
    for (uint32_t k = gwarp; k < nbig; k += (uint32_t)kBigBlocks * (kEmitThreads / 32)) {
        const uint32_t r = ws.big[k];
        if (r >= slots) continue;  // never written past the records (one entry per record)
        const Rec rec = ws.rec[r];
        const ViewInfo vi = ws.views[r / ((uint32_t)d.nblk * (uint32_t)kCell)];
        const uint32_t sub = (uint32_t)((uint64_t)__float_as_uint(rec.c.w) % (uint64_t)d.n) & (d.S - 1);
        int tx0, tx1, ty0, ty1;
        if (!record_rect(vi, rec.a, rec.b, tx0, tx1, ty0, ty1)) continue;
        const int rw = tx1 - tx0 + 1, count = rw * (ty1 - ty0 + 1);
        const float ia = __fdividef(1.f, rec.b.x), ic = __fdividef(1.f, rec.b.z);
        for (int t = lane; t < count; t += 32) {
            const int ty = ty0 + t / rw, tx = tx0 + t % rw;
            if (!tile_hit(vi, rec.a, rec.b, ia, ic, tx, ty)) continue;
            const uint32_t tile = vi.tile_base + (uint32_t)(ty * vi.tiles_x + tx);
            const uint32_t bucket = tile * d.S + sub;
            const uint32_t slot = atomicAdd(ws.cursor + bucket, 1u);
            if (slot < ws.tile_start[bucket + 1] && slot < d.pair_cap)
                put_pair(ws, radix, slot, tile, __float_as_uint(rec.a.z), r);
            else
                atomicOr(ws.err, (uint32_t)kErrPairs);
        }
    }
}

__global__ void __launch_bounds__(kEmitThreads, kEmitMinBlocks) k_emit(WsPtrs ws, Dims d) {
    // No early griddep_launch_dependents here: the tile compositor's blocks would then be
    // placed while the emission still runs, on whichever SMs free first, and the longest
    // tile lists (launched first) would crowd onto a few SMs (k_track_tile measured 110 ->
    // 131 us on the 640 x 480 / 200k frame); launched as the emission's blocks exit, they
    // spread over all SMs.
    griddep_wait();  // the predecessor's results are visible from here on
    const uint32_t cell_blocks = (uint32_t)d.V * (uint32_t)d.nblk * (uint32_t)(kCell / kEmitThreads);
    if (blockIdx.x >= cell_blocks) {
        emit_big(ws, d, (blockIdx.x - cell_blocks) * (kEmitThreads / 32) + (threadIdx.x >> 5), threadIdx.x & 31);
        return;
    }
    // kCell / kEmitThreads blocks per cell, each taking a quarter of the cell's slots: a
    // cell full of visible Gaussians (neighbours in a map built frame by frame) is spread
    // over several SMs instead of running as one long block, and empty quarters leave at once
    const uint32_t cell = blockIdx.x / (uint32_t)(kCell / kEmitThreads);
    const uint32_t first = (blockIdx.x % (uint32_t)(kCell / kEmitThreads)) * (uint32_t)kEmitThreads;
    const uint32_t cnt = ws.cell_cnt[cell];
    const uint32_t slot_id = first + threadIdx.x;  // the record slot of this thread in the cell
    if ((slot_id & ~31u) >= cnt) return;  // whole warps without records leave
    const int lane = threadIdx.x & 31;
    const int view = (int)(cell / (uint32_t)d.nblk);
    const ViewInfo vi = ws.views[view];
    const uint32_t r = cell * kCell + slot_id;
    const bool mine = slot_id < cnt;
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A;
    uint32_t sub = 0;
    if (mine) {
        const Rec rec = ws.rec[r];
        A = rec.a;
        B = rec.b;
        sub = (uint32_t)((uint64_t)__float_as_uint(rec.c.w) % (uint64_t)d.n) & (d.S - 1);
    }
    const bool radix = (d.flags & GS_SCHED_RADIX) != 0;
    // small rectangles: this lane alone, slot atomics issued eight at a time before the
    // dependent stores, so a record waits for about one atomic round trip per eight tiles
    int tx0 = 1, tx1 = 0, ty0 = 1, ty1 = 0;
    const bool has = mine && record_rect(vi, A, B, tx0, tx1, ty0, ty1);
    const int rw = tx1 - tx0 + 1;
    const int count = has ? rw * (ty1 - ty0 + 1) : 0;
    if (has && count <= kSoloTiles) {
        uint32_t hits = 0;  // bit (ty - ty0) rw + (tx - tx0) for every tile met
        const RowSpan span = row_span_setup(A.x, A.y, B.x, B.y, B.z, B.w);
        for (int ty = ty0; ty <= ty1; ++ty) {
            int a0, a1;
            row_span(vi, span, ty, tx0, tx1, a0, a1);
            if (a0 <= a1) hits |= ((1u << (a1 - a0 + 1)) - 1u) << ((ty - ty0) * rw + (a0 - tx0));
        }
        while (hits) {
            uint32_t bucket[8], slot[8];
            bool live[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                live[k] = hits != 0;
                const int t = live[k] ? __ffs(hits) - 1 : 0;
                hits &= hits - 1;
                bucket[k] = (vi.tile_base + (uint32_t)((ty0 + t / rw) * vi.tiles_x + tx0 + t % rw)) * d.S + sub;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (live[k]) slot[k] = atomicAdd(ws.cursor + bucket[k], 1u);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (live[k]) {
                    if (slot[k] < ws.tile_start[bucket[k] + 1] && slot[k] < d.pair_cap)
                        put_pair(ws, radix, slot[k], bucket[k] / d.S, __float_as_uint(A.z), r);
                    else
                        atomicOr(ws.err, (uint32_t)kErrPairs);
                }
        }
    }
    // large rectangles: those k_project listed are emitted by the blocks after the cells'
    // (emit_big); the warp splits the others
    const uint32_t rbase = cell * kCell + (slot_id & ~31u);
    record_tiles<false>(mine && !ws.big_listed[r], vi, A, B, sub, lane,
                        [&](int src, uint32_t tile, float4 As, uint32_t sb) {
        const uint32_t bucket = tile * d.S + sb;
        const uint32_t slot = atomicAdd(ws.cursor + bucket, 1u);
        if (slot < ws.tile_start[bucket + 1] && slot < d.pair_cap)
            put_pair(ws, radix, slot, tile, __float_as_uint(As.z), rbase + (uint32_t)src);
        else
            atomicOr(ws.err, (uint32_t)kErrPairs);
    });
}

cudaError_t launch_emit(const WsPtrs &ws, const Dims &d, cudaStream_t st) {
    const uint32_t cells = (uint32_t)d.V * (uint32_t)d.nblk;
    const cudaError_t e = launch_dep(k_emit, dim3(cells * (uint32_t)(kCell / kEmitThreads) + kBigBlocks),
                                     dim3(kEmitThreads), st, ws, d);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace gsk
