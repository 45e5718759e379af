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
// stored conic (Sigma'_xx = c / det, Sigma'_yy = a / det of the conic) with explicitly
// rounded operations, so k_project (counting) and k_emit (writing) enumerate the same
// tiles.  Returns false when the box misses the image.
__device__ __forceinline__ bool record_rect(const ViewInfo &vi, float4 A, float4 B, int &tx0, int &tx1, int &ty0,
                                            int &ty1) {
    const float detc = __fsub_rn(__fmul_rn(B.x, B.z), __fmul_rn(B.y, B.y));
    if (!(detc > 0.f)) return false;
    const float hx = __fsqrt_rn(__fmul_rn(B.w, __fdiv_rn(B.z, detc)));
    const float hy = __fsqrt_rn(__fmul_rn(B.w, __fdiv_rn(B.x, detc)));
    tile_rect(vi, A.x, A.y, hx, hy, tx0, tx1, ty0, ty1);
    return tx0 <= tx1 && ty0 <= ty1;
}

__device__ __forceinline__ bool tile_hit(const ViewInfo &vi, float4 A, float4 B, float ia, float ic, int tx, int ty) {
    float x0, x1, y0, y1;
    tile_bounds(vi, tx, ty, x0, x1, y0, y1);
    return ellipse_meets_rect(A.x, A.y, B.x, B.y, B.z, ia, ic, B.w, x0, x1, y0, y1);
}

// The whole warp walks the tiles of one record at a time: the record's lane broadcasts
// it and the 32 lanes split its tile rectangle, so one large Gaussian does not keep the
// other 31 lanes waiting.  body(src lane, tile, record's A, record's tag) runs for every
// tile the support meets.
template <class Body>
__device__ __forceinline__ void warp_tiles(uint32_t bits, const ViewInfo &vi_own, float4 A_own, float4 B_own,
                                           int lane, const ViewInfo *views_or_null, int view_own, uint32_t tag_own,
                                           Body &&body) {
    while (bits) {
        const int src = __ffs(bits) - 1;
        bits &= bits - 1;
        float4 A, B;
        A.x = __shfl_sync(0xffffffffu, A_own.x, src);
        A.y = __shfl_sync(0xffffffffu, A_own.y, src);
        A.z = __shfl_sync(0xffffffffu, A_own.z, src);
        A.w = __shfl_sync(0xffffffffu, A_own.w, src);
        B.x = __shfl_sync(0xffffffffu, B_own.x, src);
        B.y = __shfl_sync(0xffffffffu, B_own.y, src);
        B.z = __shfl_sync(0xffffffffu, B_own.z, src);
        B.w = __shfl_sync(0xffffffffu, B_own.w, src);
        const int view = __shfl_sync(0xffffffffu, view_own, src);
        const uint32_t tag = __shfl_sync(0xffffffffu, tag_own, src);
        const ViewInfo vi = views_or_null ? views_or_null[view] : vi_own;
        int tx0, tx1, ty0, ty1;
        if (!record_rect(vi, A, B, tx0, tx1, ty0, ty1)) continue;
        const float ia = __frcp_rn(B.x), ic = __frcp_rn(B.z);
        const int rw = tx1 - tx0 + 1, count = rw * (ty1 - ty0 + 1);
        for (int t = lane; t < count; t += 32) {
            const int ty = ty0 + t / rw, tx = tx0 + t % rw;
            if (tile_hit(vi, A, B, ia, ic, tx, ty)) body(src, vi.tile_base + (uint32_t)(ty * vi.tiles_x + tx), A, tag);
        }
    }
}

struct ViewChunk {
    ViewInfo v[32];
};

__global__ void k_copy_views(ViewInfo *dst, int count, ViewChunk chunk) {
    const int i = threadIdx.x;
    if (i < count) dst[i] = chunk.v[i];
}

cudaError_t launch_upload_views(const ViewInfo *host_views, int V, ViewInfo *dev, cudaStream_t st) {
    for (int base = 0; base < V; base += 32) {
        ViewChunk c;
        const int cnt = V - base < 32 ? V - base : 32;
        for (int k = 0; k < cnt; ++k) c.v[k] = host_views[base + k];
        k_copy_views<<<1, 32, 0, st>>>(dev + base, cnt, c);
    }
    return cudaGetLastError();
}

// Exclusive scan of the per-(tile, sub-bucket) counts by one block (the last k_project
// block): chunks of 4 x kBlock counters, vector loads, warp scans and a running carry.
__device__ void scan_tiles(const WsPtrs &ws, const Dims &d) {
    __shared__ uint32_t warp_sum[kWarps];
    __shared__ unsigned long long s_carry;
    const uint32_t TS = d.T * d.S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    uint32_t max_tile = 0;
    __syncthreads();
    for (uint32_t base = 0; base < TS; base += 4 * kBlock) {
        const uint32_t i0 = base + 4 * threadIdx.x;
        uint32_t c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = i0 + k < TS ? __ldcg(ws.tile_cnt + i0 + k) : 0u;
        const uint32_t mine = c[0] + c[1] + c[2] + c[3];
        uint32_t incl = mine;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < kWarps; ++w) {
            if (w < warp) before += warp_sum[w];
            total += warp_sum[w];
        }
        unsigned long long run = s_carry + before + (incl - mine);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k < TS) {
                const uint32_t o = (uint32_t)min(run, (unsigned long long)0xffffffffu);
                ws.tile_start[i0 + k] = o;
                ws.cursor[i0 + k] = o;
                ws.tile_cnt[i0 + k] = 0;
                run += c[k];
            }
        // longest tile list: a tile's S sub-buckets are consecutive (S divides 4)
        if (d.S <= 4) {
            for (int k = 0; k < 4; k += d.S) {
                uint32_t t = 0;
                for (uint32_t q = 0; q < d.S; ++q) t += c[k + q];
                max_tile = max(max_tile, t);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
    if (d.S > 4) {  // tiles span several threads' chunks: measure from the finished offsets
        const uint32_t total = (uint32_t)min(s_carry, (unsigned long long)0xffffffffu);
        for (uint32_t t = threadIdx.x; t < d.T; t += kBlock) {
            const uint32_t end = t + 1 < d.T ? ws.tile_start[(t + 1) * d.S] : total;
            max_tile = max(max_tile, end - ws.tile_start[t * d.S]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long total = s_carry;
        ws.tile_start[TS] = (uint32_t)min(total, (unsigned long long)0xffffffffu);
        ws.hdr->n_pairs = total;
        if (total > d.pair_cap) atomicOr(ws.err, (uint32_t)kErrPairs);
        ws.hdr->k1_done = 0;
    }
    atomicMax(&ws.hdr->max_tile, max_tile);
}

template <int DT>
__global__ void __launch_bounds__(kBlock) k_project(ProjectLaunch L) {
    const int v = blockIdx.y, b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    __shared__ float sRt[12];
    __shared__ ViewInfo sv;
    __shared__ uint32_t warp_off[kWarps];
    __shared__ uint32_t s_chunk;
    __shared__ int s_last;
    if (tid == 0) {
        load_pose(L.poses + 7 * v, sRt);
        sv = L.ws.views[v];
    }
    __syncthreads();
    if (b == 0 && tid < 12) L.ws.view_rt[12 * v + tid] = sRt[tid];
    const ViewInfo vi = sv;
    const int64_t i = (int64_t)b * kBlock + tid;
    const Settings &S = L.s;
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A, C = A;
    bool vis = false;
    if (i < L.d.n) {
        const float mx = __ldg(L.g.means + 3 * i), my = __ldg(L.g.means + 3 * i + 1), mz = __ldg(L.g.means + 3 * i + 2);
        const float x = cam_coord(sRt, 0, mx, my, mz);
        const float y = cam_coord(sRt, 1, mx, my, mz);
        const float z = cam_coord(sRt, 2, mx, my, mz);
        if (z > S.z_near) {
            float qw = ld_attr<DT>(L.g.quats, 4 * i), qx = ld_attr<DT>(L.g.quats, 4 * i + 1);
            float qy = ld_attr<DT>(L.g.quats, 4 * i + 2), qz = ld_attr<DT>(L.g.quats, 4 * i + 3);
            const float qq = qw * qw + qx * qx + qy * qy + qz * qz;
            const float qi = qq > 0.f ? rsqrtf(qq) : 0.f;
            qw *= qi; qx *= qi; qy *= qi; qz *= qi;
            float Rg[9];
            quat_to_rot(qw, qx, qy, qz, Rg);
            const float s0 = expf(ld_attr<DT>(L.g.log_scales, 3 * i));
            const float s1 = expf(ld_attr<DT>(L.g.log_scales, 3 * i + 1));
            const float s2 = expf(ld_attr<DT>(L.g.log_scales, 3 * i + 2));
            // M = W Rg diag(s): Sigma_c = M M^T
            float M[9];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                M[3 * r + 0] = (sRt[3 * r] * Rg[0] + sRt[3 * r + 1] * Rg[3] + sRt[3 * r + 2] * Rg[6]) * s0;
                M[3 * r + 1] = (sRt[3 * r] * Rg[1] + sRt[3 * r + 1] * Rg[4] + sRt[3 * r + 2] * Rg[7]) * s1;
                M[3 * r + 2] = (sRt[3 * r] * Rg[2] + sRt[3 * r + 1] * Rg[5] + sRt[3 * r + 2] * Rg[8]) * s2;
            }
            const float iz = 1.f / z;
            const float J00 = vi.fx * iz, J02 = -vi.fx * x * iz * iz;
            const float J11 = vi.fy * iz, J12 = -vi.fy * y * iz * iz;
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
            const float det = S00 * S11 - S01 * S01;
            if (det > 0.f) {
                const float idet = 1.f / det;
                const float o = 1.f / (1.f + expf(-ld_attr<DT>(L.g.logits, i)));
                float dmax2;
                if (S.alpha_min > 0.f)
                    dmax2 = o >= S.alpha_min ? 2.f * logf(o / S.alpha_min) : -1.f;
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
                }
            }
        }
    }
    // compaction: visible pairs of this block get consecutive records in Gaussian order
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
        s_chunk = run ? atomicAdd(&L.ws.hdr->n_rec, run) : 0u;
    }
    __syncthreads();
    if (vis) {
        const uint32_t rec = s_chunk + warp_off[warp] + __popc(ballot & ((1u << lane) - 1u));
        if (rec < L.d.rec_cap) {
            Rec r;
            r.a = A; r.b = B; r.c = C;
            L.ws.rec[rec] = r;
            RecGrad z;
            z.g0 = z.g1 = z.g2 = make_float4(0.f, 0.f, 0.f, 0.f);
            L.ws.rec_grad[rec] = z;
        } else {
            atomicOr(L.ws.err, (uint32_t)kErrRecords);
        }
    }
    // per-(tile, sub-bucket) pair counts, the warp sharing each visible Gaussian's tiles
    uint32_t *cnt = L.ws.tile_cnt;
    const uint32_t nsub = L.d.S;
    warp_tiles(ballot, vi, A, B, lane, nullptr, v, (uint32_t)i & (nsub - 1), [&](int, uint32_t tile, float4, uint32_t sub) {
        red_add(cnt + tile * nsub + sub, 1u);
    });
    // the last block to finish turns the per-tile counts into offsets
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&L.ws.hdr->k1_done, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        scan_tiles(L.ws, L.d);
    }
}

cudaError_t launch_project(const ProjectLaunch &L, cudaStream_t st) {
    dim3 grid(L.d.nblk, L.d.V);
    switch (L.dtype) {
        case GS_F32: k_project<GS_F32><<<grid, kBlock, 0, st>>>(L); break;
        case GS_BF16: k_project<GS_BF16><<<grid, kBlock, 0, st>>>(L); break;
        case GS_F16: k_project<GS_F16><<<grid, kBlock, 0, st>>>(L); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// One key per (record, tile met): depth bits (positive floats sort as unsigned ints) in
// the high word, the record in the low word, stored at the next free slot of the tile's
// sub-bucket.  Each warp takes 32 consecutive records and walks their tiles together
// (warp_tiles): a Gaussian close to the camera that spans thousands of tiles is split
// over 32 lanes instead of holding one thread while the rest of the grid finishes.
__global__ void __launch_bounds__(kBlock) k_emit(WsPtrs ws, Dims d) {
    const uint32_t n = min(ws.hdr->n_rec, d.rec_cap);
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) / 32 * 32; base < n; base += warps * 32) {
        const uint32_t r = base + lane;
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A;
        int view = 0;
        uint32_t sub = 0;
        if (r < n) {
            const Rec rec = ws.rec[r];
            A = rec.a;
            B = rec.b;
            const uint64_t gv = __float_as_uint(rec.c.w);
            view = (int)(gv / (uint64_t)d.n);
            sub = (uint32_t)(gv % (uint64_t)d.n) & (d.S - 1);
        }
        const uint32_t bits = __ballot_sync(0xffffffffu, r < n);
        const ViewInfo none{};
        warp_tiles(bits, none, A, B, lane, ws.views, view, sub, [&](int src, uint32_t tile, float4 As, uint32_t sb) {
            const unsigned long long key = ((unsigned long long)__float_as_uint(As.z) << 32) | (base + (uint32_t)src);
            const uint32_t bucket = tile * d.S + sb;
            const uint32_t slot = atomicAdd(ws.cursor + bucket, 1u);
            if (slot < ws.tile_start[bucket + 1] && slot < d.pair_cap)
                ws.keys[slot] = key;
            else
                atomicOr(ws.err, (uint32_t)kErrPairs);
        });
    }
}

cudaError_t launch_emit(const WsPtrs &ws, const Dims &d, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = ((uint64_t)d.rec_cap + kBlock - 1) / kBlock;
    const uint32_t grid = (uint32_t)max((uint64_t)1, min(want, (uint64_t)(sms > 0 ? sms * 8 : 1024)));
    k_emit<<<grid, kBlock, 0, st>>>(ws, d);
    return cudaGetLastError();
}

}  // namespace gsk
