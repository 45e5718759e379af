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

// Tiles met by a record's support ellipse.  The pixel box is derived from the stored
// conic (Sigma'_xx = c / det, Sigma'_yy = a / det of the conic) with explicitly rounded
// operations, so k_project (counting) and k_emit (writing) enumerate the same tiles.
template <class F>
__device__ __forceinline__ void for_each_tile(const ViewInfo &vi, float4 A, float4 B, F &&f) {
    const float detc = __fsub_rn(__fmul_rn(B.x, B.z), __fmul_rn(B.y, B.y));
    if (!(detc > 0.f)) return;
    const float hx = __fsqrt_rn(__fmul_rn(B.w, __fdiv_rn(B.z, detc)));
    const float hy = __fsqrt_rn(__fmul_rn(B.w, __fdiv_rn(B.x, detc)));
    int tx0, tx1, ty0, ty1;
    tile_rect(vi, A.x, A.y, hx, hy, tx0, tx1, ty0, ty1);
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            float x0, x1, y0, y1;
            tile_bounds(vi, tx, ty, x0, x1, y0, y1);
            if (ellipse_meets_rect(A.x, A.y, B.x, B.y, B.z, B.w, x0, x1, y0, y1)) f(tx, ty);
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

// Exclusive scan of the per-tile counts by one block (run by the last k_project block).
__device__ void scan_tiles(const WsPtrs &ws, const Dims &d) {
    __shared__ unsigned long long part[kBlock];
    const uint32_t T = d.T;
    const uint32_t per = (T + kBlock - 1) / kBlock;
    const uint32_t lo = min(T, threadIdx.x * per), hi = min(T, lo + per);
    unsigned long long s = 0;
    for (uint32_t t = lo; t < hi; ++t) s += __ldcg(ws.tile_cnt + t);
    part[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan of the partial sums
    for (int off = 1; off < kBlock; off <<= 1) {
        unsigned long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0ull;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = part[threadIdx.x] - s;
    for (uint32_t t = lo; t < hi; ++t) {
        const uint32_t c = __ldcg(ws.tile_cnt + t);
        const uint32_t o = (uint32_t)min(run, (unsigned long long)0xffffffffu);
        ws.tile_start[t] = o;
        ws.cursor[t] = o;
        ws.tile_cnt[t] = 0;
        run += c;
    }
    if (threadIdx.x == kBlock - 1) {
        const unsigned long long total = part[kBlock - 1];
        ws.tile_start[T] = (uint32_t)min(total, (unsigned long long)0xffffffffu);
        ws.hdr->n_pairs = total;
        if (total > d.pair_cap) atomicOr(ws.err, (uint32_t)kErrPairs);
        ws.hdr->k1_done = 0;
    }
}

template <int DT>
__global__ void __launch_bounds__(kBlock) k_project(ProjectLaunch L) {
    const int v = blockIdx.y, b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    __shared__ float sRt[12];
    __shared__ ViewInfo sv;
    __shared__ uint32_t warp_off[kMaskWords + 1];
    __shared__ uint32_t s_chunk;
    __shared__ int s_last;
    if (tid == 0) {
        load_pose(L.poses + 7 * v, sRt);
        sv = L.ws.views[v];
    }
    __syncthreads();
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
                    const uint32_t base = vi.tile_base;
                    const int tx_n = vi.tiles_x;
                    uint32_t *cnt = L.ws.tile_cnt;
                    int touched = 0;
                    for_each_tile(vi, A, B, [&](int tx, int ty) {
                        atomicAdd(cnt + base + (uint32_t)(ty * tx_n + tx), 1u);
                        ++touched;
                    });
                    vis = touched > 0;
                }
            }
        }
    }
    // compaction: visible pairs of this block get consecutive records in Gaussian order
    const uint32_t ballot = __ballot_sync(0xffffffffu, vis);
    const size_t cell = (size_t)v * L.d.nblk + b;
    if (lane == 0) {
        warp_off[warp] = __popc(ballot);
        L.ws.vis_mask[cell * kMaskWords + warp] = ballot;
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (int w = 0; w < kMaskWords; ++w) {
            const uint32_t c = warp_off[w];
            warp_off[w] = run;
            run += c;
        }
        s_chunk = run ? atomicAdd(&L.ws.hdr->n_rec, run) : 0u;
        L.ws.chunk_start[cell] = s_chunk;
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

// One key per (record, tile met): depth bits (positive floats sort as unsigned ints)
// in the high word, the record in the low word, stored at the tile's next free slot.
__global__ void __launch_bounds__(kBlock) k_emit(WsPtrs ws, Dims d) {
    const uint32_t n = min(ws.hdr->n_rec, d.rec_cap);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const float4 A = ws.rec[r].a, B = ws.rec[r].b;
        const uint32_t gv = __float_as_uint(ws.rec[r].c.w);
        const int v = (int)((uint64_t)gv / (uint64_t)d.n);
        const ViewInfo vi = ws.views[v];
        const unsigned long long key = ((unsigned long long)__float_as_uint(A.z) << 32) | r;
        for_each_tile(vi, A, B, [&](int tx, int ty) {
            const uint32_t tile = vi.tile_base + (uint32_t)(ty * vi.tiles_x + tx);
            const uint32_t slot = atomicAdd(ws.cursor + tile, 1u);
            if (slot < ws.tile_start[tile + 1] && slot < d.pair_cap)
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
    const uint32_t want = (d.rec_cap + kBlock - 1) / kBlock;
    const uint32_t grid = max(1u, min(want, (uint32_t)(sms > 0 ? sms * 8 : 1024)));
    k_emit<<<grid, kBlock, 0, st>>>(ws, d);
    return cudaGetLastError();
}

}  // namespace gsk
