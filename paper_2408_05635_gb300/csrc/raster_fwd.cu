// raster_fwd.cu -- front-to-back compositing of colour, depth and silhouette.
//
// One block per tile (16 x 16 by default), one thread per pixel.  The block first sorts its tile's
// list (tile_sort.cuh).  For pixel p and the tile's
// Gaussians in (depth, index) order:
//   C(p) = sum_i c_i a_i T_i   (Eq. 2)
//   D(p) = sum_i d_i a_i T_i   (Eq. 3, d_i = camera-frame depth of the mean)
//   S(p) = sum_i a_i T_i       (Eq. 4)
// with a_i = min(alpha_max, o_i exp(power_i)) the 2-D footprint of Eq. 1 and
// T_i = prod_{j<i} (1 - a_j).  Gaussians with a_i < alpha_min are skipped; the walk
// stops before the Gaussian that would take T below t_min, and the block stops as soon
// as all its pixels have stopped.  Batches of NB records (64, 128 or 256, the batch
// depth, picked per context) are gathered into shared memory by the first NB threads;
// each warp (an 8 x 4 patch of the tile) then lists the batch Gaussians whose footprint
// can reach alpha_min somewhere on its patch (the support box, then the maximum of the
// footprint over the patch rectangle: build_patch_list) and walks only those.  A smaller batch stages
// fewer Gaussians past the point where every pixel of the tile has stopped; a larger one
// takes fewer barriers.
//
// With targets, the combined loss of Sec. III-B (plus the depth-prior term) is
// evaluated in the epilogue: its per-pixel gradient goes to the workspace for the
// backward and its value is reduced per tile in double-float (summed per view by k_finalize).
#include "fwd_walk.cuh"
#include "gs_internal.cuh"
#include "tile_sort.cuh"

namespace gsk {

__device__ __forceinline__ float sgnf(float x) { return (float)((x > 0.f) - (x < 0.f)); }

template <bool LOSS, int NB, int LW>
__global__ void __launch_bounds__(kTilePix, 5) k_forward(ForwardLaunch L) {
    static_assert(NB % 32 == 0 && NB <= kBatch, "batch depth: a multiple of 32, at most kBatch");
    static_assert(LW >= 3 && (1 << LW) * kPatchH <= kTilePix, "tile width: 8 to 32 pixels");
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    __shared__ float4 sP0[NB], sC[NB], sBox[NB];
    __shared__ float4 sP1[NB];                     // (kuu, lo, -1/(2 kuu), -1/(2 kvv)): the stride of sP0, sC
    __shared__ uint16_t sList[kTilePix / 32][NB];  // byte offsets: 16 x batch position
    __shared__ unsigned long long sKeys[2 * kSortSmemKeys];  // the sort's two buffers
    __shared__ int s_view;
    __shared__ float s_loss[kTilePix / 32];
    const uint32_t tile = L.ws.tile_order[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_view = view_of_tile(L.ws.views, L.d.V, tile);
    __syncthreads();
    const int view = s_view;
    (void)view;
    const ViewInfo vi = L.ws.views[view];
    const uint32_t local = tile - vi.tile_base;
    const int tx = (int)(local % (uint32_t)vi.tiles_x), ty = (int)(local / (uint32_t)vi.tiles_x);
    constexpr int kPPR = (1 << LW) / kPatchW;  // 8 x 4 patches per patch row (tile width 2^LW)
    const int pu0 = (warp % kPPR) * kPatchW, pv0 = (warp / kPPR) * kPatchH;
    const int lu = pu0 + (lane & (kPatchW - 1)), lv = pv0 + lane / kPatchW;
    const int px = (tx << LW) + lu, py = (ty << vi.tile_lh) + lv;
    const bool inside = px < vi.width && py < vi.height;
    const float x0 = (float)(tx << LW), y0 = (float)(ty << vi.tile_lh);
    const float2 uv = make_float2((float)lu, (float)lv);  // tile-local pixel centre
    const float pu_lo = (float)pu0, pu_hi = (float)(pu0 + kPatchW - 1);
    const float pv_lo = (float)pv0, pv_hi = (float)(pv0 + kPatchH - 1);
    const Settings &S = L.s;
    const float thr = S.log2_alpha_min;

    uint32_t start;
    const uint32_t n = tile_entries(L.ws, L.d, tile, start);
    // this tile's list in (depth, Gaussian) order, unless the device-wide radix sort
    // (GS_SCHED_RADIX) has already ordered it
    if (!(L.d.flags & GS_SCHED_RADIX)) sort_tile(L.ws, start, (int)n, sKeys);
    FwdPixel walk{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !inside};
    uint32_t n_eval = 0, n_contrib = 0;
    // with the loss: this pixel's targets, loaded once the first batch is staged so their
    // latency passes during the forward walk
    const uint32_t HW = (uint32_t)vi.width * (uint32_t)vi.height;
    const uint32_t p = inside ? (uint32_t)py * (uint32_t)vi.width + (uint32_t)px : 0u;
    const uint32_t gp = vi.pix_base + p;  // pixel in the concatenated planes
    float tr = 0.f, tg = 0.f, tb = 0.f, Dt = 0.f, pr = 0.f;
    bool targets_loaded = !LOSS;
    const auto load_targets = [&]() {
        targets_loaded = true;
        if (inside) {
            const float *trgb = L.t_rgb + 3u * vi.pix_base;
            tr = trgb[p];
            tg = trgb[HW + p];
            tb = trgb[2u * HW + p];
            Dt = L.t_depth[gp];
            if (L.t_prior) pr = L.t_prior[gp];
        }
    };
    for (uint32_t b0 = 0; b0 < n; b0 += NB) {
        if (__syncthreads_count(!walk.done) == 0) break;
        const uint32_t idx = b0 + tid;
        if (tid < NB && idx < n) {  // thread tid stages batch position tid
            const uint32_t r = L.ws.sorted[start + idx];
            if (r < rec_slots(L.d)) {
                const Rec rr = L.ws.rec[r];
                const Footprint f = stage_footprint(rr.a, rr.b, x0, y0);
                sP0[tid] = f.p0;
                sP1[tid] = f.p1;
                sC[tid] = make_float4(rr.c.x, rr.c.y, rr.c.z, rr.a.z);
                sBox[tid] = stage_box(rr.b, -f.p0.x, -f.p0.y);
            } else {
                sBox[tid] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);  // empty: never listed
            }
        }
        __syncthreads();
        if (!targets_loaded) load_targets();
        const int cnt = (int)min((uint32_t)NB, n - b0);
        if (__any_sync(0xffffffffu, !walk.done)) {
            // this warp's list: the batch Gaussians whose footprint reaches its 8 x 4 patch
            const int nl = build_patch_list(sBox, sP0, sP1, sList[warp], cnt, lane, thr, pu_lo, pu_hi, pv_lo, pv_hi);
            if (!walk.done)
                fwd_walk_batch(walk, sList[warp], nl, b0, sP0, sP1, sC, uv, thr, S.alpha_max, S.t_min, n_eval,
                               n_contrib);
        }
    }
    // Eq. 4 summed equals 1 - prod(1 - a_i) = 1 - T exactly; the identity is used instead
    // of a fifth accumulator
    const float T = walk.T, cr = walk.cr, cg = walk.cg, cb = walk.cb, D = walk.D;
    const uint32_t last = walk.last;
    const float Sil = 1.f - T;
    count_pairs(n_eval, n_contrib, &L.ws.hdr->fwd_evals, &L.ws.hdr->fwd_contrib);

    if (inside) {
        if (L.rgb) {
            float *o = L.rgb + 3u * vi.pix_base;
            o[p] = cr;
            o[HW + p] = cg;
            o[2u * HW + p] = cb;
        }
        if (L.depth) L.depth[gp] = D;
        if (L.sil) L.sil[gp] = Sil;
        L.ws.t_final[gp] = T;
        L.ws.n_last[gp] = last;
    }
    if constexpr (LOSS) {
        if (!targets_loaded) load_targets();  // an empty tile list: no batch was staged
        float l = 0.f;
        if (inside) {
            const bool valid = Dt > 0.f;
            const bool M = valid && Sil > S.sil_thresh;
            float g0 = 0.f, g1 = 0.f, g2 = 0.f, gD = 0.f, gS = 0.f;
            if (M) {
                const float r0 = cr - tr, r1 = cg - tg, r2 = cb - tb;
                l += S.w_rgb * (fabsf(r0) + fabsf(r1) + fabsf(r2));
                g0 = S.w_rgb * sgnf(r0);
                g1 = S.w_rgb * sgnf(r1);
                g2 = S.w_rgb * sgnf(r2);
                const float rd = D - Dt;
                l += S.w_depth * fabsf(rd);
                gD = S.w_depth * sgnf(rd);
                if (L.t_prior) {
                    if (pr > 0.f) {
                        const float rp = D - pr;
                        l += S.w_prior * fabsf(rp);
                        gD += S.w_prior * sgnf(rp);
                    }
                }
            }
            if (valid) {
                l += S.w_vis * (1.f - Sil);
                gS = -S.w_vis;
            }
            // same planar layout as the images: colour 3 x H x W per view, then D, then S
            const uint32_t P = L.d.P;
            float *ug = L.ws.upstream + 3u * vi.pix_base;
            ug[p] = g0;
            ug[HW + p] = g1;
            ug[2u * HW + p] = g2;
            L.ws.upstream[3u * P + gp] = gD;
            L.ws.upstream[4u * P + gp] = gS;
        }
        // per-pixel terms summed over the warp in FP32 (32 terms), over the warps in
        // double-float; k_finalize sums the view's tiles in order
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
        if ((tid & 31) == 0) s_loss[tid >> 5] = l;
        __syncthreads();
        if (tid == 0) {
            DF s{0.f, 0.f};
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = df_add(s, DF{s_loss[w], 0.f});
            L.ws.tile_loss[tile] = df_pack(s);
        }
    }
}

template <int NB, int LW>
cudaError_t launch_forward_nb(const ForwardLaunch &L, cudaStream_t st) {
    if (L.t_rgb)
        return launch_dep(k_forward<true, NB, LW>, dim3(L.d.T), dim3(tile_threads(L.d)), st, L);
    else
        return launch_dep(k_forward<false, NB, LW>, dim3(L.d.T), dim3(tile_threads(L.d)), st, L);
}

template <int NB>
cudaError_t launch_forward_lw(const ForwardLaunch &L, cudaStream_t st) {
    switch (tile_lw(L.d)) {
        case 3: return launch_forward_nb<NB, 3>(L, st);
        case 4: return launch_forward_nb<NB, 4>(L, st);
        case 5: return launch_forward_nb<NB, 5>(L, st);
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_forward(const ForwardLaunch &L, cudaStream_t st) {
    if (L.d.T == 0) return cudaSuccess;
    // a batch stages at most one Gaussian per thread of the tile block
    const uint32_t nb = L.d.fwd_batch ? L.d.fwd_batch : (uint32_t)kBatch;
    if (nb > tile_threads(L.d)) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (L.d.fwd_batch) {
        case 0:
        case 256: e = launch_forward_lw<256>(L, st); break;
        case 128: e = launch_forward_lw<128>(L, st); break;
        case 64: e = launch_forward_lw<64>(L, st); break;
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace gsk
