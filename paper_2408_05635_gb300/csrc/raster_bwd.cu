// raster_bwd.cu -- reverse compositing: per-record screen-space gradients.
//
// Differentiating Eqs. 2-4 for one pixel with upstream g = dL/d(C_r, C_g, C_b, D, S):
// walking the contributors back to front with B_ch the colour of everything behind
// Gaussian i (B <- B + a_i (v_i - B), starting from the zero background) and T_i the
// transmittance in front of it (recovered from the stored final transmittance as
// T_i = T_{i+1} / (1 - a_i)); a_i is re-evaluated with the forward's footprint code,
// bit for bit, so both walks skip exactly the same Gaussians,
//   dL/da_i = T_i sum_ch g_ch (v_ch,i - B_ch),   v = (r, g, b, depth, 1),
//   dL/dc_i = a_i T_i g_C,  dL/dd_i = a_i T_i g_D,
// and through a_i = o G, G = exp(power): dL/do = dL/da G, dL/dpower = dL/da a
// (both zero where a_i is clamped at alpha_max), dpower/dmu' = conic (p - mu'),
// dpower/d(conic a, b, c) = (-dx^2 / 2, -dx dy, -dy^2 / 2).
// Only the scalar g . B enters dL/da, so the walk carries that scalar instead of B:
// g.B <- g.B + a_i (g.v_i - g.B).  The conic is constant per Gaussian, so the pixel sums
// are taken of the moments dp (dx, dy, dx^2, dx dy, dy^2), dp = dL/dpower, and the conic is
// applied once per (tile, Gaussian) when the sums are flushed.
//
// Batches of NB records (64, 128 or 256, the batch depth, picked per context) are staged
// by the first NB threads, from the tile's last contributor backwards.  Each warp owns an
// 8 x 4 patch of the tile and walks, back to front, only the staged Gaussians whose
// footprint can reach alpha_min on the patch (build_patch_list) and that precede its last
// contributor.
// Reduction: every (pixel, Gaussian) term is summed over the warp with a butterfly
// reduce-scatter (for the pose-only walk 6 values in 8 shuffles, or two Gaussians' 12 in
// 13 when it steps two at a time; 16 values in 16 otherwise),
// added by the owning lanes into a per-batch shared-memory accumulator, and flushed once
// per (tile, Gaussian) with vector float4 atomics into the record's global accumulator.
// Lanes whose pixel the Gaussian does not reach take a = 0, which leaves T and g.B
// unchanged and zeroes every term, so the walk has no divergent branch.
#include "gs_internal.cuh"
#include "bwd_walk.cuh"

namespace gsk {

// Shared accumulator slots per staged Gaussian: 0, 1 sum dp dx, dp dy; 2 sum a T g_D;
// 3 sum dL/da a_raw; 4..6 sum dp dx^2, dp dx dy, dp dy^2; 8..10 sum a T g_C; 7, 11 unused.
// POSE: only slots 0, 1, 2, 4, 5, 6 (what the pose gradient needs).
template <bool POSE, int NB, int LW>
__global__ void __launch_bounds__(kTilePix, 5) k_backward(BackwardLaunch L) {
    static_assert(NB % 32 == 0 && NB <= kBatch, "batch depth: a multiple of 32, at most kBatch");
    static_assert(LW >= 3 && (1 << LW) * kPatchH <= kTilePix, "tile width: 8 to 32 pixels");
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    __shared__ float4 sP0[NB], sC[NB], sQ[NB], sBox[NB];
    __shared__ float4 sP1[NB];  // (kuu, lo, -1/(2 kuu), -1/(2 kvv)): the stride of sP0, sC
    __shared__ float sAcc[NB * kAccStride];
    __shared__ uint16_t sList[kTilePix / 32][NB];  // byte offsets: 16 x batch position
    __shared__ int s_view;
    __shared__ uint32_t s_nmax;
    const uint32_t tile = L.ws.tile_order[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_view = view_of_tile(L.ws.views, L.d.V, tile);
        s_nmax = 0;
    }
    __syncthreads();
    const ViewInfo vi = L.ws.views[s_view];
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
    // the accumulator slot this lane adds after a reduction, or -1
    int my_slot = -1, pair_slot = -1;
    if (POSE) {
        // the paired steps' joint reduction: value 3 b3 + (b1 ? 2 : b2) of Gaussian b4
        if ((lane & 1) == 0 && !((lane & 2) && (lane & 4))) {
            const int k = ((lane & 8) ? 3 : 0) + ((lane & 2) ? 2 : ((lane & 4) ? 1 : 0));
            pair_slot = k < 3 ? k : k + 1;  // values 0..5 -> slots 0, 1, 2, 4, 5, 6
        }
        if ((lane & 3) == 0 && !((lane & 8) && (lane & 4))) {
            const int k = ((lane & 16) ? 3 : 0) + ((lane & 4) ? 2 : ((lane & 8) ? 1 : 0));
            my_slot = k < 3 ? k : k + 1;  // values 0..5 -> slots 0, 1, 2, 4, 5, 6
        }
    } else {
        int idx = 0;
        if (lane & 16) idx += 8;
        if (lane & 8) idx += 4;
        if (lane & 4) idx += 2;
        if (lane & 2) idx += 1;
        if ((lane & 1) == 0 && idx != 7 && idx != 11 && idx < kAccStride) my_slot = idx;
    }

    uint32_t start;
    const uint32_t n = tile_entries(L.ws, L.d, tile, start);
    const uint32_t HW = (uint32_t)vi.width * (uint32_t)vi.height;
    const uint32_t p = (uint32_t)py * (uint32_t)vi.width + (uint32_t)px;
    const uint32_t gp = vi.pix_base + p;
    float T = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, gD = 0.f, gS = 0.f;
    uint32_t last = 0;
    if (inside) {
        const float *ur = L.up_rgb + 3u * vi.pix_base;
        g0 = ur[p];
        g1 = ur[HW + p];
        g2 = ur[2u * HW + p];
        gD = L.up_depth[gp];
        gS = L.up_sil[gp];
        if (g0 != 0.f || g1 != 0.f || g2 != 0.f || gD != 0.f || gS != 0.f) {
            last = min(L.ws.n_last[gp], n);
            T = L.ws.t_final[gp];
        }
    }
    uint32_t wlast = last;  // largest contributor count in the warp
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, off));
    if (lane == 0 && wlast) atomicMax(&s_nmax, wlast);
    __syncthreads();
    const uint32_t nmax = s_nmax;
    float GB = 0.f;  // g . (colour, depth, 1) of everything behind, back-to-front
    uint32_t n_eval = 0, n_contrib = 0;

    for (int64_t b0 = nmax ? (int64_t)((nmax - 1) / NB) * NB : -1; b0 >= 0; b0 -= NB) {
        const int cnt = (int)min((uint32_t)NB, nmax - (uint32_t)b0);
        if (tid < cnt) {
            const uint32_t r = L.ws.sorted[start + (uint32_t)b0 + tid];
            if (r < rec_slots(L.d)) {
                const Rec rr = L.ws.rec[r];
                const Footprint f = stage_footprint(rr.a, rr.b, x0, y0);
                sP0[tid] = f.p0;
                sP1[tid] = f.p1;
                sC[tid] = make_float4(rr.c.x, rr.c.y, rr.c.z, rr.a.z);
                sQ[tid] = make_float4(rr.b.x, rr.b.y, rr.b.z, rr.a.w);
                sBox[tid] = stage_box(rr.b, -f.p0.x, -f.p0.y);
            } else {
                sBox[tid] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
            }
        }
        if (tid < NB) {  // thread tid owns the accumulator row of batch position tid
#pragma unroll
            for (int k = 0; k < kAccStride; ++k) sAcc[tid * kAccStride + k] = 0.f;
        }
        __syncthreads();
        // this warp's list, limited to entries below its largest contributor count
        const int wcnt = (int)min((int64_t)cnt, (int64_t)wlast - b0);
        const int nl = build_patch_list(sBox, sP0, sP1, sList[warp], wcnt, lane, thr, pu_lo, pu_hi, pv_lo, pv_hi);
        int e = nl - 1;
        // entries at byte offsets below lim are in front of this pixel's last contributor
        const int lim = (int)max(min((int64_t)last - b0, (int64_t)NB), (int64_t)0) * 16;
        if constexpr (POSE) {
            // two Gaussians per step: the pixel state is updated in depth order (the back
            // one first), and the two reductions are independent, so they overlap
            for (; e >= 1; e -= 2) {
                const int jA = sList[warp][e], jB = sList[warp][e - 1];
                const PolyEval pA = eval_poly(uv, at_off(sP0, jA), p1_at(sP1, jA));
                const PolyEval pB = eval_poly(uv, at_off(sP0, jB), p1_at(sP1, jB));
                const bool lA = jA < lim, lB = jB < lim;
                n_eval += lA + lB;
                const bool cA = lA && pA.poly >= thr, cB = lB && pB.poly >= thr;
                if (!__any_sync(0xffffffffu, cA || cB)) continue;
                n_contrib += cA + cB;
                const float s2 = bwd_pair_reduce(cA, pA, at_off(sC, jA), cB, pB, at_off(sC, jB), g0, g1, g2, gD,
                                                 gS, S.alpha_max, T, GB, lane);
                if (pair_slot >= 0 && s2 != 0.f)
                    atomicAdd(&sAcc[(((lane & 16) ? jB : jA) >> 4) * kAccStride + pair_slot], s2);
            }
        }
        for (; e >= 0; --e) {
            const int j = sList[warp][e];
            const bool live = j < lim;
            const PolyEval pe = eval_poly(uv, at_off(sP0, j), p1_at(sP1, j));
            n_eval += live;
            const bool c = live && pe.poly >= thr;
            if (!__any_sync(0xffffffffu, c)) continue;
            n_contrib += c;
            if constexpr (POSE) {
                float v[6];
                moments6(bwd_step(c, pe, at_off(sC, j), g0, g1, g2, gD, gS, S.alpha_max, T, GB), v);
                const float sum = warp_reduce_scatter6(v[0], v[1], v[2], v[3], v[4], v[5], lane);
                if (my_slot >= 0 && sum != 0.f) atomicAdd(&sAcc[(j >> 4) * kAccStride + my_slot], sum);
            } else {
                const float araw = ex2_approx(pe.poly);
                const float a = c ? fminf(S.alpha_max, araw) : 0.f;
                if (c) T = T * __fdividef(1.f, 1.f - a);  // transmittance in front of this Gaussian
                const float4 Cc = at_off(sC, j);
                const float gv = fmaf(g0, Cc.x, fmaf(g1, Cc.y, fmaf(g2, Cc.z, fmaf(gD, Cc.w, gS))));
                const float diff = gv - GB;
                const float dalpha = T * diff;
                GB = fmaf(a, diff, GB);
                const float w = a * T;
                const float dp = araw < S.alpha_max ? dalpha * a : 0.f;
                const float dpx = dp * pe.d.x, dpy = dp * pe.d.y;
                float vals[16] = {dpx,     dpy,     w * gD, c && araw < S.alpha_max ? dalpha * araw : 0.f,
                                  dpx * pe.d.x, dpx * pe.d.y, dpy * pe.d.y, 0.f,
                                  w * g0,  w * g1,  w * g2, 0.f, 0.f, 0.f, 0.f, 0.f};
                int slot;
                const float sum = warp_reduce_scatter<16>(vals, lane, slot);
                if (my_slot >= 0 && sum != 0.f) atomicAdd(&sAcc[(j >> 4) * kAccStride + my_slot], sum);
            }
        }
        __syncthreads();
        if (tid < cnt) {
            const uint32_t r = L.ws.sorted[start + (uint32_t)b0 + tid];
            if (r < rec_slots(L.d)) {
                const float *m = sAcc + tid * kAccStride;
                const float4 Q = sQ[tid];
                const float4 v0 = make_float4(Q.x * m[0] + Q.y * m[1], Q.y * m[0] + Q.z * m[1], m[2],
                                              POSE ? 0.f : m[3] / Q.w);
                const float4 v1 = make_float4(-0.5f * m[4], -m[5], -0.5f * m[6], 0.f);
                if (v0.x != 0.f || v0.y != 0.f || v0.z != 0.f || v0.w != 0.f) atomicAdd(&L.ws.rec_grad[r].g0, v0);
                if (v1.x != 0.f || v1.y != 0.f || v1.z != 0.f) atomicAdd(&L.ws.rec_grad[r].g1, v1);
                if constexpr (!POSE) {
                    const float4 v2 = make_float4(m[8], m[9], m[10], 0.f);
                    if (v2.x != 0.f || v2.y != 0.f || v2.z != 0.f) atomicAdd(&L.ws.rec_grad[r].g2, v2);
                }
            }
        }
        __syncthreads();
    }
    count_pairs(n_eval, n_contrib, &L.ws.hdr->bwd_evals, &L.ws.hdr->bwd_contrib);
}

template <int NB, int LW>
cudaError_t launch_backward_nb(const BackwardLaunch &L, cudaStream_t st) {
    if (L.pose_only)
        return launch_dep(k_backward<true, NB, LW>, dim3(L.d.T), dim3(tile_threads(L.d)), st, L);
    else
        return launch_dep(k_backward<false, NB, LW>, dim3(L.d.T), dim3(tile_threads(L.d)), st, L);
}

template <int NB>
cudaError_t launch_backward_lw(const BackwardLaunch &L, cudaStream_t st) {
    switch (tile_lw(L.d)) {
        case 3: return launch_backward_nb<NB, 3>(L, st);
        case 4: return launch_backward_nb<NB, 4>(L, st);
        case 5: return launch_backward_nb<NB, 5>(L, st);
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_backward(const BackwardLaunch &L, cudaStream_t st) {
    if (L.d.T == 0) return cudaSuccess;
    // a batch stages at most one Gaussian per thread of the tile block
    const uint32_t nb = L.d.bwd_batch ? L.d.bwd_batch : (uint32_t)kBatch;
    if (nb > tile_threads(L.d)) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (L.d.bwd_batch) {
        case 0:
        case 256: e = launch_backward_lw<256>(L, st); break;
        case 128: e = launch_backward_lw<128>(L, st); break;
        case 64: e = launch_backward_lw<64>(L, st); break;
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace gsk
