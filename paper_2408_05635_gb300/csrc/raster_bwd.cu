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
//
// Each warp owns an 8 x 4 patch of the tile and walks, back to front, only the staged
// Gaussians whose support box meets the patch and that precede its last contributor.
// Reduction: every (pixel, Gaussian) term is summed over the warp with a butterfly
// reduce-scatter (NV values in NV - 1 + log2(32 / NV) shuffles instead of 5 NV), added
// by the owning lanes into a per-batch shared-memory accumulator, and flushed once per
// (tile, Gaussian) with vector float4 atomics into the record's global accumulator.
#include "gs_internal.cuh"

namespace gsk {

constexpr int kAccStride = 12;  // floats per staged Gaussian in the shared accumulator

// Butterfly reduce-scatter of NV per-lane values over the warp.  After it, the lane
// holds the full warp sum of value `idx`; lanes with (lane & (32 / NV - 1)) == 0 are the
// distinct owners.
template <int NV>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NV], int lane, int &idx) {
    constexpr int LOG = NV == 16 ? 4 : (NV == 8 ? 3 : 2);
    idx = 0;
#pragma unroll
    for (int s = 0; s < LOG; ++s) {
        const int mask = 16 >> s;
        const int w = NV >> (s + 1);
        const bool up = (lane & mask) != 0;
#pragma unroll
        for (int k = 0; k < w; ++k) {
            const float send = up ? v[k] : v[k + w];
            const float keep = up ? v[k + w] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
        }
        if (up) idx += w;
    }
#pragma unroll
    for (int mask = 16 >> LOG; mask >= 1; mask >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], mask);
    return v[0];
}

// NV = 16: all ten screen-space values; NV = 8: the six the pose needs (mu', conic, depth).
// Value slots follow RecGrad: 0 d mu'_x, 1 d mu'_y, 2 d depth, 3 d opacity,
// 4..6 d conic (a, b, c), 8..10 d rgb; other slots stay zero.
template <int NV>
__global__ void __launch_bounds__(kTilePix, 5) k_backward(BackwardLaunch L) {
    __shared__ float4 sP0[kBatch], sC[kBatch], sQ[kBatch], sBox[kBatch];
    __shared__ float2 sP1[kBatch];
    __shared__ float sAcc[kBatch * kAccStride];
    __shared__ uint8_t sList[kTilePix / 32][kBatch];
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
    const int pu0 = (warp & 1) * kPatchW, pv0 = (warp >> 1) * kPatchH;
    const int lu = pu0 + (lane & (kPatchW - 1)), lv = pv0 + lane / kPatchW;
    const int px = tx * kTile + lu, py = ty * kTile + lv;
    const bool inside = px < vi.width && py < vi.height;
    const float x0 = (float)(tx * kTile), y0 = (float)(ty * kTile);
    const float fu = (float)lu, fv = (float)lv;
    const float pu_lo = (float)pu0, pu_hi = (float)(pu0 + kPatchW - 1);
    const float pv_lo = (float)pv0, pv_hi = (float)(pv0 + kPatchH - 1);
    const Settings &S = L.s;
    const float thr = S.log2_alpha_min;

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
    float B0 = 0.f, B1 = 0.f, B2 = 0.f, B3 = 0.f, B4 = 0.f;  // colour behind, per channel
    uint32_t n_eval = 0, n_contrib = 0;

    for (int64_t b0 = nmax ? (int64_t)((nmax - 1) / kBatch) * kBatch : -1; b0 >= 0; b0 -= kBatch) {
        const int cnt = (int)min((uint32_t)kBatch, nmax - (uint32_t)b0);
        if (tid < cnt) {
            const uint32_t r = L.ws.sorted[start + (uint32_t)b0 + tid];
            if (r < rec_slots(L.d)) {
                const Rec rr = L.ws.rec[r];
                const Footprint f = stage_footprint(rr.a, rr.b, x0, y0);
                sP0[tid] = f.p0;
                sP1[tid] = f.p1;
                sC[tid] = make_float4(rr.c.x, rr.c.y, rr.c.z, rr.a.z);
                sQ[tid] = make_float4(rr.b.x, rr.b.y, rr.b.z, rr.a.w);
                sBox[tid] = stage_box(rr.b, f.p0.y, f.p0.z);
            } else {
                sBox[tid] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
            }
        }
#pragma unroll
        for (int k = 0; k < kAccStride; ++k) sAcc[tid * kAccStride + k] = 0.f;
        __syncthreads();
        // this warp's list, limited to entries below its largest contributor count
        const int wcnt = (int)min((int64_t)cnt, (int64_t)wlast - b0);
        int nl = 0;
        for (int k = 0; k < wcnt; k += 32) {
            const int j = k + lane;
            bool hit = false;
            if (j < wcnt) {
                const float4 bx = sBox[j];
                hit = bx.y >= pu_lo && bx.x <= pu_hi && bx.w >= pv_lo && bx.z <= pv_hi;
            }
            const uint32_t m = __ballot_sync(0xffffffffu, hit);
            if (hit) sList[warp][nl + __popc(m & ((1u << lane) - 1u))] = (uint8_t)j;
            nl += __popc(m);
        }
        __syncwarp();
        for (int e = nl - 1; e >= 0; --e) {
            const int j = sList[warp][e];
            const uint32_t idx = (uint32_t)b0 + (uint32_t)j;
            float vals[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) vals[k] = 0.f;
            bool c = false;
            if (idx < last) {
                const PolyEval pe = eval_poly(fu, fv, sP0[j], sP1[j]);
                ++n_eval;
                if (pe.poly >= thr) {
                    c = true;
                    ++n_contrib;
                    const float araw = ex2_approx(pe.poly);
                    const float a = fminf(S.alpha_max, araw), om = 1.f - a;
                    T = T * __fdividef(1.f, om);  // transmittance in front of this Gaussian
                    const float4 Cc = sC[j];
                    const float d0 = Cc.x - B0, d1 = Cc.y - B1, d2 = Cc.z - B2, d3 = Cc.w - B3, d4 = 1.f - B4;
                    const float dalpha = T * (g0 * d0 + g1 * d1 + g2 * d2 + gD * d3 + gS * d4);
                    B0 += a * d0;
                    B1 += a * d1;
                    B2 += a * d2;
                    B3 += a * d3;
                    B4 += a * d4;
                    const float w = a * T;
                    vals[2] = w * gD;
                    if (araw < S.alpha_max) {
                        const float4 Qc = sQ[j];
                        const float dp = dalpha * a;
                        const float dx = pe.dx, dy = pe.dy;
                        vals[0] = dp * (Qc.x * dx + Qc.y * dy);
                        vals[1] = dp * (Qc.y * dx + Qc.z * dy);
                        const float hdp = -0.5f * dp;
                        vals[4] = hdp * dx * dx;
                        vals[5] = -dp * dx * dy;
                        vals[6] = hdp * dy * dy;
                        if constexpr (NV == 16) vals[3] = dalpha * araw / Qc.w;
                    }
                    if constexpr (NV == 16) {
                        vals[8] = w * g0;
                        vals[9] = w * g1;
                        vals[10] = w * g2;
                    }
                }
            }
            if (__any_sync(0xffffffffu, c)) {
                int slot;
                const float sum = warp_reduce_scatter<NV>(vals, lane, slot);
                if ((lane & (32 / NV - 1)) == 0 && slot < kAccStride && slot != 7 && slot != 11 && sum != 0.f)
                    atomicAdd(&sAcc[j * kAccStride + slot], sum);
            }
        }
        __syncthreads();
        if (tid < cnt) {
            const uint32_t r = L.ws.sorted[start + (uint32_t)b0 + tid];
            if (r < rec_slots(L.d)) {
                const float *a = sAcc + tid * kAccStride;
                const float4 v0 = make_float4(a[0], a[1], a[2], a[3]);
                const float4 v1 = make_float4(a[4], a[5], a[6], 0.f);
                if (v0.x != 0.f || v0.y != 0.f || v0.z != 0.f || v0.w != 0.f) atomicAdd(&L.ws.rec_grad[r].g0, v0);
                if (v1.x != 0.f || v1.y != 0.f || v1.z != 0.f) atomicAdd(&L.ws.rec_grad[r].g1, v1);
                if constexpr (NV == 16) {
                    const float4 v2 = make_float4(a[8], a[9], a[10], 0.f);
                    if (v2.x != 0.f || v2.y != 0.f || v2.z != 0.f) atomicAdd(&L.ws.rec_grad[r].g2, v2);
                }
            }
        }
        __syncthreads();
    }
    count_pairs(n_eval, n_contrib, &L.ws.hdr->bwd_evals, &L.ws.hdr->bwd_contrib);
}

cudaError_t launch_backward(const BackwardLaunch &L, cudaStream_t st) {
    if (L.d.T == 0) return cudaSuccess;
    if (L.pose_only)
        k_backward<8><<<L.d.T, kTilePix, 0, st>>>(L);
    else
        k_backward<16><<<L.d.T, kTilePix, 0, st>>>(L);
    return cudaGetLastError();
}

}  // namespace gsk
