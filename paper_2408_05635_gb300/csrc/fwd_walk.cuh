// fwd_walk.cuh -- one pixel's front-to-back walk of Eqs. 2-4 over a warp's list of staged
// Gaussians, shared by k_forward and the fused tracking kernel.
#pragma once

#include "gs_internal.cuh"

namespace gsk {

// The walk's pixel state: transmittance, colour and depth sums, the last contributor's
// list position + 1, the entries evaluated up to and including the last contributor (the
// entries the reverse walk evaluates for this pixel), and whether the walk has stopped on
// t_min.
struct FwdPixel {
    float T, cr, cg, cb, D;
    uint32_t last;
    uint32_t eval_last;
    bool done;
};

// Walk `px` over list entries [0, nl) (byte offsets into the staged arrays) of the batch
// that starts at list position b0.
// Two entries per step: both footprints are evaluated before the state takes the front
// one, then the back one, so the two evaluations overlap.  An entry that misses the pixel
// has alpha 0, which leaves every sum and T exactly as they are, and T >= t_min holds
// before every step, so the transmittance after both entries falls below t_min only when
// one of them stops the walk: one comparison per step, and the rare stop is resolved
// after it (the front entry if it alone reaches t_min, else the back one).  n_eval counts
// the entries evaluated before the stop (inclusive), n_contrib the contributions.
__device__ __forceinline__ void fwd_walk_batch(FwdPixel &px, const uint16_t *list, int nl, uint32_t b0,
                                               const float4 *sP0, const float4 *sP1, const float4 *sC, float2 uv,
                                               float thr, float amax, float tmin, uint32_t &n_eval,
                                               uint32_t &n_contrib) {
    float T = px.T;
    // (colour r, g) and (colour b, depth): each pair takes one two-lane FMA per entry
    float2 rg = make_float2(px.cr, px.cg), bD = make_float2(px.cb, px.D);
    int le = 0;  // list index + 1 of the last contributor in this batch (0: none)
    int e = 0;
    uint32_t contrib = 0;
    for (; e + 1 < nl; e += 2) {
        const int jA = list[e], jB = list[e + 1];
        const float pA = eval_poly(uv, at_off(sP0, jA), p1_at(sP1, jA)).poly;
        const float pB = eval_poly(uv, at_off(sP0, jB), p1_at(sP1, jB)).poly;
        const float4 CA = at_off(sC, jA), CB = at_off(sC, jB);
        const bool cA = pA >= thr, cB = pB >= thr;
        const float aA = cA ? fminf(amax, ex2_approx(pA)) : 0.f;
        const float aB = cB ? fminf(amax, ex2_approx(pB)) : 0.f;
        const float TA = T * (1.f - aA), TB = TA * (1.f - aB);
        if (TB < tmin) {
            px.done = true;
            if (TA < tmin) {  // the front entry stops the walk
                e += 1;
                break;
            }
            const float w = aA * T;  // the front entry (if it hits) contributes, the back one stops
            rg = __ffma2_rn(make_float2(CA.x, CA.y), make_float2(w, w), rg);
            bD = __ffma2_rn(make_float2(CA.z, CA.w), make_float2(w, w), bD);
            T = TA;
            le = cA ? e + 1 : le;
            contrib += (uint32_t)cA;
            e += 2;
            break;
        }
        const float w = aA * T, v = aB * TA;
        rg = __ffma2_rn(make_float2(CA.x, CA.y), make_float2(w, w), rg);
        bD = __ffma2_rn(make_float2(CA.z, CA.w), make_float2(w, w), bD);
        rg = __ffma2_rn(make_float2(CB.x, CB.y), make_float2(v, v), rg);
        bD = __ffma2_rn(make_float2(CB.z, CB.w), make_float2(v, v), bD);
        T = TB;
        le = cB ? e + 2 : (cA ? e + 1 : le);
        contrib += (uint32_t)cA + (uint32_t)cB;
    }
    if (!px.done && e < nl) {  // an odd last entry
        const int j = list[e];
        const float poly = eval_poly(uv, at_off(sP0, j), p1_at(sP1, j)).poly;
        ++e;
        if (poly >= thr) {
            const float alpha = fminf(amax, ex2_approx(poly));
            const float Tn = T * (1.f - alpha);
            if (Tn < tmin) {
                px.done = true;
            } else {
                const float w = alpha * T;
                const float4 Cc = at_off(sC, j);
                rg = __ffma2_rn(make_float2(Cc.x, Cc.y), make_float2(w, w), rg);
                bD = __ffma2_rn(make_float2(Cc.z, Cc.w), make_float2(w, w), bD);
                T = Tn;
                le = e;
                ++contrib;
            }
        }
    }
    if (le > 0) {
        px.last = b0 + (uint32_t)(list[le - 1] >> 4) + 1u;
        px.eval_last = n_eval + (uint32_t)le;
    }
    n_eval += (uint32_t)e;
    n_contrib += contrib;
    px.T = T;
    px.cr = rg.x;
    px.cg = rg.y;
    px.cb = bD.x;
    px.D = bD.y;
}

}  // namespace gsk
