// bwd_walk.cuh -- the per-pixel step and the warp reductions of the reverse compositing
// walk (differentiating Eqs. 2-4), shared by k_backward and the fused tracking kernel.
#pragma once

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

// Butterfly reduce-scatter of six per-lane values: three exchanges over lane bit 4, two
// over bit 3 (the third value of each half is summed by both partners), one over bit 2,
// then a plain sum over bits 1 and 0.  Value 3 * b4 + (b2 ? 2 : b3) ends in the lane;
// owners are the lanes with bits 1, 0 clear and not both of bits 3, 2 set.
__device__ __forceinline__ float warp_reduce_scatter6(float v0, float v1, float v2, float v3, float v4,
                                                      float v5, int lane) {
    const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0, h2 = (lane & 4) != 0;
    const float u0 = (h4 ? v3 : v0) + __shfl_xor_sync(0xffffffffu, h4 ? v0 : v3, 16);
    const float u1 = (h4 ? v4 : v1) + __shfl_xor_sync(0xffffffffu, h4 ? v1 : v4, 16);
    const float u2 = (h4 ? v5 : v2) + __shfl_xor_sync(0xffffffffu, h4 ? v2 : v5, 16);
    const float a = (h3 ? u1 : u0) + __shfl_xor_sync(0xffffffffu, h3 ? u0 : u1, 8);
    const float b = u2 + __shfl_xor_sync(0xffffffffu, u2, 8);
    float c = (h2 ? b : a) + __shfl_xor_sync(0xffffffffu, h2 ? a : b, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// Joint reduce-scatter of two Gaussians' six values in 13 shuffles instead of two times
// eight: six exchanges over lane bit 4, three over bit 3, two over bit 2 (the third value of
// each half is summed by both partners), one over bit 1 and a plain sum over bit 0.  The
// values come placed per lane: `keep` holds the Gaussian the lane keeps after the exchange
// over bit 4 (the second one for lanes with bit 4 set), `send` the other, so the first
// round needs no selection.  Value 3 * b3 + (b1 ? 2 : b2) of Gaussian b4 ends in the lane;
// owners are the lanes with bit 0 clear and not both of bits 2, 1 set (twelve of them).
__device__ __forceinline__ float warp_reduce_scatter12(const float (&keep)[6], const float (&send)[6], int lane) {
    const bool h3 = (lane & 8) != 0, h2 = (lane & 4) != 0, h1 = (lane & 2) != 0;
    float u[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) u[k] = keep[k] + __shfl_xor_sync(0xffffffffu, send[k], 16);
    float w[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) w[m] = (h3 ? u[3 + m] : u[m]) + __shfl_xor_sync(0xffffffffu, h3 ? u[m] : u[3 + m], 8);
    const float x = (h2 ? w[1] : w[0]) + __shfl_xor_sync(0xffffffffu, h2 ? w[0] : w[1], 4);
    const float y = w[2] + __shfl_xor_sync(0xffffffffu, w[2], 4);
    float c = (h1 ? y : x) + __shfl_xor_sync(0xffffffffu, h1 ? x : y, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// One back-to-front step of the pose-only walk for this lane's pixel: updates T and g.B
// and returns what the step's six moment terms are made of (all zero where c is false):
// dp = dL/dpower, (dx, dy) and a T g_D.
struct StepMom {
    float dp;
    float2 d;
    float wgD;
};

__device__ __forceinline__ StepMom bwd_step(bool c, const PolyEval &pe, float4 Cc, float g0, float g1, float g2,
                                            float gD, float gS, float amax, float &T, float &GB) {
    const float araw = ex2_approx(pe.poly);
    const float a = c ? fminf(amax, araw) : 0.f;
    if (c) T = T * __fdividef(1.f, 1.f - a);  // transmittance in front of this Gaussian
    const float gv = fmaf(g0, Cc.x, fmaf(g1, Cc.y, fmaf(g2, Cc.z, fmaf(gD, Cc.w, gS))));
    const float diff = gv - GB;
    const float dalpha = T * diff;
    GB = fmaf(a, diff, GB);
    StepMom m;
    m.dp = araw < amax ? dalpha * a : 0.f;
    m.d = pe.d;
    m.wgD = (a * T) * gD;
    return m;
}

// The six moment terms dp dx, dp dy, a T g_D, dp dx^2, dp dx dy, dp dy^2 of a step.
__device__ __forceinline__ void moments6(const StepMom &m, float (&v)[6]) {
    const float2 dpd = __fmul2_rn(make_float2(m.dp, m.dp), m.d);    // (dp dx, dp dy)
    const float2 mx = __fmul2_rn(make_float2(dpd.x, dpd.x), m.d);   // (dp dx dx, dp dx dy)
    v[0] = dpd.x;
    v[1] = dpd.y;
    v[2] = m.wgD;
    v[3] = mx.x;
    v[4] = mx.y;
    v[5] = dpd.y * m.d.y;
}

// Two steps (A, the back one, first) and their moments placed for warp_reduce_scatter12:
// lanes with bit 4 set keep B's and send A's.
__device__ __forceinline__ float bwd_pair_reduce(bool cA, const PolyEval &pA, float4 CA, bool cB, const PolyEval &pB,
                                                 float4 CB, float g0, float g1, float g2, float gD, float gS,
                                                 float amax, float &T, float &GB, int lane) {
    const StepMom mA = bwd_step(cA, pA, CA, g0, g1, g2, gD, gS, amax, T, GB);
    const StepMom mB = bwd_step(cB, pB, CB, g0, g1, g2, gD, gS, amax, T, GB);
    const bool h4 = (lane & 16) != 0;
    StepMom mk, ms;
    mk.dp = h4 ? mB.dp : mA.dp;
    ms.dp = h4 ? mA.dp : mB.dp;
    mk.d = make_float2(h4 ? mB.d.x : mA.d.x, h4 ? mB.d.y : mA.d.y);
    ms.d = make_float2(h4 ? mA.d.x : mB.d.x, h4 ? mA.d.y : mB.d.y);
    mk.wgD = h4 ? mB.wgD : mA.wgD;
    ms.wgD = h4 ? mA.wgD : mB.wgD;
    float vk[6], vs[6];
    moments6(mk, vk);
    moments6(ms, vs);
    return warp_reduce_scatter12(vk, vs, lane);
}

}  // namespace gsk
