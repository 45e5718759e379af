// raster_fused.cu -- one tracking iteration's compositing in one block per tile: the
// front-to-back walk of Eqs. 2-4 with the fused combined loss (Sec. III-B), then, in the
// same block and from the same registers, the pose-only reverse walk that differentiates
// Eqs. 2-4.
//
// It computes what k_forward<loss> followed by k_backward<pose-only> compute (the same
// footprint code, the same per-warp lists, the same reduce-scatter; see raster_fwd.cu and
// raster_bwd.cu for the arithmetic), with three differences in how the work is laid out:
//   - each pixel's upstream gradient, final transmittance and last contributor stay in
//     registers between the walks (they are still written to the workspace, so a later
//     gs_backward finds the same state as after k_forward);
//   - the batch the forward staged last is usually the one the reverse walk starts with
//     (a tile's whole list when it holds at most one batch): it is not staged again, and
//     each warp cuts the list it built for it in the forward instead of building another;
//   - a tile's reverse walk starts as soon as its own forward ends, so the tiles that end
//     the forward (the longest lists, launched first) overlap the reverse walks of the
//     others instead of leaving SMs idle before a second kernel.
#include "bwd_walk.cuh"
#include "fwd_walk.cuh"
#include "gs_internal.cuh"
#include "tile_sort.cuh"

namespace gsk {

namespace {

__device__ __forceinline__ float sgnf(float x) { return (float)((x > 0.f) - (x < 0.f)); }

// Stage batch position tid of the tile's sorted list (record r) for both walks.
__device__ __forceinline__ void stage_one(const TrackTileLaunch &L, uint32_t r, float x0, float y0, float4 *sP0,
                                          float4 *sP1, float4 *sC, float4 *sQ, float4 *sBox, int tid) {
    if (r < rec_slots(L.d)) {
        const Rec rr = L.ws.rec[r];
        const Footprint f = stage_footprint(rr.a, rr.b, x0, y0);
        sP0[tid] = f.p0;
        sP1[tid] = f.p1;
        sC[tid] = make_float4(rr.c.x, rr.c.y, rr.c.z, rr.a.z);
        sQ[tid] = make_float4(rr.b.x, rr.b.y, rr.b.z, rr.a.w);
        sBox[tid] = stage_box(rr.b, -f.p0.x, -f.p0.y);
    } else {
        sBox[tid] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);  // empty: never listed
    }
}

}  // namespace

constexpr int kFusedScratch = (2 * kSortSmemKeys * 8 > kBatch * kAccStride * 4) ? 2 * kSortSmemKeys * 8
                                                                               : kBatch * kAccStride * 4;

// Four blocks per SM (64 registers a thread): with five (48 registers) the walks spill
// and issue more instructions, and the kernel is slower.
template <int NB, int LW>
__global__ void __launch_bounds__(kTilePix, 4) k_track_tile(TrackTileLaunch L) {
    static_assert(NB % 32 == 0 && NB <= kBatch, "batch depth: a multiple of 32, at most kBatch");
    static_assert(LW >= 3 && (1 << LW) * kPatchH <= kTilePix, "tile width: 8 to 32 pixels");
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    __shared__ float4 sP0[NB], sC[NB], sQ[NB], sBox[NB];
    __shared__ float4 sP1[NB];                     // (kuu, lo, -1/(2 kuu), -1/(2 kvv)): the stride of sP0, sC
    __shared__ uint16_t sList[kTilePix / 32][NB];  // byte offsets: 16 x batch position
    // the sort's two key buffers, then (reverse walk) the per-batch accumulators
    __shared__ __align__(16) unsigned char sScratch[kFusedScratch];
    unsigned long long *sKeys = reinterpret_cast<unsigned long long *>(sScratch);
    float *sAcc = reinterpret_cast<float *>(sScratch);
    __shared__ int s_view;
    __shared__ float s_loss[kTilePix / 32];
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

    uint32_t start;
    const uint32_t n = tile_entries(L.ws, L.d, tile, start);
    // this tile's list in (depth, Gaussian) order, unless the device-wide radix sort
    // (GS_SCHED_RADIX) has already ordered it
    if (!(L.d.flags & GS_SCHED_RADIX)) sort_tile(L.ws, start, (int)n, sKeys);

    // this pixel's targets: loaded once the first batch is staged (below), so their
    // latency (host memory when the frame is read in place) passes during the forward walk
    // (loaded at the start of the block instead, in-place reads made the kernel slower)
    const uint32_t HW = (uint32_t)vi.width * (uint32_t)vi.height;
    const uint32_t p = inside ? (uint32_t)py * (uint32_t)vi.width + (uint32_t)px : 0u;
    const uint32_t gp = vi.pix_base + p;
    float tr = 0.f, tg = 0.f, tb = 0.f, Dt = 0.f, pr = 0.f;
    bool targets_loaded = false;

    // ---------------------------------------------------------------- forward (Eqs. 2-4)
    FwdPixel walk{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !inside};
    uint32_t n_eval = 0, n_contrib = 0;
    int64_t staged = -1;  // first list entry of the batch now in shared memory (block-uniform)
    int nl_staged = 0;    // length of this warp's list of the staged batch (warp-uniform)
    for (uint32_t b0 = 0; b0 < n; b0 += NB) {
        if (__syncthreads_count(!walk.done) == 0) break;
        const uint32_t idx = b0 + tid;
        if (tid < NB && idx < n) stage_one(L, L.ws.sorted[start + idx], x0, y0, sP0, sP1, sC, sQ, sBox, tid);
        staged = b0;
        __syncthreads();
        if (!targets_loaded) {
            targets_loaded = true;
            if (inside) {
                const float *trgb = L.t_rgb + 3u * vi.pix_base;
                tr = trgb[p];
                tg = trgb[HW + p];
                tb = trgb[2u * HW + p];
                Dt = L.t_depth[gp];
                if (L.t_prior) pr = L.t_prior[gp];
            }
        }
        const int cnt = (int)min((uint32_t)NB, n - b0);
        if (__any_sync(0xffffffffu, !walk.done)) {
            const int nl = build_patch_list(sBox, sP0, sP1, sList[warp], cnt, lane, thr, pu_lo, pu_hi, pv_lo, pv_hi);
            nl_staged = nl;
            if (!walk.done)
                fwd_walk_batch(walk, sList[warp], nl, b0, sP0, sP1, sC, uv, thr, S.alpha_max, S.t_min, n_eval,
                               n_contrib);
        }
    }
    float T = walk.T;
    const float cr = walk.cr, cg = walk.cg, cb = walk.cb, D = walk.D;
    uint32_t last = walk.last;
    const float Sil = 1.f - T;  // Eq. 4 summed: 1 - prod(1 - a_i)
    count_pairs(n_eval, n_contrib, &L.ws.hdr->fwd_evals, &L.ws.hdr->fwd_contrib);

    // ---------------------------------------------------------------- fused loss
    if (!targets_loaded && inside) {  // an empty tile list: no batch was staged
        const float *trgb = L.t_rgb + 3u * vi.pix_base;
        tr = trgb[p];
        tg = trgb[HW + p];
        tb = trgb[2u * HW + p];
        Dt = L.t_depth[gp];
        if (L.t_prior) pr = L.t_prior[gp];
    }
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, gD = 0.f, gS = 0.f, l = 0.f;
    if (inside) {
        L.ws.t_final[gp] = T;
        L.ws.n_last[gp] = last;
        const bool valid = Dt > 0.f;
        const bool M = valid && Sil > S.sil_thresh;
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
        const uint32_t P = L.d.P;
        float *ug = L.ws.upstream + 3u * vi.pix_base;
        ug[p] = g0;
        ug[HW + p] = g1;
        ug[2u * HW + p] = g2;
        L.ws.upstream[3u * P + gp] = gD;
        L.ws.upstream[4u * P + gp] = gS;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if (lane == 0) s_loss[warp] = l;

    // ---------------------------------------------------------------- reverse walk (pose)
    if (!(g0 != 0.f || g1 != 0.f || g2 != 0.f || gD != 0.f || gS != 0.f)) last = 0;
    // the reverse walk evaluates this pixel's entries in front of its last contributor and
    // differentiates its contributions: the forward's counts up to that entry
    const uint32_t rev_eval = last ? walk.eval_last : 0u, rev_contrib = last ? n_contrib : 0u;
    uint32_t wlast = last;  // largest contributor count in the warp
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, off));
    if (lane == 0 && wlast) atomicMax(&s_nmax, wlast);
    __syncthreads();
    if (tid == 0) {
        DF s{0.f, 0.f};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = df_add(s, DF{s_loss[w], 0.f});
        L.ws.tile_loss[tile] = df_pack(s);
    }
    const uint32_t nmax = s_nmax;
    // the paired steps' joint reduction: value 3 b3 + (b1 ? 2 : b2) of Gaussian b4; the
    // single steps': value 3 b4 + (b2 ? 2 : b3)
    int my_slot = -1, pair_slot = -1;
    if ((lane & 1) == 0 && !((lane & 2) && (lane & 4))) {
        const int k = ((lane & 8) ? 3 : 0) + ((lane & 2) ? 2 : ((lane & 4) ? 1 : 0));
        pair_slot = k < 3 ? k : k + 1;  // values 0..5 -> slots 0, 1, 2, 4, 5, 6
    }
    if ((lane & 3) == 0 && !((lane & 8) && (lane & 4))) {
        const int k = ((lane & 16) ? 3 : 0) + ((lane & 4) ? 2 : ((lane & 8) ? 1 : 0));
        my_slot = k < 3 ? k : k + 1;
    }
    float GB = 0.f;  // g . (colour, depth, 1) of everything behind, back-to-front
    for (int64_t b0 = nmax ? (int64_t)((nmax - 1) / NB) * NB : -1; b0 >= 0; b0 -= NB) {
        const int cnt = (int)min((uint32_t)NB, nmax - (uint32_t)b0);
        if (b0 != staged && tid < cnt)
            stage_one(L, L.ws.sorted[start + (uint32_t)b0 + tid], x0, y0, sP0, sP1, sC, sQ, sBox, tid);
        if (tid < NB) {  // thread tid owns the accumulator row of batch position tid
#pragma unroll
            for (int k = 0; k < kAccStride; ++k) sAcc[tid * kAccStride + k] = 0.f;
        }
        __syncthreads();
        // this warp's list, limited to entries below its largest contributor count
        const int wcnt = (int)min((int64_t)cnt, (int64_t)wlast - b0);
        int nl = 0;
        if (b0 == staged) {
            // the batch the forward ended on: its list (ascending positions) is still in
            // sList, and the entries below wcnt are the list build_patch_list would give for
            // wcnt.  A warp whose pixels had all stopped before this batch kept an older
            // list, but then wlast <= b0 and no entry is below wcnt <= 0.
            for (int k = 0; k < nl_staged; k += 32) {
                const bool below = k + lane < nl_staged && (int)sList[warp][k + lane] < wcnt * 16;
                const int m = __popc(__ballot_sync(0xffffffffu, below));
                nl += m;
                if (m < 32) break;
            }
        } else {
            nl = build_patch_list(sBox, sP0, sP1, sList[warp], wcnt, lane, thr, pu_lo, pu_hi, pv_lo, pv_hi);
        }
        int e = nl - 1;
        // entries at byte offsets below lim are in front of this pixel's last contributor
        const int lim = (int)max(min((int64_t)last - b0, (int64_t)NB), (int64_t)0) * 16;
        // two Gaussians per step: the pixel state is updated in depth order (the back one
        // first), and the two reductions are independent, so they overlap
        for (; e >= 1; e -= 2) {
            const int jA = sList[warp][e], jB = sList[warp][e - 1];
            const PolyEval pA = eval_poly(uv, at_off(sP0, jA), p1_at(sP1, jA));
            const PolyEval pB = eval_poly(uv, at_off(sP0, jB), p1_at(sP1, jB));
            const bool cA = jA < lim && pA.poly >= thr, cB = jB < lim && pB.poly >= thr;
            if (!__any_sync(0xffffffffu, cA || cB)) continue;
            const float s2 = bwd_pair_reduce(cA, pA, at_off(sC, jA), cB, pB, at_off(sC, jB), g0, g1, g2, gD, gS,
                                             S.alpha_max, T, GB, lane);
            if (pair_slot >= 0 && s2 != 0.f)
                atomicAdd(&sAcc[(((lane & 16) ? jB : jA) >> 4) * kAccStride + pair_slot], s2);
        }
        for (; e >= 0; --e) {
            const int j = sList[warp][e];
            const PolyEval pe = eval_poly(uv, at_off(sP0, j), p1_at(sP1, j));
            const bool c = j < lim && pe.poly >= thr;
            if (!__any_sync(0xffffffffu, c)) continue;
            float v[6];
            moments6(bwd_step(c, pe, at_off(sC, j), g0, g1, g2, gD, gS, S.alpha_max, T, GB), v);
            const float sum = warp_reduce_scatter6(v[0], v[1], v[2], v[3], v[4], v[5], lane);
            if (my_slot >= 0 && sum != 0.f) atomicAdd(&sAcc[(j >> 4) * kAccStride + my_slot], sum);
        }
        __syncthreads();
        if (tid < cnt) {
            const uint32_t r = L.ws.sorted[start + (uint32_t)b0 + tid];
            if (r < rec_slots(L.d)) {
                const float *m = sAcc + tid * kAccStride;
                const float4 Q = sQ[tid];
                const float4 v0 = make_float4(Q.x * m[0] + Q.y * m[1], Q.y * m[0] + Q.z * m[1], m[2], 0.f);
                const float4 v1 = make_float4(-0.5f * m[4], -m[5], -0.5f * m[6], 0.f);
                if (v0.x != 0.f || v0.y != 0.f || v0.z != 0.f) atomicAdd(&L.ws.rec_grad[r].g0, v0);
                if (v1.x != 0.f || v1.y != 0.f || v1.z != 0.f) atomicAdd(&L.ws.rec_grad[r].g1, v1);
            }
        }
        __syncthreads();
        staged = -1;  // every later batch is staged again
    }
    count_pairs(rev_eval, rev_contrib, &L.ws.hdr->bwd_evals, &L.ws.hdr->bwd_contrib);
}

template <int NB, int LW>
cudaError_t launch_track_tile_nb(const TrackTileLaunch &L, cudaStream_t st) {
    return launch_dep(k_track_tile<NB, LW>, dim3(L.d.T), dim3(tile_threads(L.d)), st, L);
}

template <int NB>
cudaError_t launch_track_tile_lw(const TrackTileLaunch &L, cudaStream_t st) {
    switch (tile_lw(L.d)) {
        case 3: return launch_track_tile_nb<NB, 3>(L, st);
        case 4: return launch_track_tile_nb<NB, 4>(L, st);
        case 5: return launch_track_tile_nb<NB, 5>(L, st);
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_track_tile(const TrackTileLaunch &L, cudaStream_t st) {
    if (L.d.T == 0) return cudaSuccess;
    if (!L.t_rgb || !L.t_depth) return cudaErrorInvalidValue;
    // one batch depth for both walks; a batch stages at most one Gaussian per thread
    const uint32_t nb = L.d.fwd_batch ? L.d.fwd_batch : (uint32_t)kBatch;
    if (nb > tile_threads(L.d) || (L.d.bwd_batch ? L.d.bwd_batch : (uint32_t)kBatch) != nb)
        return cudaErrorInvalidValue;
    cudaError_t e;
    switch (nb) {
        case 256: e = launch_track_tile_lw<256>(L, st); break;
        case 128: e = launch_track_tile_lw<128>(L, st); break;
        case 64: e = launch_track_tile_lw<64>(L, st); break;
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace gsk
