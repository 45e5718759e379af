// gs_internal.cuh -- device data layout and helpers shared by the rasterizer kernels.
//
// Pipeline of one rendering pass (every step is a kernel of this library):
//   k_project   Gaussian x view: projection, opacity-aware support, compaction into
//               visible records, per-tile pair counts.
//   k_scan_tiles  tile offsets, tile launch order (longest lists first).
//   k_emit      visible record: one 64-bit key (depth bits << 32 | record) per tile met.
//   k_forward   tile: sort its keys by (depth, Gaussian index), then Eqs. 2-4 front to
//               back; optional fused combined loss.
//   k_backward  tile: reverse compositing; per-record screen-space gradients.
//   k_bproject  record: chain rule to parameters and pose; per-cell pose partials.
//   k_finalize  view: FP64 sums of the loss and pose partials; (tracking) the decoupled
//               Adam step.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gsk {

constexpr int kTile = 16;                 // default tile edge in pixels
constexpr int kTilePix = kTile * kTile;   // most pixels (= threads) per tile block
// A screen tile is tile_w x tile_h pixels, one thread each: tile_w in {8, 16, 32},
// tile_h in {4, 8, 16, 32}, 64 <= tile_w tile_h <= kTilePix (16 x 16 by default).  The
// warps of a tile block own 8 x 4 patches, tile_w / 8 of them per patch row.
constexpr int kBlock = 256;               // threads per Gaussian-parallel block
constexpr int kWarps = kBlock / 32;       // warps per Gaussian-parallel block
constexpr int kCell = kBlock;             // Gaussians (and record slots) per cell
constexpr int kBatch = 256;               // default (and largest) compositing batch depth
// The compositors are compiled for batch depths 64, 128 and 256 (Gaussians staged into
// shared memory per batch).  The first NB threads of the tile block stage one Gaussian
// each and own one accumulator row each, and the per-warp lists hold batch positions as
// bytes: NB must not exceed 256 nor the tile's thread count (the host checks the latter).
static_assert(kBatch <= kTilePix && kBatch <= 256, "a batch stages at most one Gaussian per tile thread");
constexpr int kSubMax = 4;                // most per-tile sub-buckets a workspace is laid out for
constexpr int kBigCell = 2;               // large records a cell needs to list them for k_emit's extra blocks
constexpr int kBigListCap = 2048;         // entries of that list (a listed record per extra warp and pass: 4)

enum ErrFlag : uint32_t { kErrRecords = 1u, kErrPairs = 2u, kErrTimeout = 4u };

// One view: intrinsics, image and tile-grid geometry, offsets in the concatenated arrays.
struct ViewInfo {
    float fx, fy, cx, cy;
    int32_t width, height, tiles_x, tiles_y;
    uint32_t tile_base;  // first global tile index of the view
    uint32_t pix_base;   // first pixel of the view in the concatenated planes
    float tan_lim_x, tan_lim_y;  // clamp of the image-plane tangent at which J is taken
    int32_t tile_lw, tile_lh;    // log2 of the tile width and height in pixels
};

// Tangent limit of the EWA Jacobian along one image axis: jac_clip half-extents of the
// view (the mean's x_c / z beyond it is clamped for J only); infinite when disabled.
inline float jacobian_tangent_limit(float jac_clip, int32_t extent, double focal) {
    return jac_clip > 0.f ? (float)((double)jac_clip * 0.5 * (double)extent / focal) : INFINITY;
}
static_assert(sizeof(ViewInfo) == 56, "ViewInfo layout");

// Small counters at the start of the workspace (cleared before every projection).
struct DevHeader {
    unsigned long long n_pairs;      // total (Gaussian, tile) pairs of the projection
    unsigned long long n_rec;        // visible (Gaussian, view) records of the projection
    unsigned long long fwd_evals;    // (pixel, Gaussian) footprints evaluated by k_forward
    unsigned long long fwd_contrib;  // ... of which contributed (alpha >= alpha_min, before the stop)
    unsigned long long bwd_evals;    // footprints evaluated by k_backward
    unsigned long long bwd_contrib;  // ... of which were differentiated
    uint32_t max_tile;               // longest tile list of the projection
    uint32_t n_big;                  // records listed in WsPtrs::big (the scan copies the count)
    unsigned long long pad1;
};
static_assert(sizeof(DevHeader) == 64, "DevHeader layout");

// Double-float: the unevaluated sum hi + lo of two FP32 values (about 46 significant bits
// after additions), added with Knuth's error-free TwoSum of the high parts followed by a
// Fast2Sum renormalisation (Dekker, 1971).  The fixed-order loss and pose sums use it so
// they run on the FP32 pipes: FP64 issue on this GPU is a small fraction of FP32.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, t);
    return DF{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}
__device__ __forceinline__ DF df_load(const float2 &x) { return DF{x.x, x.y}; }
__device__ __forceinline__ float2 df_pack(DF a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ DF df_shfl_xor(DF a, int mask) {
    return DF{__shfl_xor_sync(0xffffffffu, a.hi, mask), __shfl_xor_sync(0xffffffffu, a.lo, mask)};
}

// A visible (Gaussian, view) pair, as the compositors read it (48 bytes).
//   a = (mu'_x, mu'_y, depth, opacity)
//   b = (conic a, conic b, conic c, dmax2)   conic = inverse of Sigma' = [[a, b], [b, c]]
//   c = (r, g, b, bits of view * n + gaussian)
// Records live in cells: cell (v, k) holds the visible Gaussians of view v among
// Gaussians [256 k, 256 k + 256), packed at the front of its 256 slots in Gaussian
// order, so record index order is (view, Gaussian) order and no allocation counter is
// needed.
struct __align__(16) Rec {
    float4 a, b, c;
};

// Per-record screen-space gradient accumulators (48 bytes).
//   g0 = (d mu'_x, d mu'_y, d depth, d opacity), g1 = (d conic a, b, c, 0), g2 = (d r, g, b, 0)
struct __align__(16) RecGrad {
    float4 g0, g1, g2;
};

// Device pointers into one workspace (computed on the host from the problem sizes).
struct WsPtrs {
    uint32_t *err;         // ErrFlag bits, latched until gs_sync_status clears them
    DevHeader *hdr;
    uint32_t *tile_cnt;    // T x S, per-(tile, sub-bucket) pair counts (zero between projections)
    ViewInfo *views;       // V
    float *view_rt;        // V x 12, FP32 rotation and translation of each pose (k_project)
    uint32_t *cell_cnt;    // V x nblk, visible records per cell
    uint32_t *tile_start;  // T x S + 1, exclusive scan of the counts
    uint32_t *cursor;      // T x S, emission cursors
    uint32_t *tile_order;  // T, tiles by descending list length (launch order of the tile kernels)
    uint32_t *big;         // kBigListCap: large records of crowded cells (more than kSoloTiles
                           // candidate tiles, kBigCell of them in one cell), listed by k_project
                           // (count at tile_cnt[T x S], moved to hdr->n_big by the scan) and
                           // emitted by k_emit's extra blocks
    uint8_t *big_listed;   // V x nblk x 256: 1 where the record is in `big` (its cell's warps skip it)
    Rec *rec;              // V x nblk x 256 record slots
    RecGrad *rec_grad;     // same slots
    unsigned long long *keys;  // pair_capacity
    uint32_t *sorted;      // pair_capacity, record ids in (tile, depth, gaussian) order
    float *t_final;        // P, transmittance after the last contributor
    uint32_t *n_last;      // P, tile-list index + 1 of the last contributor
    float *upstream;       // 5 x P: dL/dC (planar like the images), dL/dD, dL/dS of the fused loss
    float2 *tile_loss;     // T, combined loss of each tile's pixels (fused loss), double-float
    float2 *pose_part;     // V x nblk x 6, pose-gradient sum of each cell's records, double-float
    unsigned long long *rkeys;  // pair_capacity: the radix sort's second key buffer
    uint32_t *rvals;       // pair_capacity: its second value buffer
    uint32_t *rhist;       // 256 x radix_blocks(pair_capacity) digit counts
    uint32_t *rtotal;      // 256 digit totals
    uint32_t *scan_part;   // the multi-block scan's per-block sums, longest lists, record
                           // counts and launch-order bucket counts, or nullptr (one-block scan)
};

// Multi-block form of the tile scan (problems with more counters than one block takes in
// one pass): kMBThreads threads a block, kMBPer counters a thread, kMBuckets launch-order
// buckets.  scan_blocks(c) blocks for c counters; ws.scan_part holds (3 + kMBuckets) words
// per block.
constexpr int kMBThreads = 256;
constexpr int kMBPer = 8;
constexpr uint32_t kMBChunk = (uint32_t)kMBThreads * kMBPer;
constexpr int kMBuckets = 64;
__host__ __device__ inline uint32_t scan_blocks(uint64_t counters) {
    return (uint32_t)((counters + kMBChunk - 1) / kMBChunk);
}

struct Dims {
    int64_t n;             // Gaussians
    int32_t V;             // views
    int32_t nblk;          // ceil(n / kBlock): cells per view
    uint32_t T;            // tiles over all views
    uint32_t S;            // sub-buckets per tile (1, 2 or 4): a tile's pairs are counted and
                           // placed through S counters picked by Gaussian index, so no single
                           // counter takes every pair of a crowded tile; the S sub-ranges are
                           // contiguous, so the tile's list is still one range
    uint32_t P;            // pixels over all views
    uint32_t pair_cap;
    uint32_t fwd_batch;    // Gaussians staged per forward batch: 64, 128 or 256 (0: kBatch)
    uint32_t bwd_batch;    // Gaussians staged per backward batch: 64, 128 or 256 (0: kBatch)
    uint32_t tile_threads; // threads (= pixels) of a tile block: tile_w x tile_h (0: kTilePix)
    uint32_t tile_lw;      // log2 of the tile width, 3 to 5 (0: 16-pixel tiles)
    uint32_t flags;        // GS_SCHED_* bits of the launch schedule
};

struct Settings {
    float alpha_min, alpha_max, t_min, dilation, z_near, sil_thresh;
    float log2_alpha_min;  // skip threshold on the footprint exponent (-inf when alpha_min = 0)
    float w_rgb, w_depth, w_vis, w_prior;
    double lr_rot, lr_trans, beta1, beta2, eps;
};

struct GaussPtrs {
    const float *means;
    const void *quats, *log_scales, *logits, *rgb;
};

// Block-wide sum of two per-thread counters, added once per block to the header.
__device__ __forceinline__ void count_pairs(uint32_t evals, uint32_t contrib, unsigned long long *e_out,
                                            unsigned long long *c_out) {
    __shared__ unsigned long long s_e, s_c;
    if (threadIdx.x == 0) s_e = s_c = 0ull;
    __syncthreads();
    const uint32_t we = __reduce_add_sync(0xffffffffu, evals), wc = __reduce_add_sync(0xffffffffu, contrib);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_e, (unsigned long long)we);
        atomicAdd(&s_c, (unsigned long long)wc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(e_out), "l"(s_e) : "memory");
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(c_out), "l"(s_c) : "memory");
    }
}

// Fire-and-forget global add (no value returned, so the thread does not wait for it).
__device__ __forceinline__ void red_add(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ------------------------------------------------------------------ attribute loads

template <int DT> __device__ __forceinline__ float ld_attr(const void *p, int64_t i);
template <> __device__ __forceinline__ float ld_attr<GS_F32>(const void *p, int64_t i) {
    return __ldg(static_cast<const float *>(p) + i);
}
template <> __device__ __forceinline__ float ld_attr<GS_BF16>(const void *p, int64_t i) {
    return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]);
}
template <> __device__ __forceinline__ float ld_attr<GS_F16>(const void *p, int64_t i) {
    return __half2float(static_cast<const __half *>(p)[i]);
}

// ------------------------------------------------------------------ geometry helpers

// Rotation matrix (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float R[9]) {
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - w * z);
    R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);
    R[7] = 2.f * (y * z + w * x);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

// Pose (7 doubles) -> FP32 rotation (9) and translation (3), an exactly specified FP32
// computation: every input rounded to FP32, |q|^2 summed left to right, the unit
// quaternion q / sqrt(|q|^2) with a correctly rounded square root and division, then the
// rotation entries with every operation rounded (no contraction).  The camera-frame
// depth below is therefore an exactly specified FP32 number: the depth order of
// Eqs. 2-4 and the near-plane test are decided on it.
__device__ __forceinline__ void load_pose(const double *pose, float Rt[12]) {
    float w = __double2float_rn(pose[0]), x = __double2float_rn(pose[1]);
    float y = __double2float_rn(pose[2]), z = __double2float_rn(pose[3]);
    const float ss = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(w, w), __fmul_rn(x, x)), __fmul_rn(y, y)), __fmul_rn(z, z));
    const float nrm = __fsqrt_rn(ss);
    w = __fdiv_rn(w, nrm);
    x = __fdiv_rn(x, nrm);
    y = __fdiv_rn(y, nrm);
    z = __fdiv_rn(z, nrm);
    Rt[0] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(__fmul_rn(y, y), __fmul_rn(z, z))));
    Rt[1] = __fmul_rn(2.f, __fsub_rn(__fmul_rn(x, y), __fmul_rn(w, z)));
    Rt[2] = __fmul_rn(2.f, __fadd_rn(__fmul_rn(x, z), __fmul_rn(w, y)));
    Rt[3] = __fmul_rn(2.f, __fadd_rn(__fmul_rn(x, y), __fmul_rn(w, z)));
    Rt[4] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(__fmul_rn(x, x), __fmul_rn(z, z))));
    Rt[5] = __fmul_rn(2.f, __fsub_rn(__fmul_rn(y, z), __fmul_rn(w, x)));
    Rt[6] = __fmul_rn(2.f, __fsub_rn(__fmul_rn(x, z), __fmul_rn(w, y)));
    Rt[7] = __fmul_rn(2.f, __fadd_rn(__fmul_rn(y, z), __fmul_rn(w, x)));
    Rt[8] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y))));
    Rt[9] = __double2float_rn(pose[4]);
    Rt[10] = __double2float_rn(pose[5]);
    Rt[11] = __double2float_rn(pose[6]);
}

// Camera-frame coordinate r of mean m: fma(R_r0, m0, fma(R_r1, m1, fma(R_r2, m2, t_r))).
__device__ __forceinline__ float cam_coord(const float Rt[12], int r, float m0, float m1, float m2) {
    return __fmaf_rn(Rt[3 * r], m0, __fmaf_rn(Rt[3 * r + 1], m1, __fmaf_rn(Rt[3 * r + 2], m2, Rt[9 + r])));
}

// Opacity-aware tile rectangle [tx0, tx1] x [ty0, ty1] of a support ellipse whose
// axis-aligned half-extents are hx, hy pixels (one pixel of margin).  Empty if tx0 > tx1.
__device__ __forceinline__ void tile_rect(const ViewInfo &vi, float mx, float my, float hx, float hy, int &tx0,
                                          int &tx1, int &ty0, int &ty1) {
    const float lim = 1.0e7f;
    const float x0 = fminf(fmaxf(floorf(mx - hx) - 1.f, -1.f), lim);
    const float x1 = fminf(fmaxf(ceilf(mx + hx) + 1.f, -1.f), lim);
    const float y0 = fminf(fmaxf(floorf(my - hy) - 1.f, -1.f), lim);
    const float y1 = fminf(fmaxf(ceilf(my + hy) + 1.f, -1.f), lim);
    const int px0 = max((int)x0, 0), px1 = min((int)x1, vi.width - 1);
    const int py0 = max((int)y0, 0), py1 = min((int)y1, vi.height - 1);
    if (px0 > px1 || py0 > py1 || x1 < 0.f || y1 < 0.f) {
        tx0 = 1; tx1 = 0; ty0 = 1; ty1 = 0;
        return;
    }
    tx0 = px0 >> vi.tile_lw; tx1 = px1 >> vi.tile_lw;  // px, py >= 0: shifts divide
    ty0 = py0 >> vi.tile_lh; ty1 = py1 >> vi.tile_lh;
}

// Does the support ellipse q(d) = a dx^2 + 2 b dx dy + c dy^2 <= dmax2 meet the
// rectangle of pixel centres [x0, x1] x [y0, y1]?  The minimum of the convex form over
// the rectangle is 0 when the centre is inside, otherwise it lies on an edge, where
// it is a 1-D quadratic minimised in closed form (ia = 1/a, ic = 1/c).  The minimiser
// only has to be close: the threshold carries a relative margin of 1e-3, far above the
// FP32 error, so no tile with a pixel at alpha >= alpha_min is dropped.  Every operation
// is an explicitly rounded intrinsic so k_project and k_emit take identical decisions.
__device__ __forceinline__ float qform(float a, float b, float c, float dx, float dy) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a, __fmul_rn(dx, dx)), __fmul_rn(2.f, __fmul_rn(b, __fmul_rn(dx, dy)))),
                     __fmul_rn(c, __fmul_rn(dy, dy)));
}

__device__ __forceinline__ bool ellipse_meets_rect(float mx, float my, float a, float b, float c, float ia, float ic,
                                                   float dmax2, float x0, float x1, float y0, float y1) {
    if (!(dmax2 < INFINITY)) return true;
    if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return true;
    const float lx = __fsub_rn(x0, mx), hx = __fsub_rn(x1, mx);
    const float ly = __fsub_rn(y0, my), hy = __fsub_rn(y1, my);
    const float nb = -b;
    float best = INFINITY;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dx = e ? hx : lx;  // vertical edge: dy free, minimum at dy = -b dx / c
        const float dy = fminf(fmaxf(__fmul_rn(__fmul_rn(nb, dx), ic), ly), hy);
        best = fminf(best, qform(a, b, c, dx, dy));
        const float ey = e ? hy : ly;  // horizontal edge: dx free, minimum at dx = -b dy / a
        const float ex = fminf(fmaxf(__fmul_rn(__fmul_rn(nb, ey), ia), lx), hx);
        best = fminf(best, qform(a, b, c, ex, ey));
    }
    return best <= __fadd_rn(__fmul_rn(dmax2, 1.001f), 1e-3f);
}

// Pixel-centre rectangle of tile (tx, ty) >= 0, clipped to the image.
__device__ __forceinline__ void tile_bounds(const ViewInfo &vi, int tx, int ty, float &x0, float &x1, float &y0,
                                            float &y1) {
    x0 = (float)(tx << vi.tile_lw);
    y0 = (float)(ty << vi.tile_lh);
    x1 = (float)min(((tx + 1) << vi.tile_lw) - 1, vi.width - 1);
    y1 = (float)min(((ty + 1) << vi.tile_lh) - 1, vi.height - 1);
}

// ------------------------------------------------------------------ per-tile footprint
//
// For a tile with origin (x0, y0) and tile-local pixel centre (u, v) = (px - x0, py - y0),
// the footprint of Eq. 1, alpha_raw = o exp(power) with
//   power = -1/2 [a dx^2 + 2 b dx dy + c dy^2],  (dx, dy) = (u - cu, v - cv),
//   (cu, cv) = mu' - (x0, y0),
// is evaluated as alpha_raw = 2^poly with
//   poly = dx (kuu dx + kuv dy) + kvv dy^2 + lo,
//   kuu = -L a / 2, kuv = -L b, kvv = -L c / 2, lo = log2 o,   L = log2(e),
// so log2(e) and the opacity are folded into the staged coefficients; per pixel the
// footprint costs two subtractions, five multiply-adds and one ex2.  (Expanding the
// quadratic in u, v would save two operations but cancels catastrophically for sharp
// Gaussians centred far from the tile origin.)  A Gaussian is skipped where
// poly < log2(alpha_min).  Staging and evaluation use explicitly rounded operations and
// are shared by the forward and the backward, so both take bit-identical decisions.
// The staged layout pairs the operands of Blackwell's two-lane FP32 instructions: the
// negated centre (dx and dy in one addition: u + (-cu) is u - cu exactly) and the two
// coefficients multiplied by dy (one multiplication); each lane of those instructions
// rounds like the scalar operation, so the values are those of the scalar sequence.
constexpr float kLog2e = 1.4426950408889634f;

struct Footprint {
    float4 p0;  // (-cu, -cv, kuv, kvv)
    float4 p1;  // (kuu, lo, -1/(2 kuu), -1/(2 kvv)): the last two for footprint_meets_rect
};

// Programmatic dependent launch.  The kernels of a tracking iteration form one chain on a
// stream; launched with launch_dep, a kernel's blocks may be scheduled while its
// predecessor's last blocks still run (the predecessor lets them in with
// griddep_launch_dependents, or by exiting), and each block first waits in griddep_wait
// until the predecessor grid has completed and its memory is visible.  Every kernel
// launched this way calls griddep_wait before touching global memory, so completion stays
// transitive along the chain.  Both are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
inline cudaError_t launch_dep(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ Footprint stage_footprint(const float4 A, const float4 B, float x0, float y0) {
    Footprint f;
    f.p0 = make_float4(__fsub_rn(x0, A.x), __fsub_rn(y0, A.y), __fmul_rn(-kLog2e, B.y), __fmul_rn(-0.5f * kLog2e, B.z));
    const float kuu = __fmul_rn(-0.5f * kLog2e, B.x);
    f.p1 = make_float4(kuu, lg2_approx(A.w), -0.5f / kuu, -0.5f / f.p0.w);
    return f;
}

// Conservative support box of a staged Gaussian in tile-local pixel coordinates
// (umin, umax, vmin, vmax): the ellipse poly >= log2(alpha_min) has half-extents
// sqrt(dmax2 Sigma'_xx), sqrt(dmax2 Sigma'_yy), widened by a relative 1e-3 and 0.01 px so
// FP32 rounding can never drop a pixel with alpha >= alpha_min.
// a b - c d with Kahan's fused correction (analysed by Jeannerod, Louvet and Muller, 2013):
// the rounding error of c d is recovered exactly by an FMA, so the difference of two
// nearly equal products keeps ~2 ulp of relative accuracy instead of losing the digits the
// products share.  Explicit intrinsics: every caller computes bit-identical results.
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

// Tiles [a0, a1] of row ty (within the record's tile columns [tx0, tx1]) that the support
// ellipse q(d) <= R, R = dmax2 (1 + 1e-3) + 1e-3 (the margin of ellipse_meets_rect), meets.
// The ellipse cut by the row's band of pixel centres [y0, y1] is convex, so its x-extent is
// one interval: on the right boundary x = mx + (-b dy + sqrt(a R - det dy^2)) / a, concave
// in dy = y - my, the maximum mx + sqrt(R c / det) is reached at dy = -b sqrt(R / (c det)),
// and outside the band at the nearer band edge; the left boundary mirrors it.  A tile
// meets the ellipse iff its pixel-centre columns overlap that interval, so this finds the
// same tiles as testing each tile of the row, at the cost of one row.  The interval is
// widened by 1e-3 px + 1e-6 |x| against the rounding of the square roots.  Explicitly
// rounded operations: k_project and k_emit enumerate identical tiles.  The quantities that
// do not depend on the row (RowSpan) are computed once per record by row_span_setup.
struct RowSpan {
    float mx, my, b, R, det, Y, X, t, ia, aR;  // aR = a R
    bool all;                                  // unbounded support: every column
};

__device__ __forceinline__ RowSpan row_span_setup(float mx, float my, float a, float b, float c, float dmax2) {
    RowSpan s;
    s.mx = mx;
    s.my = my;
    s.b = b;
    s.all = !(dmax2 < INFINITY);
    s.R = __fadd_rn(__fmul_rn(dmax2, 1.001f), 1e-3f);
    s.det = diff_of_products(a, c, b, b);
    s.aR = __fmul_rn(a, s.R);
    s.Y = __fsqrt_rn(__fdiv_rn(s.aR, s.det));                         // y half-extent of the ellipse
    s.X = __fsqrt_rn(__fdiv_rn(__fmul_rn(s.R, c), s.det));            // x half-extent of the ellipse
    s.t = __fmul_rn(b, __fsqrt_rn(__fdiv_rn(s.R, __fmul_rn(c, s.det))));  // |dy| of the x-extremes
    s.ia = __fdiv_rn(1.f, a);
    return s;
}

__device__ __forceinline__ void row_span(const ViewInfo &vi, const RowSpan &s, int ty, int tx0, int tx1, int &a0,
                                         int &a1) {
    a0 = tx0;
    a1 = tx1;
    if (s.all) return;
    const float yb0 = (float)(ty << vi.tile_lh), yb1 = (float)min(((ty + 1) << vi.tile_lh) - 1, vi.height - 1);
    const float ly = fmaxf(__fsub_rn(yb0, s.my), -s.Y), hy = fminf(__fsub_rn(yb1, s.my), s.Y);
    if (!(ly <= hy)) {
        a0 = 1;
        a1 = 0;
        return;
    }
    // boundary offsets at the band edges: -b dy / a -+ sqrt(a R - det dy^2) / a
    const float rl = __fsqrt_rn(fmaxf(__fsub_rn(s.aR, __fmul_rn(s.det, __fmul_rn(ly, ly))), 0.f));
    const float rh = __fsqrt_rn(fmaxf(__fsub_rn(s.aR, __fmul_rn(s.det, __fmul_rn(hy, hy))), 0.f));
    const float cl = __fmul_rn(__fmul_rn(-s.b, ly), s.ia), ch = __fmul_rn(__fmul_rn(-s.b, hy), s.ia);
    float xr, xl;
    if (-s.t >= ly && -s.t <= hy)
        xr = s.X;
    else
        xr = fmaxf(__fadd_rn(cl, __fmul_rn(rl, s.ia)), __fadd_rn(ch, __fmul_rn(rh, s.ia)));
    if (s.t >= ly && s.t <= hy)
        xl = -s.X;
    else
        xl = fminf(__fsub_rn(cl, __fmul_rn(rl, s.ia)), __fsub_rn(ch, __fmul_rn(rh, s.ia)));
    xl = __fsub_rn(__fadd_rn(s.mx, xl), __fadd_rn(1e-3f, __fmul_rn(1e-6f, fabsf(__fadd_rn(s.mx, xl)))));
    xr = __fadd_rn(__fadd_rn(s.mx, xr), __fadd_rn(1e-3f, __fmul_rn(1e-6f, fabsf(__fadd_rn(s.mx, xr)))));
    // tile tx spans pixel centres [TW tx, TW tx + TW - 1]: it meets [xl, xr] iff
    // TW tx + TW - 1 >= xl and TW tx <= xr (TW a power of two: multiplying by 1 / TW is
    // exact, the same as dividing)
    const float TW = (float)(1 << vi.tile_lw), iTW = __fdiv_rn(1.f, TW);
    const float lo = fmaxf(ceilf(__fmul_rn(__fsub_rn(xl, __fsub_rn(TW, 1.f)), iTW)), -1.f);
    const float hi = fminf(floorf(__fmul_rn(xr, iTW)), 1.0e7f);
    a0 = max(tx0, (int)lo);
    a1 = min(tx1, (int)hi);
}

__device__ __forceinline__ float4 stage_box(const float4 B, float cu, float cv) {
    const float detc = diff_of_products(B.x, B.z, B.y, B.y);
    if (!(detc > 0.f) || !(B.w < INFINITY)) return make_float4(-INFINITY, INFINITY, -INFINITY, INFINITY);
    const float hx = sqrtf(B.w * B.z / detc) * 1.001f + 0.01f;
    const float hy = sqrtf(B.w * B.x / detc) * 1.001f + 0.01f;
    return make_float4(cu - hx, cu + hx, cv - hy, cv + hy);
}

// Pixel layout of a tile block of width 2^lw: warp w owns the 8 x 4 patch at
// ((w mod 2^(lw-3)) * 8, (w >> (lw-3)) * 4); lane l its pixel (l & 7, l >> 3) inside it.
constexpr int kPatchW = 8, kPatchH = 4;

struct PolyEval {
    float2 d;  // (dx, dy)
    float poly;
};

// poly at the tile-local pixel centre uv = (u, v): dx = u - cu, dy = v - cv,
// t = kuu dx + kuv dy (kuv dy rounded first), poly = dx t + (kvv dy dy + lo).
__device__ __forceinline__ PolyEval eval_poly(float2 uv, float4 p0, float2 p1) {
    PolyEval e;
    e.d = __fadd2_rn(uv, make_float2(p0.x, p0.y));
    const float2 m = __fmul2_rn(make_float2(p0.z, p0.w), make_float2(e.d.y, e.d.y));  // (kuv dy, kvv dy)
    const float t = __fmaf_rn(p1.x, e.d.x, m.x);
    e.poly = __fmaf_rn(e.d.x, t, __fmaf_rn(m.y, e.d.y, p1.y));
    return e;
}

// Can a pixel position of the rectangle [u_lo, u_hi] x [v_lo, v_hi] (tile-local) reach
// poly >= thr, i.e. alpha >= alpha_min?  poly = lo + kuu dx^2 + kuv dx dy + kvv dy^2 has
// a concave quadratic part (kuu, kvv < 0: the conic is positive definite), whose maximum
// over the rectangle is 0 with the mean inside and otherwise lies on the boundary: on each
// edge, the maximiser of a concave quadratic in one variable, clamped to the edge.  The
// comparison keeps a margin of 2^-16 of the terms' magnitude over the rectangle (FP32
// rounding of this maximum, and of eval_poly at any pixel of it, is a few ulp of that), so
// no entry with a pixel at alpha >= alpha_min is dropped; degenerate footprints pass.
__device__ __forceinline__ bool footprint_meets_rect(float4 p0, float4 p1, float thr, float u_lo, float u_hi,
                                                     float v_lo, float v_hi) {
    const float kuu = p1.x, kuv = p0.z, kvv = p0.w, lo = p1.y;
    if (!(kuu < 0.f && kvv < 0.f)) return true;
    const float x0 = u_lo + p0.x, x1 = u_hi + p0.x, y0 = v_lo + p0.y, y1 = v_hi + p0.y;
    float q = 0.f;  // max of the quadratic part over the rectangle
    if (!(x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f)) {
        const float ru = p1.z, rv = p1.w;  // -0.5 / kuu, -0.5 / kvv, divided once at staging
        const auto f = [&](float dx, float dy) { return fmaf(dx, fmaf(kuu, dx, kuv * dy), kvv * dy * dy); };
        const float ya = fminf(fmaxf(kuv * x0 * rv, y0), y1), yb = fminf(fmaxf(kuv * x1 * rv, y0), y1);
        const float xa = fminf(fmaxf(kuv * y0 * ru, x0), x1), xb = fminf(fmaxf(kuv * y1 * ru, x0), x1);
        q = fmaxf(fmaxf(f(x0, ya), f(x1, yb)), fmaxf(f(xa, y0), f(xb, y1)));
    }
    const float DX = fmaxf(fabsf(x0), fabsf(x1)), DY = fmaxf(fabsf(y0), fabsf(y1));
    const float mag = fabsf(lo) - kuu * DX * DX + fabsf(kuv) * DX * DY - kvv * DY * DY;
    return lo + q >= thr - 0x1p-16f * mag;
}

// Staged Gaussians are addressed by byte offset: a warp's list holds 16 x the batch
// position, and sP0, sP1 and sC all have a 16-byte stride, so one list entry addresses
// all three without index arithmetic.
template <class T>
__device__ __forceinline__ const T &at_off(const T *base, int off) {
    return *reinterpret_cast<const T *>(reinterpret_cast<const char *>(base) + off);
}
__device__ __forceinline__ float2 p1_at(const float4 *sP1, int off) {
    const float4 &q = at_off(sP1, off);
    return make_float2(q.x, q.y);
}

// A warp's list of the batch positions [0, cnt) whose footprint reaches its pixel
// rectangle [pu_lo, pu_hi] x [pv_lo, pv_hi]: the support box first, then the exact
// footprint test; entries are byte offsets (16 x position) in ascending order.  Returns
// the count (warp-uniform).
__device__ __forceinline__ int build_patch_list(const float4 *sBox, const float4 *sP0, const float4 *sP1,
                                                uint16_t *list, int cnt, int lane, float thr, float pu_lo,
                                                float pu_hi, float pv_lo, float pv_hi) {
    int nl = 0;
    for (int k = 0; k < cnt; k += 32) {
        const int j = k + lane;
        bool hit = false;
        if (j < cnt) {
            const float4 bx = sBox[j];
            hit = bx.y >= pu_lo && bx.x <= pu_hi && bx.w >= pv_lo && bx.z <= pv_hi;
            if (hit) hit = footprint_meets_rect(sP0[j], sP1[j], thr, pu_lo, pu_hi, pv_lo, pv_hi);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) list[nl + __popc(m & ((1u << lane) - 1u))] = (uint16_t)(j << 4);
        nl += __popc(m);
    }
    __syncwarp();
    return nl;
}

// Global tile -> view (binary search over the views' first tiles).
__device__ __forceinline__ int view_of_tile(const ViewInfo *views, int V, uint32_t tile) {
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Entries of a tile's list: [start, start + count) of the key / sorted arrays, clamped to
// the pair capacity so an overflow (latched in the error flags) can never make a kernel
// read past its buffers.  k_project and k_emit enumerate the same (record, tile) pairs,
// so every slot of the range is written; record ids are bounds-checked where used
// (rec_slots(d) = V x nblk x 256).
__device__ __forceinline__ uint32_t tile_entries(const WsPtrs &ws, const Dims &d, uint32_t tile, uint32_t &start) {
    start = min(ws.tile_start[tile * d.S], d.pair_cap);
    const uint32_t end = min(ws.tile_start[(tile + 1) * d.S], d.pair_cap);
    return end > start ? end - start : 0u;
}

__device__ __host__ __forceinline__ uint32_t rec_slots(const Dims &d) {
    return (uint32_t)d.V * (uint32_t)d.nblk * (uint32_t)kCell;
}

// Threads (= pixels) of a tile block.
__device__ __host__ __forceinline__ uint32_t tile_threads(const Dims &d) {
    return d.tile_threads ? d.tile_threads : (uint32_t)kTilePix;
}

// log2 of the tile width (the compositors are compiled per tile width).
__device__ __host__ __forceinline__ uint32_t tile_lw(const Dims &d) { return d.tile_lw ? d.tile_lw : 4u; }

// ------------------------------------------------------------------ host-side launchers

struct ProjectLaunch {
    WsPtrs ws;
    Dims d;
    Settings s;
    GaussPtrs g;
    int dtype;
    const double *poses;
};

// Also zeroes zero_bytes (a multiple of 4) at `zero` in the same launch.
cudaError_t launch_upload_views(const ViewInfo *host_views, int V, ViewInfo *dev, void *zero, size_t zero_bytes,
                                cudaStream_t st);
cudaError_t launch_project(const ProjectLaunch &L, cudaStream_t st);
cudaError_t launch_scan_tiles(const WsPtrs &ws, const Dims &d, cudaStream_t st);
cudaError_t launch_emit(const WsPtrs &ws, const Dims &d, cudaStream_t st);

struct ForwardLaunch {
    WsPtrs ws;
    Dims d;
    Settings s;
    float *rgb, *depth, *sil;  // outputs (nullable)
    const float *t_rgb, *t_depth, *t_prior;  // targets (t_rgb == nullptr -> no loss)
};
cudaError_t launch_forward(const ForwardLaunch &L, cudaStream_t st);

struct BackwardLaunch {
    WsPtrs ws;
    Dims d;
    Settings s;
    const float *up_rgb, *up_depth, *up_sil;  // upstream planes (P each, rgb 3P)
    bool pose_only;                            // skip opacity / colour gradients
};
cudaError_t launch_backward(const BackwardLaunch &L, cudaStream_t st);

// Forward with the fused loss and the pose-only reverse walk of each tile in one kernel
// (the tracking step under GS_SCHED_FUSED); needs targets and fwd_batch == bwd_batch.
struct TrackTileLaunch {
    WsPtrs ws;
    Dims d;
    Settings s;
    const float *t_rgb, *t_depth, *t_prior;
};
cudaError_t launch_track_tile(const TrackTileLaunch &L, cudaStream_t st);

// The device-wide LSD radix sort of the (tile, depth) keys k_emit writes under
// GS_SCHED_RADIX (radix_sort.cu); its result replaces the compositors' per-tile sort.
struct RadixLaunch {
    WsPtrs ws;
    Dims d;
};
uint32_t radix_blocks(uint32_t pair_cap);
int radix_passes(uint32_t tiles);
cudaError_t launch_radix_sort(const RadixLaunch &L, cudaStream_t st);

struct BprojLaunch {
    WsPtrs ws;
    Dims d;
    Settings s;
    GaussPtrs g;
    int dtype;
    bool want_pose;           // write the per-cell pose partials
    gs_gaussians_grad grads;  // parameter gradients (each nullable)
};
cudaError_t launch_bproject(const BprojLaunch &L, cudaStream_t st);

// Per-view reductions in a fixed order: loss from the tile partials, pose gradient from
// the cell partials, and (tracking) the decoupled Adam step.
struct FinalizeLaunch {
    WsPtrs ws;
    Dims d;
    Settings s;
    double *loss_out;   // n_views, or nullptr
    double *pose_grad;  // n_views x 6, or nullptr
    double *poses;      // updated in place by the Adam step, or nullptr
    double *adam;       // n_views x 16 (with poses)
    double *host_result;  // page-locked host memory (device address), n_views x 8: the updated
                          // pose and the loss, written at the end; or nullptr
    bool pose;          // reduce the pose partials
};
cudaError_t launch_finalize(const FinalizeLaunch &L, cudaStream_t st);

}  // namespace gsk
