// gs_abi.cu -- the C ABI declared in include/gs.h: context, workspace layout, launch
// sequencing and the CUDA-graph tracking loop.  No device memory is allocated here:
// every device buffer, the workspace included, belongs to the caller.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gs_internal.cuh"

using namespace gsk;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Tile shapes a schedule may use (one thread per pixel, 8 x 4 warp patches).
bool valid_tile(int32_t w, int32_t h) {
    const bool wok = w == 8 || w == 16 || w == 32, hok = h == 4 || h == 8 || h == 16 || h == 32;
    return wok && hok && w * h >= 64 && w * h <= kTilePix;
}

int ilog2(int32_t v) {
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return l;
}

// Most sub-buckets a problem of T tiles uses: T x sub-buckets stays within 2^22 counters.
uint32_t max_sub(uint64_t T) {
    uint32_t s = kSubMax;
    while (s > 1 && T * s > (1ull << 22)) s >>= 1;
    return s;
}

struct Layout {
    size_t err, hdr, tile_cnt, zero_end;
    size_t views, view_rt, cell_cnt, tile_start, cursor, tile_order, big, big_listed, rec, rec_grad, keys, sorted, t_final, n_last,
        upstream, tile_loss, pose_part, rkeys, rvals, rhist, rtotal, scan_part, total;
};

struct Problem {
    Dims d{};
    std::vector<ViewInfo> views;
    Layout lay{};
};

struct GraphKey {
    const void *ws = nullptr;
    size_t ws_bytes = 0;
    const void *ptrs[16] = {};
    int64_t n = 0;
    int dtype = 0;
    int iters = 0;
    std::vector<ViewInfo> views;
    uint32_t pair_cap = 0;
    uint32_t prof_mask = 0;
    uint32_t sched[4] = {};  // sub-buckets, forward and backward batch depths, flags
    bool operator==(const GraphKey &o) const {
        if (ws != o.ws || ws_bytes != o.ws_bytes || n != o.n || dtype != o.dtype || iters != o.iters ||
            pair_cap != o.pair_cap || prof_mask != o.prof_mask || sched[0] != o.sched[0] ||
            sched[1] != o.sched[1] || sched[2] != o.sched[2] || sched[3] != o.sched[3] ||
            views.size() != o.views.size())
            return false;
        for (int k = 0; k < 16; ++k)
            if (ptrs[k] != o.ptrs[k]) return false;
        return views.empty() || std::memcmp(views.data(), o.views.data(), views.size() * sizeof(ViewInfo)) == 0;
    }
};

}  // namespace

struct gs_ctx {
    gs_config cfg{};
    Settings s{};
    gs_schedule sched{gsk::kTile, gsk::kTile, gsk::kSubMax, gsk::kBatch, gsk::kBatch, 0};
    std::string err;
    // state bound by the last gs_project
    bool bound = false;
    Problem prob;
    WsPtrs ws{};
    void *ws_base = nullptr;
    GaussPtrs g{};
    int dtype = 0;
    const double *poses = nullptr;
    bool have_loss = false;
    bool grads_used = false;  // the record accumulators were consumed by a gs_backward
    // tracking graph
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    GraphKey graph_key;
    // profiling markers: a named event ends that kernel, the event before it starts it;
    // prof_mask selects kernels (bit k: kKernelNames[k]); adjacent: the last recorded
    // event directly precedes the next launch, so it can serve as that kernel's start
    uint32_t prof_mask = 0;
    bool adjacent = false;
    std::vector<cudaEvent_t> events;
    std::vector<const char *> names;
    size_t n_marks = 0;
    std::vector<const char *> graph_names;  // markers baked into the tracking graph
    // markers inside a captured graph sit on a side branch (mark_stream, forked from the
    // launch stream at each marker and joined at the end of the capture), so no kernel of
    // the main chain waits for an event node
    cudaStream_t mark_stream = nullptr;
    cudaEvent_t fork_ev = nullptr;
    bool side_open = false;
    // the targets' upload of gs_track_step_upload: a branch forked before the first
    // projection and joined before the first compositor
    cudaStream_t up_stream = nullptr;
    cudaEvent_t up_fork = nullptr, up_join = nullptr;
};

namespace {

gs_status fail(gs_ctx *ctx, gs_status st, const char *msg) {
    if (ctx) ctx->err = msg;
    return st;
}

gs_status cuda_fail(gs_ctx *ctx, cudaError_t e, const char *where) {
    if (ctx) ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
    return GS_ERR_CUDA;
}

const char *const kKernelNames[] = {"k_project", "k_scan_tiles", "k_emit", "k_forward",
                                    "k_backward", "k_bproject", "k_finalize", "k_track_tile", "k_radix_sort"};
constexpr uint32_t kAllKernels = (1u << (sizeof(kKernelNames) / sizeof(kKernelNames[0]))) - 1u;

bool selected(const gs_ctx *ctx, const char *name) {
    for (size_t k = 0; k < sizeof(kKernelNames) / sizeof(kKernelNames[0]); ++k)
        if (std::strcmp(kKernelNames[k], name) == 0) return (ctx->prof_mask >> k) & 1u;
    return false;
}

cudaError_t record_mark(gs_ctx *ctx, cudaStream_t st, const char *name) {
    if (ctx->n_marks == ctx->events.size()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        ctx->events.push_back(ev);
        ctx->names.push_back(nullptr);
    }
    const size_t k = ctx->n_marks++;
    ctx->names[k] = name;
    ctx->adjacent = true;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusNone) return cudaEventRecord(ctx->events[k], st);
    // captured: an event-record node on the side branch, after everything enqueued so far
    if (!ctx->mark_stream) {
        if ((e = cudaStreamCreateWithFlags(&ctx->mark_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(ctx->fork_ev, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ctx->mark_stream, ctx->fork_ev, 0)) != cudaSuccess) return e;
    ctx->side_open = true;
    return cudaEventRecordWithFlags(ctx->events[k], ctx->mark_stream, cudaEventRecordExternal);
}

// Join the markers' side branch back into the captured stream `st` (a capture must end
// with every forked stream joined); a no-op when no marker was captured.
cudaError_t join_marks(gs_ctx *ctx, cudaStream_t st) {
    if (!ctx->side_open) return cudaSuccess;
    ctx->side_open = false;
    cudaError_t e = cudaEventRecord(ctx->fork_ev, ctx->mark_stream);
    return e != cudaSuccess ? e : cudaStreamWaitEvent(st, ctx->fork_ev, 0);
}

// Profiling marker before the launch of kernel `name` (only when it is selected and the
// last marker does not already sit right before it).
cudaError_t mark_begin(gs_ctx *ctx, cudaStream_t st, const char *name) {
    if (!ctx->prof_mask || ctx->adjacent || !selected(ctx, name)) return cudaSuccess;
    return record_mark(ctx, st, nullptr);
}

// Profiling marker after the launch of kernel `name`.
cudaError_t mark(gs_ctx *ctx, cudaStream_t st, const char *name) {
    if (!ctx->prof_mask) return cudaSuccess;
    if (!selected(ctx, name)) {
        ctx->adjacent = false;
        return cudaSuccess;
    }
    return record_mark(ctx, st, name);
}

void reset_marks(gs_ctx *ctx) {
    ctx->n_marks = 0;
    ctx->adjacent = false;
}

Settings settings_of(const gs_config &c) {
    Settings s;
    s.alpha_min = c.alpha_min;
    s.alpha_max = c.alpha_max;
    s.t_min = c.t_min;
    s.dilation = c.dilation;
    s.z_near = c.z_near;
    s.sil_thresh = c.sil_thresh;
    s.log2_alpha_min = c.alpha_min > 0.f ? (float)std::log2((double)c.alpha_min) : -INFINITY;
    s.w_rgb = c.w_rgb;
    s.w_depth = c.w_depth;
    s.w_vis = c.w_vis;
    s.w_prior = c.w_prior;
    s.lr_rot = c.lr_rot;
    s.lr_trans = c.lr_trans;
    s.beta1 = c.beta1;
    s.beta2 = c.beta2;
    s.eps = c.eps;
    return s;
}

gs_status build_problem(gs_ctx *ctx, const gs_problem *p, Problem &out) {
    if (!p || !p->cameras) return fail(ctx, GS_ERR_INVALID_ARG, "problem or cameras is NULL");
    if (p->n_views < 1) return fail(ctx, GS_ERR_INVALID_ARG, "n_views must be >= 1");
    if (p->n_gaussians < 0) return fail(ctx, GS_ERR_INVALID_ARG, "n_gaussians must be >= 0");
    const uint64_t nv = (uint64_t)p->n_gaussians * (uint64_t)p->n_views;
    if (nv >= (1ull << 32)) return fail(ctx, GS_ERR_INVALID_ARG, "n_gaussians * n_views must be < 2^32");
    if (p->pair_capacity < 1 || p->pair_capacity >= (int64_t)(1ll << 32))
        return fail(ctx, GS_ERR_INVALID_ARG, "pair_capacity must be in [1, 2^32)");
    if (p->record_capacity != 0) return fail(ctx, GS_ERR_INVALID_ARG, "record_capacity is reserved and must be 0");
    Dims d{};
    d.n = p->n_gaussians;
    d.V = p->n_views;
    d.nblk = (int32_t)((p->n_gaussians + kBlock - 1) / kBlock);
    if (d.nblk == 0) d.nblk = 1;
    if ((uint64_t)d.nblk * kCell * (uint64_t)p->n_views >= (1ull << 32))
        return fail(ctx, GS_ERR_INVALID_ARG, "n_gaussians * n_views too large for 32-bit record slots");
    d.pair_cap = (uint32_t)p->pair_capacity;
    out.views.resize(p->n_views);
    const int32_t tw = ctx->sched.tile_w, th = ctx->sched.tile_h;
    uint64_t T = 0, P = 0;
    for (int v = 0; v < p->n_views; ++v) {
        const gs_camera &c = p->cameras[v];
        if (c.width < 1 || c.height < 1 || !(c.fx > 0) || !(c.fy > 0))
            return fail(ctx, GS_ERR_INVALID_ARG, "camera with non-positive size or focal length");
        ViewInfo vi{};
        vi.fx = (float)c.fx;
        vi.fy = (float)c.fy;
        vi.cx = (float)c.cx;
        vi.cy = (float)c.cy;
        vi.width = c.width;
        vi.height = c.height;
        vi.tiles_x = (c.width + tw - 1) / tw;
        vi.tiles_y = (c.height + th - 1) / th;
        vi.tile_lw = ilog2(tw);
        vi.tile_lh = ilog2(th);
        vi.tile_base = (uint32_t)T;
        vi.pix_base = (uint32_t)P;
        vi.tan_lim_x = jacobian_tangent_limit(ctx->cfg.jac_clip, c.width, c.fx);
        vi.tan_lim_y = jacobian_tangent_limit(ctx->cfg.jac_clip, c.height, c.fy);
        T += (uint64_t)vi.tiles_x * vi.tiles_y;
        P += (uint64_t)c.width * c.height;
        if (T >= (1ull << 27) || 5 * P >= (1ull << 32))
            return fail(ctx, GS_ERR_INVALID_ARG, "too many pixels or tiles in one call");
        out.views[v] = vi;
    }
    // the layout has room for the tiles and tile counters of every allowed tile shape, so
    // the workspace size does not depend on the schedule
    uint64_t lay_tiles = 0, lay_cnt = 0;
    for (int32_t w = 8; w <= 32; w *= 2)
        for (int32_t h = 4; h <= 32; h *= 2) {
            if (!valid_tile(w, h)) continue;
            uint64_t t = 0;
            for (int v = 0; v < p->n_views; ++v)
                t += (uint64_t)((p->cameras[v].width + w - 1) / w) * (uint64_t)((p->cameras[v].height + h - 1) / h);
            lay_tiles = std::max(lay_tiles, t);
            lay_cnt = std::max(lay_cnt, t * max_sub(t));
        }
    if (lay_tiles >= (1ull << 27)) return fail(ctx, GS_ERR_INVALID_ARG, "too many pixels or tiles in one call");
    d.T = (uint32_t)T;
    d.P = (uint32_t)P;
    d.S = std::min(max_sub(T), (uint32_t)ctx->sched.sub_buckets);
    d.fwd_batch = (uint32_t)ctx->sched.fwd_batch;
    d.bwd_batch = (uint32_t)ctx->sched.bwd_batch;
    d.flags = (uint32_t)ctx->sched.flags;
    d.tile_threads = (uint32_t)(tw * th);
    d.tile_lw = (uint32_t)ilog2(tw);
    out.d = d;
    Layout &L = out.lay;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    L.err = take(sizeof(uint32_t));
    // zeroed before every projection: [hdr, zero_end)
    L.hdr = take(sizeof(DevHeader));
    L.tile_cnt = take(sizeof(uint32_t) * ((size_t)lay_cnt + 1));
    L.zero_end = o;
    const size_t cells = (size_t)d.V * d.nblk;
    L.views = take(sizeof(ViewInfo) * d.V);
    L.view_rt = take(sizeof(float) * 12 * d.V);
    L.cell_cnt = take(sizeof(uint32_t) * cells);
    L.tile_start = take(sizeof(uint32_t) * ((size_t)lay_cnt + 1));
    L.cursor = take(sizeof(uint32_t) * ((size_t)lay_cnt + 1));
    L.tile_order = take(sizeof(uint32_t) * (size_t)lay_tiles);
    L.big = take(sizeof(uint32_t) * kBigListCap);
    L.big_listed = take(cells * kCell);
    L.rec = take(sizeof(Rec) * cells * kCell);
    L.rec_grad = take(sizeof(RecGrad) * cells * kCell);
    L.keys = take(sizeof(unsigned long long) * (size_t)d.pair_cap);
    L.sorted = take(sizeof(uint32_t) * (size_t)d.pair_cap);
    L.t_final = take(sizeof(float) * (size_t)d.P);
    L.n_last = take(sizeof(uint32_t) * (size_t)d.P);
    L.upstream = take(sizeof(float) * 5 * (size_t)d.P);
    L.tile_loss = take(sizeof(float2) * (size_t)lay_tiles);
    L.pose_part = take(sizeof(float2) * 6 * cells);
    // the radix sort's second key / value buffers and digit counts (GS_SCHED_RADIX)
    L.rkeys = take(sizeof(unsigned long long) * (size_t)d.pair_cap);
    L.rvals = take(sizeof(uint32_t) * (size_t)d.pair_cap);
    L.rhist = take(sizeof(uint32_t) * 256 * (size_t)radix_blocks(d.pair_cap));
    L.rtotal = take(sizeof(uint32_t) * 256);
    L.scan_part = take(sizeof(uint32_t) * (3 + kMBuckets) * (size_t)scan_blocks(lay_cnt));
    L.total = o;
    return GS_OK;
}

WsPtrs ws_ptrs(void *base, const Layout &L) {
    char *b = static_cast<char *>(base);
    WsPtrs w;
    w.err = reinterpret_cast<uint32_t *>(b + L.err);
    w.hdr = reinterpret_cast<DevHeader *>(b + L.hdr);
    w.tile_cnt = reinterpret_cast<uint32_t *>(b + L.tile_cnt);
    w.views = reinterpret_cast<ViewInfo *>(b + L.views);
    w.view_rt = reinterpret_cast<float *>(b + L.view_rt);
    w.cell_cnt = reinterpret_cast<uint32_t *>(b + L.cell_cnt);
    w.tile_start = reinterpret_cast<uint32_t *>(b + L.tile_start);
    w.cursor = reinterpret_cast<uint32_t *>(b + L.cursor);
    w.tile_order = reinterpret_cast<uint32_t *>(b + L.tile_order);
    w.big = reinterpret_cast<uint32_t *>(b + L.big);
    w.big_listed = reinterpret_cast<uint8_t *>(b + L.big_listed);
    w.rec = reinterpret_cast<Rec *>(b + L.rec);
    w.rec_grad = reinterpret_cast<RecGrad *>(b + L.rec_grad);
    w.keys = reinterpret_cast<unsigned long long *>(b + L.keys);
    w.sorted = reinterpret_cast<uint32_t *>(b + L.sorted);
    w.t_final = reinterpret_cast<float *>(b + L.t_final);
    w.n_last = reinterpret_cast<uint32_t *>(b + L.n_last);
    w.upstream = reinterpret_cast<float *>(b + L.upstream);
    w.tile_loss = reinterpret_cast<float2 *>(b + L.tile_loss);
    w.pose_part = reinterpret_cast<float2 *>(b + L.pose_part);
    w.rkeys = reinterpret_cast<unsigned long long *>(b + L.rkeys);
    w.rvals = reinterpret_cast<uint32_t *>(b + L.rvals);
    w.rhist = reinterpret_cast<uint32_t *>(b + L.rhist);
    w.rtotal = reinterpret_cast<uint32_t *>(b + L.rtotal);
    w.scan_part = reinterpret_cast<uint32_t *>(b + L.scan_part);
    return w;
}

gs_status check_gaussians(gs_ctx *ctx, const gs_gaussians *g, const Problem &pr) {
    if (!g) return fail(ctx, GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n != pr.d.n) return fail(ctx, GS_ERR_INVALID_ARG, "gaussians.n differs from problem.n_gaussians");
    if (g->dtype_attr != GS_F32 && g->dtype_attr != GS_BF16 && g->dtype_attr != GS_F16)
        return fail(ctx, GS_ERR_INVALID_ARG, "unknown dtype_attr");
    if (g->n > 0 && (!g->means || !g->log_scales || !g->opacity_logits || !g->rgb))
        return fail(ctx, GS_ERR_INVALID_ARG, "a Gaussian attribute pointer is NULL");
    return GS_OK;
}

// Write the view table into the workspace (kernel arguments carry it, so the upload is
// stream-ordered and safe to capture; it is redone on every call because the library
// cannot tell whether the caller reused the workspace memory for something else).  The
// same launch zeroes the latched error flags, the header and the tile counters; later
// iterations of a call find the counters zeroed by the scan that consumed them and the
// header by the projection.
cudaError_t upload_views(const Problem &pr, const WsPtrs &w, void *ws, cudaStream_t st) {
    return launch_upload_views(pr.views.data(), (int)pr.views.size(), w.views, static_cast<char *>(ws) + pr.lay.err,
                               pr.lay.zero_end - pr.lay.err, st);
}

// One projection pass: project, scan the tile counts, emit keys.
cudaError_t enqueue_project(gs_ctx *ctx, const Problem &pr, const WsPtrs &w, const GaussPtrs &g, int dtype,
                            const double *poses, cudaStream_t st) {
    cudaError_t e;
    ProjectLaunch P;
    P.ws = w;
    P.d = pr.d;
    P.s = ctx->s;
    P.g = g;
    P.dtype = dtype;
    P.poses = poses;
    if ((e = mark_begin(ctx, st, "k_project")) != cudaSuccess) return e;
    if ((e = launch_project(P, st)) != cudaSuccess) return e;
    if ((e = mark(ctx, st, "k_project")) != cudaSuccess) return e;
    if ((e = mark_begin(ctx, st, "k_scan_tiles")) != cudaSuccess) return e;
    if ((e = launch_scan_tiles(w, pr.d, st)) != cudaSuccess) return e;
    if ((e = mark(ctx, st, "k_scan_tiles")) != cudaSuccess) return e;
    if ((e = mark_begin(ctx, st, "k_emit")) != cudaSuccess) return e;
    if ((e = launch_emit(w, pr.d, st)) != cudaSuccess) return e;
    if ((e = mark(ctx, st, "k_emit")) != cudaSuccess) return e;
    if (!(pr.d.flags & GS_SCHED_RADIX)) return cudaSuccess;
    RadixLaunch X;
    X.ws = w;
    X.d = pr.d;
    if ((e = mark_begin(ctx, st, "k_radix_sort")) != cudaSuccess) return e;
    if ((e = launch_radix_sort(X, st)) != cudaSuccess) return e;
    return mark(ctx, st, "k_radix_sort");
}

cudaError_t enqueue_forward(gs_ctx *ctx, const Problem &pr, const WsPtrs &w, const gs_targets *t, float *rgb,
                            float *depth, float *sil, cudaStream_t st) {
    cudaError_t e;
    ForwardLaunch F;
    F.ws = w;
    F.d = pr.d;
    F.s = ctx->s;
    F.rgb = rgb;
    F.depth = depth;
    F.sil = sil;
    F.t_rgb = t ? t->rgb : nullptr;
    F.t_depth = t ? t->depth : nullptr;
    F.t_prior = t ? t->depth_prior : nullptr;
    if ((e = mark_begin(ctx, st, "k_forward")) != cudaSuccess) return e;
    if ((e = launch_forward(F, st)) != cudaSuccess) return e;
    return mark(ctx, st, "k_forward");
}

// Both compositors of a pose-only tracking iteration with the fused loss: k_forward then
// k_backward, or k_track_tile when the schedule fuses them (GS_SCHED_FUSED).
cudaError_t enqueue_compositing(gs_ctx *ctx, const Problem &pr, const WsPtrs &w, const gs_targets *t,
                                cudaStream_t st) {
    cudaError_t r;
    if (pr.d.flags & GS_SCHED_FUSED) {
        TrackTileLaunch K;
        K.ws = w;
        K.d = pr.d;
        K.s = ctx->s;
        K.t_rgb = t->rgb;
        K.t_depth = t->depth;
        K.t_prior = t->depth_prior;
        if ((r = mark_begin(ctx, st, "k_track_tile")) != cudaSuccess) return r;
        if ((r = launch_track_tile(K, st)) != cudaSuccess) return r;
        return mark(ctx, st, "k_track_tile");
    }
    if ((r = enqueue_forward(ctx, pr, w, t, nullptr, nullptr, nullptr, st)) != cudaSuccess) return r;
    BackwardLaunch B;
    B.ws = w;
    B.d = pr.d;
    B.s = ctx->s;
    B.up_rgb = w.upstream;
    B.up_depth = w.upstream + 3u * pr.d.P;
    B.up_sil = w.upstream + 4u * pr.d.P;
    B.pose_only = true;
    if ((r = mark_begin(ctx, st, "k_backward")) != cudaSuccess) return r;
    if ((r = launch_backward(B, st)) != cudaSuccess) return r;
    return mark(ctx, st, "k_backward");
}

bool valid_batch(int32_t b) { return b == 64 || b == 128 || b == 256; }

bool valid_schedule(const gs_schedule &sc) {
    const int32_t sb = sc.sub_buckets, px = sc.tile_w * sc.tile_h;
    return valid_tile(sc.tile_w, sc.tile_h) && (sb == 1 || sb == 2 || sb == 4) && valid_batch(sc.fwd_batch) &&
           valid_batch(sc.bwd_batch) && sc.fwd_batch <= px && sc.bwd_batch <= px &&
           (sc.flags & ~(GS_SCHED_FUSED | GS_SCHED_RADIX)) == 0 &&
           (!(sc.flags & GS_SCHED_FUSED) || sc.fwd_batch == sc.bwd_batch);
}

// Device time of one pass of `enqueue`, averaged over `reps` passes after one untimed
// pass, with two events on the stream.
template <class F>
cudaError_t time_passes(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps, F &&enqueue, float &ms) {
    cudaError_t e = enqueue();
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
    for (int r = 0; r < reps; ++r)
        if ((e = enqueue()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
    float t = 0.f;
    if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) return e;
    ms = t / (float)reps;
    return cudaSuccess;
}

// The fastest candidate, unless it is within 1 % of the first (the default), which then
// stays: timing noise does not move the schedule.
int pick(const float *ms, int n) {
    int b = 0;
    for (int k = 1; k < n; ++k)
        if (ms[k] < ms[b]) b = k;
    return ms[b] < 0.99f * ms[0] ? b : 0;
}

}  // namespace

extern "C" {

void gs_default_config(gs_config *c) {
    if (!c) return;
    c->tile_w = kTile;
    c->tile_h = kTile;  // the default schedule's tile
    c->alpha_min = 1.0f / 255.0f;
    c->alpha_max = 0.99f;
    c->t_min = 1e-4f;
    c->dilation = 0.0f;
    c->z_near = 0.2f;
    c->jac_clip = 1.3f;
    c->sil_thresh = 0.99f;
    c->w_rgb = 0.5f;
    c->w_depth = 1.0f;
    c->w_vis = 0.1f;
    c->w_prior = 0.5f;
    c->lr_rot = 2e-3;
    c->lr_trans = 2e-3;
    c->beta1 = 0.9;
    c->beta2 = 0.999;
    c->eps = 1e-8;
}

const char *gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "GS_OK";
        case GS_ERR_INVALID_ARG: return "GS_ERR_INVALID_ARG";
        case GS_ERR_CUDA: return "GS_ERR_CUDA";
        case GS_ERR_OOM: return "GS_ERR_OOM";
        case GS_ERR_WORKSPACE: return "GS_ERR_WORKSPACE";
        case GS_ERR_CAPACITY: return "GS_ERR_CAPACITY";
        case GS_ERR_TIMEOUT: return "GS_ERR_TIMEOUT";
        case GS_ERR_UNSUPPORTED: return "GS_ERR_UNSUPPORTED";
        case GS_ERR_STATE: return "GS_ERR_STATE";
    }
    return "GS_ERR_UNKNOWN";
}

gs_status gs_create(gs_ctx **out, const gs_config *cfg) {
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    gs_config c;
    gs_default_config(&c);
    if (cfg) c = *cfg;
    if (!valid_tile(c.tile_w, c.tile_h)) return GS_ERR_UNSUPPORTED;
    if (!(c.alpha_min >= 0.f) || !(c.alpha_max > c.alpha_min) || !(c.alpha_max <= 1.f) || !(c.t_min >= 0.f) ||
        !(c.t_min < 1.f) || !(c.dilation >= 0.f) || !(c.z_near > 0.f) || !(c.jac_clip >= 0.f) || !(c.lr_rot >= 0) || !(c.lr_trans >= 0) ||
        !(c.beta1 >= 0 && c.beta1 < 1) || !(c.beta2 >= 0 && c.beta2 < 1) || !(c.eps > 0))
        return GS_ERR_INVALID_ARG;
    gs_ctx *ctx = new (std::nothrow) gs_ctx();
    if (!ctx) return GS_ERR_OOM;
    ctx->cfg = c;
    ctx->s = settings_of(c);
    ctx->sched.tile_w = c.tile_w;
    ctx->sched.tile_h = c.tile_h;
    ctx->sched.fwd_batch = ctx->sched.bwd_batch = std::min(kBatch, c.tile_w * c.tile_h);
    *out = ctx;
    return GS_OK;
}

gs_status gs_destroy(gs_ctx *ctx) {
    if (!ctx) return GS_OK;
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->mark_stream) cudaStreamDestroy(ctx->mark_stream);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
    if (ctx->up_fork) cudaEventDestroy(ctx->up_fork);
    if (ctx->up_join) cudaEventDestroy(ctx->up_join);
    for (cudaEvent_t ev : ctx->events) cudaEventDestroy(ev);
    delete ctx;
    return GS_OK;
}

const char *gs_last_error(const gs_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

gs_status gs_workspace_size(const gs_ctx *ctx, const gs_problem *prob, size_t *bytes) {
    gs_ctx *c = const_cast<gs_ctx *>(ctx);
    if (!ctx || !bytes) return fail(c, GS_ERR_INVALID_ARG, "NULL context or output");
    Problem pr;
    gs_status st = build_problem(c, prob, pr);
    if (st != GS_OK) return st;
    *bytes = pr.lay.total;
    return GS_OK;
}

gs_status gs_project(gs_ctx *ctx, const gs_problem *prob, const gs_gaussians *g, const double *poses, void *ws,
                     size_t ws_bytes, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    Problem pr;
    gs_status st = build_problem(ctx, prob, pr);
    if (st != GS_OK) return st;
    if ((st = check_gaussians(ctx, g, pr)) != GS_OK) return st;
    if (!poses) return fail(ctx, GS_ERR_INVALID_ARG, "poses is NULL");
    if (!ws || ws_bytes < pr.lay.total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
        return fail(ctx, GS_ERR_WORKSPACE, "workspace NULL, smaller than gs_workspace_size or not 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const WsPtrs w = ws_ptrs(ws, pr.lay);
    GaussPtrs gp{g->means, g->quats, g->log_scales, g->opacity_logits, g->rgb};
    reset_marks(ctx);
    cudaError_t e = upload_views(pr, w, ws, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "view upload");
    e = enqueue_project(ctx, pr, w, gp, g->dtype_attr, poses, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "projection");
    ctx->bound = true;
    ctx->prob = std::move(pr);
    ctx->ws = w;
    ctx->ws_base = ws;
    ctx->g = gp;
    ctx->dtype = g->dtype_attr;
    ctx->poses = poses;
    ctx->have_loss = false;
    ctx->grads_used = false;
    return GS_OK;
}

gs_status gs_forward(gs_ctx *ctx, const gs_targets *targets, float *rgb, float *depth, float *sil, double *loss,
                     void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->bound) return fail(ctx, GS_ERR_STATE, "gs_forward before gs_project");
    if (targets && (!targets->rgb || !targets->depth))
        return fail(ctx, GS_ERR_INVALID_ARG, "targets need rgb and depth");
    if (loss && !targets) return fail(ctx, GS_ERR_INVALID_ARG, "loss requested without targets");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = enqueue_forward(ctx, ctx->prob, ctx->ws, targets, rgb, depth, sil, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "forward");
    if (loss) {
        FinalizeLaunch F{};
        F.ws = ctx->ws;
        F.d = ctx->prob.d;
        F.s = ctx->s;
        F.loss_out = loss;
        e = mark_begin(ctx, s, "k_finalize");
        if (e == cudaSuccess) e = launch_finalize(F, s);
        if (e == cudaSuccess) e = mark(ctx, s, "k_finalize");
        if (e != cudaSuccess) return cuda_fail(ctx, e, "loss reduction");
    }
    ctx->have_loss = targets != nullptr;
    return GS_OK;
}

gs_status gs_backward(gs_ctx *ctx, const float *d_rgb, const float *d_depth, const float *d_sil,
                      gs_gaussians_grad *grads, double *pose_grad, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->bound) return fail(ctx, GS_ERR_STATE, "gs_backward before gs_project");
    const int given = (d_rgb != nullptr) + (d_depth != nullptr) + (d_sil != nullptr);
    if (given != 0 && given != 3) return fail(ctx, GS_ERR_INVALID_ARG, "give all three upstream maps or none");
    if (given == 0 && !ctx->have_loss)
        return fail(ctx, GS_ERR_STATE, "no upstream maps and no fused loss from gs_forward");
    if (ctx->grads_used) return fail(ctx, GS_ERR_STATE, "one gs_backward per gs_project");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Problem &pr = ctx->prob;
    BackwardLaunch B;
    B.ws = ctx->ws;
    B.d = pr.d;
    B.s = ctx->s;
    const uint32_t P = pr.d.P;
    B.up_rgb = given ? d_rgb : ctx->ws.upstream;
    B.up_depth = given ? d_depth : ctx->ws.upstream + 3u * P;
    B.up_sil = given ? d_sil : ctx->ws.upstream + 4u * P;
    gs_gaussians_grad none{};
    const gs_gaussians_grad &G = grads ? *grads : none;
    const bool params = G.means || G.quats || G.log_scales || G.opacity_logits || G.rgb;
    B.pose_only = !(G.opacity_logits || G.rgb);
    cudaError_t e = mark_begin(ctx, s, "k_backward");
    if (e == cudaSuccess) e = launch_backward(B, s);
    if (e == cudaSuccess) e = mark(ctx, s, "k_backward");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "backward");
    if (!params && !pose_grad) {
        ctx->grads_used = true;
        return GS_OK;
    }
    BprojLaunch J;
    J.ws = ctx->ws;
    J.d = pr.d;
    J.s = ctx->s;
    J.g = ctx->g;
    J.dtype = ctx->dtype;
    J.want_pose = pose_grad != nullptr;
    J.grads = G;
    e = mark_begin(ctx, s, "k_bproject");
    if (e == cudaSuccess) e = launch_bproject(J, s);
    if (e == cudaSuccess) e = mark(ctx, s, "k_bproject");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "backward projection");
    if (pose_grad) {
        FinalizeLaunch F{};
        F.ws = ctx->ws;
        F.d = pr.d;
        F.s = ctx->s;
        F.pose_grad = pose_grad;
        F.pose = true;
        e = mark_begin(ctx, s, "k_finalize");
        if (e == cudaSuccess) e = launch_finalize(F, s);
        if (e == cudaSuccess) e = mark(ctx, s, "k_finalize");
        if (e != cudaSuccess) return cuda_fail(ctx, e, "pose reduction");
    }
    ctx->grads_used = true;
    return GS_OK;
}

namespace {

bool pinned_host(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error an unregistered pointer may leave
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// The upload branch of gs_track_step_upload: src -> targets on ctx->up_stream after
// everything enqueued on q so far (the colour planes, depth and prior in three copies, one
// after the other: several copies at once were slower here, 51 against 31 us for the
// 6.1 MB frame); join_upload makes q wait for it.
cudaError_t fork_upload(gs_ctx *ctx, const gs_targets *targets, const gs_host_targets *src, uint32_t P,
                        cudaStream_t q) {
    cudaError_t e = cudaSuccess;
    if (!ctx->up_stream) {
        if ((e = cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&ctx->up_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&ctx->up_join, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(ctx->up_fork, q)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ctx->up_stream, ctx->up_fork, 0)) != cudaSuccess) return e;
    const size_t plane = sizeof(float) * (size_t)P;
    // the targets' device buffers are the destination of this call's upload
    if ((e = cudaMemcpyAsync(const_cast<float *>(targets->rgb), src->rgb, 3 * plane, cudaMemcpyHostToDevice,
                             ctx->up_stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(const_cast<float *>(targets->depth), src->depth, plane, cudaMemcpyHostToDevice,
                             ctx->up_stream)) != cudaSuccess)
        return e;
    if (src->depth_prior &&
        (e = cudaMemcpyAsync(const_cast<float *>(targets->depth_prior), src->depth_prior, plane,
                             cudaMemcpyHostToDevice, ctx->up_stream)) != cudaSuccess)
        return e;
    return cudaEventRecord(ctx->up_join, ctx->up_stream);
}

cudaError_t join_upload(gs_ctx *ctx, cudaStream_t q) { return cudaStreamWaitEvent(q, ctx->up_join, 0); }

gs_status track_step(gs_ctx *ctx, const gs_problem *prob, const gs_gaussians *g, const gs_targets *targets,
                     const gs_host_targets *src, double *poses, double *adam_state, double *loss_hist, int32_t iters,
                     void *ws, size_t ws_bytes, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (iters < 1) return fail(ctx, GS_ERR_INVALID_ARG, "iters must be >= 1");
    // without device targets (gs_track_step_upload only) the kernels read the frame in
    // place: src's page-locked arrays through their device addresses
    const bool in_place = src && !targets;
    gs_targets src_dev{};
    if (in_place) {
        if (!src->rgb || !src->depth) return fail(ctx, GS_ERR_INVALID_ARG, "src needs rgb and depth");
        const float *const host[3] = {src->rgb, src->depth, src->depth_prior};
        const float **dev[3] = {&src_dev.rgb, &src_dev.depth, &src_dev.depth_prior};
        for (int k = 0; k < 3; ++k) {
            if (!host[k]) continue;
            void *d = nullptr;
            if (!pinned_host(host[k]) || cudaHostGetDevicePointer(&d, const_cast<float *>(host[k]), 0) != cudaSuccess) {
                cudaGetLastError();
                return fail(ctx, GS_ERR_INVALID_ARG, "src arrays must be page-locked host memory mapped into the device's "
                                                     "address space");
            }
            *dev[k] = static_cast<const float *>(d);
        }
        targets = &src_dev;
    }
    if (!targets || !targets->rgb || !targets->depth) return fail(ctx, GS_ERR_INVALID_ARG, "targets need rgb and depth");
    if (!poses || !adam_state) return fail(ctx, GS_ERR_INVALID_ARG, "poses and adam_state are required");
    if (src) {
        if (!src->rgb || !src->depth || !src->depth_prior != !targets->depth_prior)
            return fail(ctx, GS_ERR_INVALID_ARG, "src needs rgb and depth, and a depth prior exactly when targets has one");
        if (!pinned_host(src->rgb) || !pinned_host(src->depth) || (src->depth_prior && !pinned_host(src->depth_prior)) ||
            (src->result && !pinned_host(src->result)))
            return fail(ctx, GS_ERR_INVALID_ARG, "src arrays must be page-locked host memory");
    }
    double *result_dev = nullptr;  // the device's address of src->result
    if (src && src->result && cudaHostGetDevicePointer(reinterpret_cast<void **>(&result_dev), src->result, 0) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GS_ERR_INVALID_ARG, "src->result is not mapped into the device's address space");
    }
    Problem pr;
    gs_status st = build_problem(ctx, prob, pr);
    if (st != GS_OK) return st;
    if ((st = check_gaussians(ctx, g, pr)) != GS_OK) return st;
    if (!ws || ws_bytes < pr.lay.total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
        return fail(ctx, GS_ERR_WORKSPACE, "workspace NULL, smaller than gs_workspace_size or not 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const WsPtrs w = ws_ptrs(ws, pr.lay);
    GaussPtrs gp{g->means, g->quats, g->log_scales, g->opacity_logits, g->rgb};

    auto enqueue_all = [&](cudaStream_t q) -> cudaError_t {
        // the frame's upload runs beside the view upload and the first projection, scan and
        // emission
        const bool upload = src && !in_place;
        cudaError_t r0 = upload ? fork_upload(ctx, targets, src, pr.d.P, q) : cudaSuccess;
        if (r0 != cudaSuccess) return r0;
        // the view table and the per-call reset, as the graph's first node (its arguments
        // are part of the graph's key); flags latch over all iterations of the call
        if ((r0 = upload_views(pr, w, ws, q)) != cudaSuccess) return r0;
        for (int it = 0; it < iters; ++it) {
            cudaError_t r = cudaSuccess;
            if ((r = enqueue_project(ctx, pr, w, gp, g->dtype_attr, poses, q)) != cudaSuccess) return r;
            if (it == 0 && upload && (r = join_upload(ctx, q)) != cudaSuccess) return r;
            if ((r = enqueue_compositing(ctx, pr, w, targets, q)) != cudaSuccess) return r;
            BprojLaunch J;
            J.ws = w;
            J.d = pr.d;
            J.s = ctx->s;
            J.g = gp;
            J.dtype = g->dtype_attr;
            J.want_pose = true;
            J.grads = gs_gaussians_grad{};
            if ((r = mark_begin(ctx, q, "k_bproject")) != cudaSuccess) return r;
            if ((r = launch_bproject(J, q)) != cudaSuccess) return r;
            if ((r = mark(ctx, q, "k_bproject")) != cudaSuccess) return r;
            FinalizeLaunch F{};
            F.ws = w;
            F.d = pr.d;
            F.s = ctx->s;
            F.loss_out = loss_hist ? loss_hist + (size_t)it * pr.d.V : nullptr;
            F.pose = true;
            F.poses = poses;
            F.adam = adam_state;
            F.host_result = it == iters - 1 ? result_dev : nullptr;
            if ((r = mark_begin(ctx, q, "k_finalize")) != cudaSuccess) return r;
            if ((r = launch_finalize(F, q)) != cudaSuccess) return r;
            if ((r = mark(ctx, q, "k_finalize")) != cudaSuccess) return r;
        }
        return join_marks(ctx, q);
    };

    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream query");
    reset_marks(ctx);
    if (cap != cudaStreamCaptureStatusNone) {
        // the caller is capturing: record the kernels into its graph directly
        e = enqueue_all(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tracking enqueue");
    } else {
        GraphKey key;
        key.ws = ws;
        key.ws_bytes = ws_bytes;
        const void *ptrs[16] = {g->means, g->quats, g->log_scales, g->opacity_logits, g->rgb, targets->rgb,
                                targets->depth, targets->depth_prior, poses, adam_state, loss_hist, nullptr,
                                src ? src->rgb : nullptr, src ? src->depth : nullptr,
                                src ? src->depth_prior : nullptr, src ? src->result : nullptr};
        for (int k = 0; k < 16; ++k) key.ptrs[k] = ptrs[k];
        key.n = g->n;
        key.dtype = g->dtype_attr;
        key.iters = iters;
        key.views = pr.views;
        key.pair_cap = pr.d.pair_cap;
        key.prof_mask = ctx->prof_mask;
        key.sched[0] = pr.d.S;
        key.sched[1] = pr.d.fwd_batch;
        key.sched[2] = pr.d.bwd_batch;
        key.sched[3] = pr.d.flags;
        if (!ctx->graph_exec || !(ctx->graph_key == key)) {
            if (ctx->graph_exec) {
                cudaGraphExecDestroy(ctx->graph_exec);
                ctx->graph_exec = nullptr;
            }
            if (!ctx->cap_stream) {
                e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "capture stream");
            }
            e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "begin capture");
            cudaError_t e_enq = enqueue_all(ctx->cap_stream);
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(ctx->cap_stream, &graph);
            if (e_enq != cudaSuccess) {
                ctx->side_open = false;
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(ctx, e_enq, "tracking capture");
            }
            if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
            e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                ctx->graph_exec = nullptr;
                return cuda_fail(ctx, e, "graph instantiate");
            }
            ctx->graph_key = key;
            ctx->graph_names.assign(ctx->names.begin(), ctx->names.begin() + ctx->n_marks);
        }
        ctx->n_marks = ctx->graph_names.size();
        std::copy(ctx->graph_names.begin(), ctx->graph_names.end(), ctx->names.begin());
        e = cudaGraphLaunch(ctx->graph_exec, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    }
    ctx->bound = true;
    ctx->prob = std::move(pr);
    ctx->ws = w;
    ctx->ws_base = ws;
    ctx->g = gp;
    ctx->dtype = g->dtype_attr;
    ctx->poses = poses;
    ctx->have_loss = true;
    ctx->grads_used = true;
    return GS_OK;
}

}  // namespace

gs_status gs_track_step(gs_ctx *ctx, const gs_problem *prob, const gs_gaussians *g, const gs_targets *targets,
                        double *poses, double *adam_state, double *loss_hist, int32_t iters, void *ws,
                        size_t ws_bytes, void *stream) {
    return track_step(ctx, prob, g, targets, nullptr, poses, adam_state, loss_hist, iters, ws, ws_bytes, stream);
}

gs_status gs_track_step_upload(gs_ctx *ctx, const gs_problem *prob, const gs_gaussians *g, const gs_targets *targets,
                               const gs_host_targets *src, double *poses, double *adam_state, double *loss_hist,
                               int32_t iters, void *ws, size_t ws_bytes, void *stream) {
    if (!src) return ctx ? fail(ctx, GS_ERR_INVALID_ARG, "src is NULL") : GS_ERR_INVALID_ARG;
    return track_step(ctx, prob, g, targets, src, poses, adam_state, loss_hist, iters, ws, ws_bytes, stream);
}

gs_status gs_get_schedule(const gs_ctx *ctx, gs_schedule *out) {
    if (!ctx || !out) return GS_ERR_INVALID_ARG;
    *out = ctx->sched;
    return GS_OK;
}

gs_status gs_set_schedule(gs_ctx *ctx, const gs_schedule *sched) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!sched) return fail(ctx, GS_ERR_INVALID_ARG, "schedule is NULL");
    if (!valid_schedule(*sched))
        return fail(ctx, GS_ERR_INVALID_ARG,
                    "tile_w in {8, 16, 32}, tile_h in {4, 8, 16, 32} with 64 to 256 pixels, sub_buckets 1, 2 or 4, "
                    "batch depths 64, 128 or 256 and at most the tile's pixels");
    ctx->sched = *sched;
    return GS_OK;
}

gs_status gs_autotune(gs_ctx *ctx, const gs_problem *prob, const gs_gaussians *g, const double *poses,
                      const gs_targets *targets, int32_t pose_only, int32_t reps, void *ws, size_t ws_bytes,
                      gs_tune_entry *table, int32_t cap, int32_t *count, gs_schedule *best, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (reps < 1 || reps > 1000) return fail(ctx, GS_ERR_INVALID_ARG, "reps must be in [1, 1000]");
    if (cap < 0 || (cap > 0 && !table)) return fail(ctx, GS_ERR_INVALID_ARG, "table is NULL or cap negative");
    if (!targets || !targets->rgb || !targets->depth) return fail(ctx, GS_ERR_INVALID_ARG, "targets need rgb and depth");
    if (!poses) return fail(ctx, GS_ERR_INVALID_ARG, "poses is NULL");
    Problem pr;
    gs_status st = build_problem(ctx, prob, pr);
    if (st != GS_OK) return st;
    if ((st = check_gaussians(ctx, g, pr)) != GS_OK) return st;
    if (!ws || ws_bytes < pr.lay.total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
        return fail(ctx, GS_ERR_WORKSPACE, "workspace NULL, smaller than gs_workspace_size or not 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &capst);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream query");
    if (capst != cudaStreamCaptureStatusNone)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_autotune synchronises and cannot be captured");
    const WsPtrs w = ws_ptrs(ws, pr.lay);
    const GaussPtrs gp{g->means, g->quats, g->log_scales, g->opacity_logits, g->rgb};
    // the passes overwrite whatever projection was bound; no profiling markers inside them
    ctx->bound = false;
    const uint32_t prof_saved = ctx->prof_mask;
    const gs_schedule sched_saved = ctx->sched;
    ctx->prof_mask = 0;
    reset_marks(ctx);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    gs_tune_entry ent[17];
    int n_ent = 0;
    gs_schedule cur = ctx->sched;
    bool overflow = false;  // the context's own schedule overflowed the pair capacity

    // The problem (views, tile grid, sizes) of schedule `sc`, on the same workspace layout.
    auto problem_for = [&](const gs_schedule &sc, Problem &out) -> gs_status {
        ctx->sched = sc;
        const gs_status r = build_problem(ctx, prob, out);
        ctx->sched = sched_saved;
        return r;
    };
    // One pass of stage `which` (0: all, 1: binning, 2: forward, 3: backward, 4: both
    // compositors as the tracking step runs them, 5: binning, sort and both compositors as
    // the caller will run them).
    auto enqueue_stage = [&](int which, const Problem &q) -> cudaError_t {
        cudaError_t r = cudaSuccess;
        if (which == 4) return enqueue_compositing(ctx, q, w, targets, s);
        if (which == 5 && pose_only) {
            r = enqueue_project(ctx, q, w, gp, g->dtype_attr, poses, s);
            return r == cudaSuccess ? enqueue_compositing(ctx, q, w, targets, s) : r;
        }
        if (which == 5) which = 0;
        if (which <= 1) r = enqueue_project(ctx, q, w, gp, g->dtype_attr, poses, s);
        if (r == cudaSuccess && (which == 0 || which == 2))
            r = enqueue_forward(ctx, q, w, targets, nullptr, nullptr, nullptr, s);
        if (r == cudaSuccess && (which == 0 || which == 3)) {
            BackwardLaunch B;
            B.ws = w;
            B.d = q.d;
            B.s = ctx->s;
            B.up_rgb = w.upstream;
            B.up_depth = w.upstream + 3u * q.d.P;
            B.up_sil = w.upstream + 4u * q.d.P;
            B.pose_only = pose_only != 0;
            r = launch_backward(B, s);
        }
        return r;
    };
    // Did the work enqueued since the last check overflow a capacity?  Clears the flag.
    auto overflowed = [&](bool &flag) -> cudaError_t {
        uint32_t err = 0;
        cudaError_t r = cudaStreamSynchronize(s);
        if (r == cudaSuccess) r = cudaMemcpy(&err, w.err, sizeof(err), cudaMemcpyDeviceToHost);
        if (r == cudaSuccess && err) r = cudaMemset(w.err, 0, sizeof(err));
        flag = (err & (kErrRecords | kErrPairs | kErrTimeout)) != 0;
        return r;
    };
    // Time the candidates of one stage (the first is the current setting) and keep the
    // fastest in `cur`; candidates that overflow are recorded with ms = -1.
    auto stage = [&](int which, const gs_schedule *cand, int ncand) -> cudaError_t {
        float ms[4];
        int idx[4], nv = 0;
        for (int k = 0; k < ncand; ++k) {
            Problem q;
            if (problem_for(cand[k], q) != GS_OK) continue;
            // an untimed pass through the whole chain (binning, forward, backward) leaves
            // the state this stage's passes read, then the overflow check
            cudaError_t r = upload_views(q, w, ws, s);
            if (r == cudaSuccess) r = enqueue_stage(0, q);
            bool of = false;
            if (r == cudaSuccess) r = overflowed(of);
            if (r != cudaSuccess) return r;
            if (of) {
                if (k == 0) overflow = true;
                ent[n_ent++] = gs_tune_entry{which, -1.f, cand[k]};
                continue;
            }
            float t = 0.f;
            r = time_passes(s, ev[0], ev[1], reps, [&]() { return enqueue_stage(which, q); }, t);
            if (r != cudaSuccess) return r;
            ent[n_ent++] = gs_tune_entry{which, t, cand[k]};
            ms[nv] = t;
            idx[nv++] = k;
        }
        if (nv > 0 && idx[0] == 0) cur = cand[idx[pick(ms, nv)]];
        else if (nv > 0) {  // the current setting overflowed: the fastest of the others
            int b = 0;
            for (int k = 1; k < nv; ++k)
                if (ms[k] < ms[b]) b = k;
            cur = cand[idx[b]];
        }
        return cudaSuccess;
    };

    e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    // stage 0: tile shapes (the current one first), batch depths capped at the threads
    if (e == cudaSuccess) {
        const int32_t shapes[4][2] = {{16, 16}, {32, 8}, {16, 8}, {8, 8}};
        gs_schedule cand[4];
        int nc = 0;
        cand[nc++] = cur;
        for (const auto &sh : shapes) {
            if (sh[0] == cur.tile_w && sh[1] == cur.tile_h) continue;
            gs_schedule c = cur;
            c.tile_w = sh[0];
            c.tile_h = sh[1];
            c.fwd_batch = std::min(c.fwd_batch, c.tile_w * c.tile_h);
            c.bwd_batch = std::min(c.bwd_batch, c.tile_w * c.tile_h);
            if (nc < 4 && valid_schedule(c)) cand[nc++] = c;
        }
        e = stage(0, cand, nc);
    }
    // stage 1: sub-buckets; stages 2 and 3: batch depths up to the tile's threads
    const int32_t subs[3] = {4, 2, 1}, batches[3] = {256, 128, 64};
    for (int which = 1; which <= 3 && e == cudaSuccess; ++which) {
        gs_schedule cand[4];
        int nc = 0;
        cand[nc++] = cur;
        for (int k = 0; k < 3; ++k) {
            gs_schedule c = cur;
            int32_t &field = which == 1 ? c.sub_buckets : (which == 2 ? c.fwd_batch : c.bwd_batch);
            const int32_t v = which == 1 ? subs[k] : batches[k];
            if (v == field) continue;
            field = v;
            if (which == 1) {  // the problem may allow fewer sub-buckets than asked
                Problem q;
                if (problem_for(c, q) != GS_OK || q.d.S != (uint32_t)v) continue;
            }
            if (valid_schedule(c)) cand[nc++] = c;
        }
        e = stage(which, cand, nc);
    }
    // stage 4 (tracking): the two compositors as two kernels or as one (GS_SCHED_FUSED)
    if (e == cudaSuccess && pose_only) {
        gs_schedule c = cur;
        c.flags ^= GS_SCHED_FUSED;
        if (c.flags & GS_SCHED_FUSED) c.bwd_batch = c.fwd_batch;
        const gs_schedule cand[2] = {cur, c};
        e = stage(4, cand, valid_schedule(c) ? 2 : 1);
    }
    // stage 5: the per-tile sort or the device-wide radix sort (GS_SCHED_RADIX)
    if (e == cudaSuccess) {
        gs_schedule c = cur;
        c.flags ^= GS_SCHED_RADIX;
        const gs_schedule cand[2] = {cur, c};
        e = stage(5, cand, 2);
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    ctx->prof_mask = prof_saved;
    ctx->sched = sched_saved;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
    if (table)
        for (int k = 0; k < n_ent && k < cap; ++k) table[k] = ent[k];
    if (count) *count = n_ent;
    if (overflow)
        return fail(ctx, GS_ERR_CAPACITY, "the problem overflowed its capacities during tuning; schedule unchanged");
    ctx->sched = cur;
    if (best) *best = cur;
    ctx->err.clear();  // a candidate the problem could not take left its message
    return GS_OK;
}

gs_status gs_set_profiling(gs_ctx *ctx, int32_t enable) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    ctx->prof_mask = enable ? kAllKernels : 0u;
    reset_marks(ctx);
    return GS_OK;
}

gs_status gs_set_profiling_mask(gs_ctx *ctx, uint32_t mask) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (mask & ~kAllKernels) return fail(ctx, GS_ERR_INVALID_ARG, "profiling mask selects an unknown kernel");
    ctx->prof_mask = mask;
    reset_marks(ctx);
    return GS_OK;
}

gs_status gs_kernel_times(gs_ctx *ctx, gs_kernel_time *out, int32_t cap, int32_t *count) {
    if (!ctx || !count || cap < 0 || (cap > 0 && !out)) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->prof_mask || ctx->n_marks < 2) return fail(ctx, GS_ERR_STATE, "profiling off or nothing recorded");
    cudaError_t e = cudaEventSynchronize(ctx->events[ctx->n_marks - 1]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event synchronize");
    int32_t k = 0;
    for (size_t m = 1; m < ctx->n_marks; ++m) {
        if (!ctx->names[m]) continue;
        if (k < cap) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ctx->events[m - 1], ctx->events[m]);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "event elapsed time");
            std::snprintf(out[k].name, sizeof out[k].name, "%s", ctx->names[m]);
            out[k].ms = ms;
        }
        ++k;
    }
    *count = k;
    return GS_OK;
}

gs_status gs_pose_partials(gs_ctx *ctx, float *out, int64_t cap, int64_t *count, void *stream) {
    if (!ctx || !count || cap < 0 || (cap > 0 && !out)) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->bound) return fail(ctx, GS_ERR_STATE, "no projection is bound");
    const int64_t n = (int64_t)ctx->prob.d.V * (int64_t)ctx->prob.d.nblk * 12;
    *count = n;
    if (cap < n) return GS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(out, ctx->ws.pose_part, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pose partials copy");
    return GS_OK;
}

gs_status gs_sync_status(gs_ctx *ctx, void *stream, gs_counts *counts) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->bound) return fail(ctx, GS_ERR_STATE, "no workspace bound");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    DevHeader h{};
    uint32_t err = 0;
    if ((e = cudaMemcpy(&h, ctx->ws.hdr, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(ctx, e, "header read");
    if ((e = cudaMemcpy(&err, ctx->ws.err, sizeof(err), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(ctx, e, "flag read");
    if (err && (e = cudaMemset(ctx->ws.err, 0, sizeof(err))) != cudaSuccess) return cuda_fail(ctx, e, "flag clear");
    if (counts) {
        counts->n_records = (int64_t)h.n_rec;
        counts->n_pairs = (int64_t)h.n_pairs;
        counts->err_flags = err;
        counts->reserved = 0;
        counts->fwd_evals = (int64_t)h.fwd_evals;
        counts->fwd_contrib = (int64_t)h.fwd_contrib;
        counts->bwd_evals = (int64_t)h.bwd_evals;
        counts->bwd_contrib = (int64_t)h.bwd_contrib;
        counts->max_tile = h.max_tile;
    }
    if (err & kErrTimeout) return fail(ctx, GS_ERR_TIMEOUT, "a bounded device wait expired");
    if (err & (kErrRecords | kErrPairs)) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "capacity exceeded: %llu pairs (capacity %u)", (unsigned long long)h.n_pairs,
                      ctx->prob.d.pair_cap);
        return fail(ctx, GS_ERR_CAPACITY, msg);
    }
    return GS_OK;
}

}  // extern "C"
