// gs_static.cu -- gs_render_static: the single-view render with its scratch memory in a
// file-scope device array instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need a render: a
// plugin or a real-time loop running under a host application whose memory pool it
// does not own (a custom allocator, a pre-reserved budget, a context where
// cudaMalloc / cudaFree are forbidden because they synchronise the device).  This entry
// point lets them render with no allocation at all: the scratch lives in the static
// array below, which every GPU that loads this library holds until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "gs_internal.cuh"

using namespace gsk;

namespace {

// Limits of one call (also in include/gs.h).
constexpr int64_t kMaxGaussians = GS_STATIC_MAX_GAUSSIANS;
constexpr int64_t kMaxPixels = GS_STATIC_MAX_PIXELS;
constexpr int64_t kMaxPairs = GS_STATIC_MAX_PAIRS;
constexpr size_t kAlign = 256;

constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte layout of the scratch for the largest call (tile counts use the largest tile
// grid a kMaxPixels image can have: one pixel row or column of ragged tiles per side).
constexpr int64_t kMaxCells = (kMaxGaussians + kBlock - 1) / kBlock;
constexpr int64_t kMaxTiles = kMaxPixels / (kTile * kTile) + 2 * (kMaxPixels / kTile) + 2;
constexpr size_t kScratchBytes =
    up(4) + up(sizeof(DevHeader)) + up(4 * (4 * kMaxTiles + 1)) + up(sizeof(ViewInfo)) + up(12 * 4) +
    up(4 * kMaxCells) + 2 * up(4 * (4 * kMaxTiles + 1)) + up(4 * kMaxTiles) + up(4 * kBigListCap) + up(kMaxCells * kCell) +
    2 * up(48 * kMaxCells * kCell) +
    up(8 * kMaxPairs) + up(4 * kMaxPairs) + up(4 * kMaxPixels) + up(4 * kMaxPixels) + up(20 * kMaxPixels) +
    up(8 * kMaxTiles) + up(48 * kMaxCells);

// The scratch.  In host code this name is only a stand-in: its device address comes
// from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Device address of g_scratch on the current device (looked up on the first call).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" gs_status gs_render_static(const gs_config *cfg, const gs_gaussians *g, const gs_camera *cam,
                                      const double *pose, const gs_targets *targets, float *rgb, float *depth,
                                      float *sil, double *loss, uint32_t *err_flags, void *stream) {
    if (!cfg || !g || !cam || !pose) return GS_ERR_INVALID_ARG;
    if (cfg->tile_w != kTile || cfg->tile_h != kTile) return GS_ERR_UNSUPPORTED;
    if (g->n < 0 || g->n > kMaxGaussians) return GS_ERR_INVALID_ARG;
    if (cam->width < 1 || cam->height < 1 || (int64_t)cam->width * cam->height > kMaxPixels || !(cam->fx > 0) ||
        !(cam->fy > 0))
        return GS_ERR_INVALID_ARG;
    if (g->dtype_attr != GS_F32 && g->dtype_attr != GS_BF16 && g->dtype_attr != GS_F16) return GS_ERR_INVALID_ARG;
    if (g->n > 0 && (!g->means || !g->log_scales || !g->opacity_logits || !g->rgb))
        return GS_ERR_INVALID_ARG;
    if (targets && (!targets->rgb || !targets->depth)) return GS_ERR_INVALID_ARG;
    if (loss && !targets) return GS_ERR_INVALID_ARG;

    // sizes and settings of this call
    ViewInfo vi{};
    vi.fx = (float)cam->fx;
    vi.fy = (float)cam->fy;
    vi.cx = (float)cam->cx;
    vi.cy = (float)cam->cy;
    vi.width = cam->width;
    vi.height = cam->height;
    vi.tiles_x = (cam->width + kTile - 1) / kTile;
    vi.tiles_y = (cam->height + kTile - 1) / kTile;
    static_assert(kTile == 16, "the static render uses 16 x 16 tiles");
    vi.tile_lw = vi.tile_lh = 4;  // 16 x 16 tiles
    vi.tan_lim_x = jacobian_tangent_limit(cfg->jac_clip, cam->width, cam->fx);
    vi.tan_lim_y = jacobian_tangent_limit(cfg->jac_clip, cam->height, cam->fy);
    Dims d{};
    d.n = g->n;
    d.V = 1;
    d.nblk = (int32_t)((g->n + kBlock - 1) / kBlock);
    if (d.nblk == 0) d.nblk = 1;
    d.T = (uint32_t)(vi.tiles_x * vi.tiles_y);
    d.S = 4;
    d.tile_threads = kTilePix;
    d.tile_lw = 4;
    d.P = (uint32_t)(cam->width * cam->height);
    d.pair_cap = (uint32_t)kMaxPairs;
    if ((int64_t)d.T > kMaxTiles) return GS_ERR_INVALID_ARG;
    Settings s{};
    s.alpha_min = cfg->alpha_min;
    s.alpha_max = cfg->alpha_max;
    s.t_min = cfg->t_min;
    s.dilation = cfg->dilation;
    s.z_near = cfg->z_near;
    s.sil_thresh = cfg->sil_thresh;
    s.log2_alpha_min = cfg->alpha_min > 0.f ? (float)std::log2((double)cfg->alpha_min) : -INFINITY;
    s.w_rgb = cfg->w_rgb;
    s.w_depth = cfg->w_depth;
    s.w_vis = cfg->w_vis;
    s.w_prior = cfg->w_prior;

    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return GS_ERR_CUDA;
    char *b = static_cast<char *>(base);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char *p = b + o;
        o += up(bytes);
        return p;
    };
    WsPtrs w{};
    w.err = reinterpret_cast<uint32_t *>(take(4));
    w.hdr = reinterpret_cast<DevHeader *>(take(sizeof(DevHeader)));
    w.tile_cnt = reinterpret_cast<uint32_t *>(take(4 * ((size_t)d.T * d.S + 1)));
    const size_t zero_bytes = o;  // err word, header and tile counts start at zero
    w.views = reinterpret_cast<ViewInfo *>(take(sizeof(ViewInfo)));
    w.view_rt = reinterpret_cast<float *>(take(12 * 4));
    w.cell_cnt = reinterpret_cast<uint32_t *>(take(4 * (size_t)d.nblk));
    w.tile_start = reinterpret_cast<uint32_t *>(take(4 * ((size_t)d.T * d.S + 1)));
    w.cursor = reinterpret_cast<uint32_t *>(take(4 * ((size_t)d.T * d.S + 1)));
    w.tile_order = reinterpret_cast<uint32_t *>(take(4 * (size_t)d.T));
    w.big = reinterpret_cast<uint32_t *>(take(4 * (size_t)kBigListCap));
    w.big_listed = reinterpret_cast<uint8_t *>(take((size_t)d.nblk * kCell));
    w.rec = reinterpret_cast<Rec *>(take(sizeof(Rec) * (size_t)d.nblk * kCell));
    w.rec_grad = reinterpret_cast<RecGrad *>(take(sizeof(RecGrad) * (size_t)d.nblk * kCell));
    w.keys = reinterpret_cast<unsigned long long *>(take(8 * (size_t)d.pair_cap));
    w.sorted = reinterpret_cast<uint32_t *>(take(4 * (size_t)d.pair_cap));
    w.t_final = reinterpret_cast<float *>(take(4 * (size_t)d.P));
    w.n_last = reinterpret_cast<uint32_t *>(take(4 * (size_t)d.P));
    w.upstream = reinterpret_cast<float *>(take(20 * (size_t)d.P));
    w.tile_loss = reinterpret_cast<float2 *>(take(8 * (size_t)d.T));
    w.pose_part = reinterpret_cast<float2 *>(take(48 * (size_t)d.nblk));
    if (o > kScratchBytes) return GS_ERR_WORKSPACE;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (launch_upload_views(&vi, 1, w.views, base, zero_bytes, st) != cudaSuccess) return GS_ERR_CUDA;
    ProjectLaunch P{};
    P.ws = w;
    P.d = d;
    P.s = s;
    P.g = GaussPtrs{g->means, g->quats, g->log_scales, g->opacity_logits, g->rgb};
    P.dtype = g->dtype_attr;
    P.poses = pose;
    if (launch_project(P, st) != cudaSuccess) return GS_ERR_CUDA;
    if (launch_scan_tiles(w, d, st) != cudaSuccess) return GS_ERR_CUDA;
    if (launch_emit(w, d, st) != cudaSuccess) return GS_ERR_CUDA;
    ForwardLaunch F{};
    F.ws = w;
    F.d = d;
    F.s = s;
    F.rgb = rgb;
    F.depth = depth;
    F.sil = sil;
    F.t_rgb = targets ? targets->rgb : nullptr;
    F.t_depth = targets ? targets->depth : nullptr;
    F.t_prior = targets ? targets->depth_prior : nullptr;
    if (launch_forward(F, st) != cudaSuccess) return GS_ERR_CUDA;
    if (loss) {
        FinalizeLaunch Z{};
        Z.ws = w;
        Z.d = d;
        Z.s = s;
        Z.loss_out = loss;
        if (launch_finalize(Z, st) != cudaSuccess) return GS_ERR_CUDA;
    }
    if (err_flags && cudaMemcpyAsync(err_flags, w.err, 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return GS_ERR_CUDA;
    return GS_OK;
}
