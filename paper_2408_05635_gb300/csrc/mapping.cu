// mapping.cu -- the map side of the method: Gaussians made from an RGB-D frame (the first
// frame, Sec. III-A, and the new observations of a keyframe, Sec. III-C), the
// gradient-based update of every Gaussian parameter with the keyframe poses fixed, and
// the removal of Gaussians whose opacity fell away (duplicate removal, Sec. III-C).
//
// All three are HBM-bound passes over flat arrays.  The two that change the number of
// Gaussians are stable compactions in two launches: a block-count pass, then an emit
// pass in which every block sums the counts of the blocks before it (at most a few
// thousand words, read from L2) and scatters its items in order.  No block waits on
// another, and the live count stays on the device.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "gs_internal.cuh"

namespace {

constexpr int kCompactThreads = 1024;
constexpr int kGroups = 5;  // means, quats, log_scales, opacity_logits, rgb
// Values per Gaussian of each group, and the group's first row in a moment array (in units
// of capacity); isotropic maps (Eq. 1 as written) have no quaternion and one log-radius.
__host__ __device__ constexpr int group_width(int s, bool iso) {
    return s == 1 ? (iso ? 0 : 4) : (s == 2 ? (iso ? 1 : 3) : (s == 3 ? 1 : 3));
}
__host__ __device__ constexpr int group_offset(int s, bool iso) {
    return iso ? (s == 0 ? 0 : (s <= 2 ? 3 : (s == 3 ? 4 : 5))) : (s == 0 ? 0 : (s == 1 ? 3 : (s == 2 ? 7 : (s == 3 ? 10 : 11))));
}
__host__ __device__ constexpr int values_per_gaussian(bool iso) { return iso ? 8 : 14; }

struct MapView {
    float *p[kGroups];
    void *lp[kGroups];  // lp[0] is always NULL (the means have no low-precision copy)
    int32_t lowp_dt;
    bool iso;      // no quaternions, one log-radius
    int64_t cap;
    float *state;  // m: groups at cap * group_offset; v: values_per_gaussian cap further
};

MapView view_of(const gs_map &m) {
    MapView v{};
    v.p[0] = m.means;
    v.p[1] = m.quats;
    v.p[2] = m.log_scales;
    v.p[3] = m.opacity_logits;
    v.p[4] = m.rgb;
    v.lp[0] = nullptr;
    v.lp[1] = m.lowp_quats;
    v.lp[2] = m.lowp_log_scales;
    v.lp[3] = m.lowp_opacity_logits;
    v.lp[4] = m.lowp_rgb;
    v.lowp_dt = m.lowp_dtype;
    v.iso = m.quats == nullptr;
    v.cap = m.capacity;
    v.state = m.adam_state;
    return v;
}

__device__ __forceinline__ void store_lowp(void *base, int64_t i, float x, int dt) {
    if (dt == GS_BF16)
        static_cast<__nv_bfloat16 *>(base)[i] = __float2bfloat16_rn(x);
    else
        static_cast<__half *>(base)[i] = __float2half_rn(x);
}

__device__ __forceinline__ void copy_lowp(const void *src, int64_t i, void *dst, int64_t j, int dt) {
    if (dt == GS_BF16)
        static_cast<__nv_bfloat16 *>(dst)[j] = static_cast<const __nv_bfloat16 *>(src)[i];
    else
        static_cast<__half *>(dst)[j] = static_cast<const __half *>(src)[i];
}

// Sum of counts[0, b) over the block, and the total when b is the last block.
__device__ uint32_t block_prefix(const uint32_t *counts, uint32_t b) {
    __shared__ uint32_t s_w[kCompactThreads / 32];
    uint32_t acc = 0;
    for (uint32_t k = threadIdx.x; k < b; k += blockDim.x) acc += counts[k];
    acc = __reduce_add_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    uint32_t tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_w[w];
    __syncthreads();
    return tot;
}

// Exclusive rank of this thread's flag within the block, and the block's count.
__device__ uint32_t block_rank(bool flag, uint32_t &count) {
    __shared__ uint32_t s_w[kCompactThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t bal = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) s_w[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = lane < nw ? s_w[lane] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < nw) s_w[lane] = incl - x;
        if (lane == nw - 1) s_w[kCompactThreads / 32] = incl;
    }
    __syncthreads();
    const uint32_t r = s_w[warp] + __popc(bal & ((1u << lane) - 1u));
    count = s_w[kCompactThreads / 32];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ new Gaussians

struct AddLaunch {
    MapView map;
    int64_t *n;
    const double *pose;
    const float *rgb, *depth, *sil;
    float sil_add;
    double fx, fy, cx, cy;
    int32_t width, height;
    uint32_t *counts;  // scratch: one word per block
    int64_t *n0;       // scratch: the live count before the call
    uint32_t *err;
};

__device__ __forceinline__ bool add_flag(const AddLaunch &L, int64_t p, int64_t P) {
    if (p >= P) return false;
    const float d = L.depth[p];
    return d > 0.f && (L.sil == nullptr || L.sil[p] < L.sil_add);
}

__global__ void __launch_bounds__(kCompactThreads) k_add_count(AddLaunch L) {
    const int64_t P = (int64_t)L.width * L.height;
    const int64_t p = (int64_t)blockIdx.x * kCompactThreads + threadIdx.x;
    const uint32_t c = (uint32_t)__syncthreads_count(add_flag(L, p, P));
    if (threadIdx.x == 0) {
        L.counts[blockIdx.x] = c;
        if (blockIdx.x == 0) *L.n0 = *L.n;
    }
}

__global__ void __launch_bounds__(kCompactThreads) k_add_emit(AddLaunch L) {
    __shared__ double s_R[9], s_t[3];
    const int64_t P = (int64_t)L.width * L.height;
    const int64_t p = (int64_t)blockIdx.x * kCompactThreads + threadIdx.x;
    if (threadIdx.x == 0) {
        // world->camera rotation of the pose's unit quaternion (renormalised), in FP64
        double w = L.pose[0], x = L.pose[1], y = L.pose[2], z = L.pose[3];
        const double inv = 1.0 / sqrt(w * w + x * x + y * y + z * z);
        w *= inv; x *= inv; y *= inv; z *= inv;
        s_R[0] = 1.0 - 2.0 * (y * y + z * z); s_R[1] = 2.0 * (x * y - w * z); s_R[2] = 2.0 * (x * z + w * y);
        s_R[3] = 2.0 * (x * y + w * z); s_R[4] = 1.0 - 2.0 * (x * x + z * z); s_R[5] = 2.0 * (y * z - w * x);
        s_R[6] = 2.0 * (x * z - w * y); s_R[7] = 2.0 * (y * z + w * x); s_R[8] = 1.0 - 2.0 * (x * x + y * y);
        s_t[0] = L.pose[4]; s_t[1] = L.pose[5]; s_t[2] = L.pose[6];
    }
    const uint32_t before = block_prefix(L.counts, blockIdx.x);
    const bool flag = add_flag(L, p, P);
    uint32_t count;
    const uint32_t r = block_rank(flag, count);
    const int64_t n0 = *L.n0;
    const int64_t i = n0 + before + r;
    const MapView &M = L.map;
    if (flag && i < M.cap) {
        const int64_t v = p / L.width, u = p - v * L.width;
        const double d = (double)L.depth[p];
        // the pixel's sample point at depth d in the camera frame (inverse of pi_m), then
        // world = R^T (x_c - t)
        const double xc0 = ((double)u - L.cx) / L.fx * d - s_t[0];
        const double xc1 = ((double)v - L.cy) / L.fy * d - s_t[1];
        const double xc2 = d - s_t[2];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            M.p[0][3 * i + k] = (float)(s_R[k] * xc0 + s_R[3 + k] * xc1 + s_R[6 + k] * xc2);
        const float ls = (float)log(d / (0.5 * (L.fx + L.fy)));
        const float q[4] = {1.f, 0.f, 0.f, 0.f};
        const float c[3] = {L.rgb[p], L.rgb[P + p], L.rgb[2 * P + p]};
        const int wl = group_width(2, M.iso);
        if (!M.iso) {
#pragma unroll
            for (int k = 0; k < 4; ++k) M.p[1][4 * i + k] = q[k];
        }
        for (int k = 0; k < wl; ++k) M.p[2][wl * i + k] = ls;
        M.p[3][i] = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) M.p[4][3 * i + k] = c[k];
        if (M.lp[2]) {
            if (M.lp[1]) {
#pragma unroll
                for (int k = 0; k < 4; ++k) store_lowp(M.lp[1], 4 * i + k, q[k], M.lowp_dt);
            }
            for (int k = 0; k < wl; ++k) store_lowp(M.lp[2], wl * i + k, ls, M.lowp_dt);
            store_lowp(M.lp[3], i, 0.f, M.lowp_dt);
#pragma unroll
            for (int k = 0; k < 3; ++k) store_lowp(M.lp[4], 3 * i + k, c[k], M.lowp_dt);
        }
        if (M.state) {
            const int vp = values_per_gaussian(M.iso);
#pragma unroll
            for (int s = 0; s < kGroups; ++s) {
                const int w = group_width(s, M.iso);
                float *m = M.state + M.cap * group_offset(s, M.iso);
                float *vv = m + vp * M.cap;
                for (int k = 0; k < w; ++k) {
                    m[w * i + k] = 0.f;
                    vv[w * i + k] = 0.f;
                }
            }
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        int64_t n1 = n0 + before + count;
        if (n1 > M.cap) {
            n1 = M.cap;
            if (L.err) atomicOr(L.err, 1u);
        }
        *L.n = n1;
    }
}

// ------------------------------------------------------------------ Adam

struct AdamLaunch {
    float *p[kGroups];
    const float *g[kGroups];
    void *lp[kGroups];
    float *m[kGroups], *v[kGroups];
    float lr[kGroups];
    int width[kGroups];
    float b1, b2, omb1, omb2, c1, c2, eps;
    int32_t lowp_dt;
    const int64_t *n;
};

__device__ __forceinline__ float adam_one(float &p, float g, float &m, float &v, float lr, const AdamLaunch &L) {
    m = L.b1 * m + L.omb1 * g;
    v = L.b2 * v + L.omb2 * (g * g);
    const float mh = m * L.c1, vh = v * L.c2;
    p = p - lr * (mh / (sqrtf(vh) + L.eps));
    return p;
}

// blockIdx.y selects the group; a grid-stride loop over its float4 quads, the ragged
// tail (fewer than four values) taken by block 0.
__global__ void __launch_bounds__(256) k_map_adam(AdamLaunch L) {
    const int s = blockIdx.y;
    if (L.g[s] == nullptr || L.width[s] == 0) return;
    const int64_t len = (int64_t)L.width[s] * (*L.n);
    const float lr = L.lr[s];
    float *p = L.p[s], *m = L.m[s], *v = L.v[s];
    const float *g = L.g[s];
    void *lp = L.lp[s];
    const int64_t nq = len >> 2;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        float4 P4 = reinterpret_cast<float4 *>(p)[q];
        const float4 G4 = __ldg(reinterpret_cast<const float4 *>(g) + q);
        float4 M4 = reinterpret_cast<float4 *>(m)[q];
        float4 V4 = reinterpret_cast<float4 *>(v)[q];
        adam_one(P4.x, G4.x, M4.x, V4.x, lr, L);
        adam_one(P4.y, G4.y, M4.y, V4.y, lr, L);
        adam_one(P4.z, G4.z, M4.z, V4.z, lr, L);
        adam_one(P4.w, G4.w, M4.w, V4.w, lr, L);
        reinterpret_cast<float4 *>(p)[q] = P4;
        reinterpret_cast<float4 *>(m)[q] = M4;
        reinterpret_cast<float4 *>(v)[q] = V4;
        if (lp) {
            if (L.lowp_dt == GS_BF16) {
                __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(lp) + 2 * q;
                o[0] = __floats2bfloat162_rn(P4.x, P4.y);
                o[1] = __floats2bfloat162_rn(P4.z, P4.w);
            } else {
                __half2 *o = reinterpret_cast<__half2 *>(lp) + 2 * q;
                o[0] = __floats2half2_rn(P4.x, P4.y);
                o[1] = __floats2half2_rn(P4.z, P4.w);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < (len & 3)) {
        const int64_t k = 4 * nq + threadIdx.x;
        float pk = p[k], mk = m[k], vk = v[k];
        adam_one(pk, g[k], mk, vk, lr, L);
        p[k] = pk;
        m[k] = mk;
        v[k] = vk;
        if (lp) store_lowp(lp, k, pk, L.lowp_dt);
    }
}

// ------------------------------------------------------------------ removal

struct PruneLaunch {
    MapView src, dst;
    const int64_t *n_src;
    int64_t *n_dst;
    float logit_min;
    uint32_t *counts;
    int64_t *n0;
};

__global__ void __launch_bounds__(kCompactThreads) k_prune_count(PruneLaunch L) {
    const int64_t i = (int64_t)blockIdx.x * kCompactThreads + threadIdx.x;
    const int64_t n = *L.n_src;
    const bool keep = i < n && L.src.p[3][i] >= L.logit_min;
    const uint32_t c = (uint32_t)__syncthreads_count(keep);
    if (threadIdx.x == 0) {
        L.counts[blockIdx.x] = c;
        if (blockIdx.x == 0) *L.n0 = n;
    }
}

__global__ void __launch_bounds__(kCompactThreads) k_prune_emit(PruneLaunch L) {
    const int64_t i = (int64_t)blockIdx.x * kCompactThreads + threadIdx.x;
    const int64_t n = *L.n0;
    const uint32_t before = block_prefix(L.counts, blockIdx.x);
    const bool keep = i < n && L.src.p[3][i] >= L.logit_min;
    uint32_t count;
    const uint32_t r = block_rank(keep, count);
    const MapView &S = L.src, &D = L.dst;
    if (keep) {
        const int64_t j = (int64_t)before + r;
        const int vp = values_per_gaussian(S.iso);
#pragma unroll
        for (int s = 0; s < kGroups; ++s) {
            const int w = group_width(s, S.iso);
            for (int k = 0; k < w; ++k) D.p[s][w * j + k] = S.p[s][w * i + k];
            if (s > 0 && S.lp[s] && D.lp[s] && S.lowp_dt == D.lowp_dt)
                for (int k = 0; k < w; ++k) copy_lowp(S.lp[s], w * i + k, D.lp[s], w * j + k, D.lowp_dt);
            if (S.state && D.state) {
                const float *sm = S.state + S.cap * group_offset(s, S.iso);
                float *dm = D.state + D.cap * group_offset(s, S.iso);
                for (int k = 0; k < w; ++k) {
                    dm[w * j + k] = sm[w * i + k];
                    dm[vp * D.cap + w * j + k] = sm[vp * S.cap + w * i + k];
                }
            }
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *L.n_dst = (int64_t)before + count;
}

// ------------------------------------------------------------------ host side

constexpr size_t kScratchHead = 256;  // the saved live count, then one word per block

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool map_ok(const gs_map *m) {
    if (!m || m->capacity < 0 || (m->capacity & 3) != 0) return false;
    const bool iso = m->quats == nullptr;  // isotropic: no quaternions anywhere
    const float *f[5] = {m->means, iso ? m->means : m->quats, m->log_scales, m->opacity_logits, m->rgb};
    for (const float *q : f)
        if (!q || !aligned16(q)) return false;
    if (iso && m->lowp_quats) return false;
    const void *l[4] = {iso ? m->lowp_log_scales : m->lowp_quats, m->lowp_log_scales, m->lowp_opacity_logits,
                        m->lowp_rgb};
    const bool any = l[0] || l[1] || l[2] || l[3];
    if (any) {
        if (m->lowp_dtype != GS_BF16 && m->lowp_dtype != GS_F16) return false;
        for (const void *q : l)
            if (!q || !aligned16(q)) return false;
    }
    return !m->adam_state || aligned16(m->adam_state);
}

size_t scratch_bytes_for(int64_t items) {
    const int64_t blocks = (items + kCompactThreads - 1) / kCompactThreads;
    return kScratchHead + (size_t)(4 * blocks + 255) / 256 * 256;
}

}  // namespace

extern "C" {

void gs_default_map_config(gs_map_config *c) {
    if (!c) return;
    c->lr_means = 1e-4;
    c->lr_quats = 1e-3;
    c->lr_log_scales = 1e-3;
    c->lr_opacity_logits = 5e-2;
    c->lr_rgb = 2.5e-3;
    c->beta1 = 0.9;
    c->beta2 = 0.999;
    c->eps = 1e-15;
    c->sil_add = 0.5f;
    c->opacity_min = 0.005f;
}

size_t gs_map_scratch_bytes(int64_t items) { return items < 0 ? 0 : scratch_bytes_for(items); }

gs_status gs_map_add(const gs_map_config *cfg, const gs_map *map, int64_t *n, const gs_camera *cam,
                     const double *pose, const float *rgb, const float *depth, const float *sil, void *scratch,
                     size_t scratch_bytes, uint32_t *err_flags, void *stream) {
    if (!cfg || !map_ok(map) || !n || !cam || !pose || !rgb || !depth || !scratch) return GS_ERR_INVALID_ARG;
    if (cam->width < 1 || cam->height < 1 || !(cam->fx > 0) || !(cam->fy > 0)) return GS_ERR_INVALID_ARG;
    const int64_t P = (int64_t)cam->width * cam->height;
    if (P >= (1ll << 31) || (reinterpret_cast<uintptr_t>(scratch) & 255u) != 0 ||
        scratch_bytes < scratch_bytes_for(P))
        return GS_ERR_INVALID_ARG;
    AddLaunch L{};
    L.map = view_of(*map);
    L.n = n;
    L.pose = pose;
    L.rgb = rgb;
    L.depth = depth;
    L.sil = sil;
    L.sil_add = cfg->sil_add;
    L.fx = cam->fx;
    L.fy = cam->fy;
    L.cx = cam->cx;
    L.cy = cam->cy;
    L.width = cam->width;
    L.height = cam->height;
    L.n0 = static_cast<int64_t *>(scratch);
    L.counts = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + kScratchHead);
    L.err = err_flags;
    const unsigned blocks = (unsigned)((P + kCompactThreads - 1) / kCompactThreads);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_add_count<<<blocks, kCompactThreads, 0, st>>>(L);
    k_add_emit<<<blocks, kCompactThreads, 0, st>>>(L);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_map_adam_step(const gs_map_config *cfg, const gs_map *map, const int64_t *n,
                           const gs_gaussians_grad *grads, int64_t step, void *stream) {
    if (!cfg || !map_ok(map) || !map->adam_state || !n || !grads || step < 1) return GS_ERR_INVALID_ARG;
    if (!(cfg->beta1 >= 0 && cfg->beta1 < 1) || !(cfg->beta2 >= 0 && cfg->beta2 < 1) || !(cfg->eps >= 0))
        return GS_ERR_INVALID_ARG;
    const float *gp[5] = {grads->means, grads->quats, grads->log_scales, grads->opacity_logits, grads->rgb};
    for (const float *q : gp)
        if (q && !aligned16(q)) return GS_ERR_INVALID_ARG;
    const MapView M = view_of(*map);
    const double lr[5] = {cfg->lr_means, cfg->lr_quats, cfg->lr_log_scales, cfg->lr_opacity_logits, cfg->lr_rgb};
    AdamLaunch L{};
    for (int s = 0; s < kGroups; ++s) {
        L.p[s] = M.p[s];
        L.g[s] = gp[s];
        L.lp[s] = M.lp[s];
        L.m[s] = M.state + M.cap * group_offset(s, M.iso);
        L.v[s] = L.m[s] + values_per_gaussian(M.iso) * M.cap;
        L.lr[s] = (float)lr[s];
        L.width[s] = group_width(s, M.iso);
    }
    L.b1 = (float)cfg->beta1;
    L.b2 = (float)cfg->beta2;
    L.omb1 = (float)(1.0 - cfg->beta1);
    L.omb2 = (float)(1.0 - cfg->beta2);
    L.c1 = (float)(1.0 / (1.0 - std::pow(cfg->beta1, (double)step)));
    L.c2 = (float)(1.0 / (1.0 - std::pow(cfg->beta2, (double)step)));
    L.eps = (float)cfg->eps;
    L.lowp_dt = M.lowp_dt;
    L.n = n;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GS_ERR_CUDA;
    // about four resident 256-thread blocks per SM per group; quads beyond a group's
    // live length exit at once
    const int64_t quads = (4 * M.cap + 3) / 4;
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * sms, (quads + 255) / 256));
    k_map_adam<<<dim3(gx, kGroups), 256, 0, static_cast<cudaStream_t>(stream)>>>(L);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_map_prune(const gs_map_config *cfg, const gs_map *src, const int64_t *n_src, const gs_map *dst,
                       int64_t *n_dst, void *scratch, size_t scratch_bytes, void *stream) {
    if (!cfg || !map_ok(src) || !map_ok(dst) || !n_src || !n_dst || !scratch) return GS_ERR_INVALID_ARG;
    if (dst->capacity < src->capacity || src->capacity >= (1ll << 31) || !(cfg->opacity_min > 0.f) ||
        !(cfg->opacity_min < 1.f))
        return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(scratch) & 255u) != 0 || scratch_bytes < scratch_bytes_for(src->capacity))
        return GS_ERR_INVALID_ARG;
    if (src->means == dst->means || (src->quats == nullptr) != (dst->quats == nullptr)) return GS_ERR_INVALID_ARG;
    PruneLaunch L{};
    L.src = view_of(*src);
    L.dst = view_of(*dst);
    L.n_src = n_src;
    L.n_dst = n_dst;
    const double o = (double)cfg->opacity_min;
    L.logit_min = (float)std::log(o / (1.0 - o));
    L.n0 = static_cast<int64_t *>(scratch);
    L.counts = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + kScratchHead);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, (src->capacity + kCompactThreads - 1) / kCompactThreads);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_prune_count<<<blocks, kCompactThreads, 0, st>>>(L);
    k_prune_emit<<<blocks, kCompactThreads, 0, st>>>(L);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
