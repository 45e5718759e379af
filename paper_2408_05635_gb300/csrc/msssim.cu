// msssim.cu -- multi-scale structural similarity (Wang, Simoncelli and Bovik, 2003) of a
// rendered colour image against its observation, the image-quality measure of Sec. IV.
//
// Per scale and channel, one thread per valid window position computes the local
// statistics under the 11 x 11 Gaussian window (sigma 1.5) directly, centred on the
// window's middle pixel so that the variances do not cancel in FP32, and each block
// adds its l and cs terms in FP64.  A one-block pass sums the block partials in a fixed
// order; 2 x 2 average pooling makes the next scale.  The last launch combines the
// scales with the published exponents.  This is an evaluation pass, not the tracking
// path: about 20 small launches at 640 x 480.
#include <algorithm>
#include <cmath>

#include "gs_internal.cuh"

namespace {

constexpr int kWin = 11;
constexpr int kScales = 5;
constexpr int kSsimThreads = 256;
constexpr int kRedThreads = 512;
struct Window {
    float g[kWin];  // the normalised 1-D Gaussian (sigma 1.5); the 2-D window is its outer product
};
struct Weights {
    double b[kScales];  // published scale exponents
};

struct Level {
    const float *x, *y;  // 3 planes each, w x h
    int w, h;
};

// Terms of one scale: blockIdx.z = channel; partials[(z * nblk + block) * 2 + {0, 1}] =
// sums of l and cs over the block's window positions.
__global__ void __launch_bounds__(kSsimThreads) k_ssim_terms(Level L, Window W, double *partials, int nblk) {
    const int ow = L.w - kWin + 1, oh = L.h - kWin + 1;
    const int ch = blockIdx.z;
    const int64_t o = (int64_t)blockIdx.x * kSsimThreads + threadIdx.x;
    double l = 0.0, cs = 0.0;
    if (o < (int64_t)ow * oh) {
        const int oy = (int)(o / ow), ox = (int)(o % ow);
        const float *X = L.x + (int64_t)ch * L.w * L.h, *Y = L.y + (int64_t)ch * L.w * L.h;
        const int64_t c0 = (int64_t)(oy + kWin / 2) * L.w + ox + kWin / 2;
        const float cx = X[c0], cy = Y[c0];
        float sx = 0.f, sy = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
        for (int i = 0; i < kWin; ++i) {
            const float *xr = X + (int64_t)(oy + i) * L.w + ox, *yr = Y + (int64_t)(oy + i) * L.w + ox;
            float rx = 0.f, ry = 0.f, rxx = 0.f, ryy = 0.f, rxy = 0.f;
#pragma unroll
            for (int j = 0; j < kWin; ++j) {
                const float a = xr[j] - cx, b = yr[j] - cy, w = W.g[j];
                rx = fmaf(w, a, rx);
                ry = fmaf(w, b, ry);
                rxx = fmaf(w * a, a, rxx);
                ryy = fmaf(w * b, b, ryy);
                rxy = fmaf(w * a, b, rxy);
            }
            const float wi = W.g[i];
            sx = fmaf(wi, rx, sx);
            sy = fmaf(wi, ry, sy);
            sxx = fmaf(wi, rxx, sxx);
            syy = fmaf(wi, ryy, syy);
            sxy = fmaf(wi, rxy, sxy);
        }
        // shifted moments: variances and covariance do not depend on the shift
        const double mx = (double)cx + sx, my = (double)cy + sy;
        const double vx = (double)sxx - (double)sx * sx, vy = (double)syy - (double)sy * sy;
        const double cxy = (double)sxy - (double)sx * sy;
        const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
        l = (2.0 * mx * my + C1) / (mx * mx + my * my + C1);
        cs = (2.0 * cxy + C2) / (vx + vy + C2);
    }
    __shared__ double s[2][kSsimThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        l += __shfl_xor_sync(0xffffffffu, l, off);
        cs += __shfl_xor_sync(0xffffffffu, cs, off);
    }
    if ((threadIdx.x & 31) == 0) {
        s[0][threadIdx.x >> 5] = l;
        s[1][threadIdx.x >> 5] = cs;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double acc = 0.0;
        for (int w = 0; w < kSsimThreads / 32; ++w) acc += s[threadIdx.x][w];
        partials[((int64_t)ch * nblk + blockIdx.x) * 2 + threadIdx.x] = acc;
    }
}

// Means of the scale's terms per channel: terms[(scale * 3 + ch) * 2 + {0, 1}].
__global__ void __launch_bounds__(kRedThreads) k_ssim_reduce(const double *partials, int nblk, int64_t count,
                                                             double *terms, int scale) {
    const int ch = blockIdx.x;
    double l = 0.0, cs = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kRedThreads) {
        l += partials[((int64_t)ch * nblk + b) * 2];
        cs += partials[((int64_t)ch * nblk + b) * 2 + 1];
    }
    __shared__ double s[2][kRedThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        l += __shfl_xor_sync(0xffffffffu, l, off);
        cs += __shfl_xor_sync(0xffffffffu, cs, off);
    }
    if ((threadIdx.x & 31) == 0) {
        s[0][threadIdx.x >> 5] = l;
        s[1][threadIdx.x >> 5] = cs;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double acc = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) acc += s[threadIdx.x][w];
        terms[(scale * 3 + ch) * 2 + threadIdx.x] = acc / (double)count;
    }
}

// 2 x 2 average pooling of both images' three planes (odd last rows / columns dropped).
__global__ void k_pool2(Level in, float *x, float *y) {
    const int w = in.w / 2, h = in.h / 2;
    const int64_t n = (int64_t)3 * w * h;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(k / ((int64_t)w * h));
        const int64_t r = k - (int64_t)ch * w * h;
        const int py = (int)(r / w), px = (int)(r % w);
        const int64_t base = (int64_t)ch * in.w * in.h + (int64_t)(2 * py) * in.w + 2 * px;
        x[k] = 0.25f * ((in.x[base] + in.x[base + in.w]) + (in.x[base + 1] + in.x[base + in.w + 1]));
        y[k] = 0.25f * ((in.y[base] + in.y[base + in.w]) + (in.y[base + 1] + in.y[base + in.w + 1]));
    }
}

// out[1 + ch] = l_5^b5 prod_j max(cs_j, 0)^bj per channel, out[0] = their mean.
__global__ void k_msssim_combine(const double *terms, Weights B, double *out) {
    if (threadIdx.x != 0) return;
    double mean = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        double v = 1.0;
        for (int j = 0; j < kScales; ++j) {
            v *= pow(fmax(terms[(j * 3 + ch) * 2 + 1], 0.0), B.b[j]);
            if (j == kScales - 1) v *= pow(fmax(terms[(j * 3 + ch) * 2], 0.0), B.b[j]);
        }
        out[1 + ch] = v;
        mean += v;
    }
    out[0] = mean / 3.0;
}

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

size_t scratch_layout(int W, int H, size_t *pyr_bytes, size_t *part_bytes) {
    size_t pyr = 0;
    int w = W, h = H;
    for (int j = 1; j < kScales; ++j) {
        w /= 2;
        h /= 2;
        pyr += align256(2 * 3 * (size_t)w * h * sizeof(float));
    }
    const int64_t ow = W - kWin + 1, oh = H - kWin + 1;
    const int64_t nblk = (ow * oh + kSsimThreads - 1) / kSsimThreads;
    const size_t part = align256((size_t)3 * nblk * 2 * sizeof(double));
    *pyr_bytes = pyr;
    *part_bytes = part;
    return pyr + part + align256(kScales * 3 * 2 * sizeof(double));
}

}  // namespace

extern "C" {

size_t gs_msssim_scratch_bytes(int32_t width, int32_t height) {
    if (width < 1 || height < 1) return 0;
    size_t a, b;
    return scratch_layout(width, height, &a, &b);
}

gs_status gs_msssim(const float *rgb, const float *rgb_t, int32_t width, int32_t height, double *out, void *scratch,
                    size_t scratch_bytes, void *stream) {
    if (!rgb || !rgb_t || !out || !scratch) return GS_ERR_INVALID_ARG;
    // the coarsest scale (1/16) must still hold one 11 x 11 window
    if (width < 16 * kWin || height < 16 * kWin || (int64_t)width * height >= (1ll << 31)) return GS_ERR_INVALID_ARG;
    size_t pyr, part;
    const size_t need = scratch_layout(width, height, &pyr, &part);
    if (scratch_bytes < need || (reinterpret_cast<uintptr_t>(scratch) & 255u) != 0) return GS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Window win;
    {
        double sum = 0.0, gd[kWin];
        for (int i = 0; i < kWin; ++i) {
            const double x = i - (kWin - 1) / 2.0;
            gd[i] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
            sum += gd[i];
        }
        for (int i = 0; i < kWin; ++i) win.g[i] = (float)(gd[i] / sum);
    }
    const Weights wts{{0.0448, 0.2856, 0.3001, 0.2363, 0.1333}};
    char *base = static_cast<char *>(scratch);
    double *partials = reinterpret_cast<double *>(base + pyr);
    double *terms = reinterpret_cast<double *>(base + pyr + part);
    Level L{rgb, rgb_t, width, height};
    size_t off = 0;
    for (int j = 0; j < kScales; ++j) {
        const int64_t ow = L.w - kWin + 1, oh = L.h - kWin + 1;
        const int nblk = (int)((ow * oh + kSsimThreads - 1) / kSsimThreads);
        k_ssim_terms<<<dim3(nblk, 1, 3), kSsimThreads, 0, st>>>(L, win, partials, nblk);
        k_ssim_reduce<<<3, kRedThreads, 0, st>>>(partials, nblk, ow * oh, terms, j);
        if (j + 1 < kScales) {
            const int w = L.w / 2, h = L.h / 2;
            float *x = reinterpret_cast<float *>(base + off);
            float *y = x + (size_t)3 * w * h;
            off += align256(2 * 3 * (size_t)w * h * sizeof(float));
            const int64_t n = (int64_t)3 * w * h;
            k_pool2<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(L, x, y);
            L = Level{x, y, w, h};
        }
    }
    k_msssim_combine<<<1, 32, 0, st>>>(terms, wts, out);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
