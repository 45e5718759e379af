// metrics.cu -- image-quality sums of a rendered view against its RGB-D observation, the
// quantities behind the evaluation of Sec. IV (PSNR of the colour, the average depth
// error): one block, FP64 accumulation in a fixed order, so repeated calls agree bit for
// bit.  It reads each pixel once; at 640 x 480 it is a few microseconds.
#include "gs_internal.cuh"

namespace {

constexpr int kMetricThreads = 1024;

__global__ void __launch_bounds__(kMetricThreads) k_image_metrics(const float *rgb, const float *depth,
                                                                 const float *rgb_t, const float *depth_t,
                                                                 int64_t P, double *out) {
    double se = 0.0, ad = 0.0, sd = 0.0, cnt = 0.0;
    for (int64_t p = threadIdx.x; p < P; p += kMetricThreads) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double e = (double)rgb[c * P + p] - (double)rgb_t[c * P + p];
            se += e * e;
        }
        const float dt = depth_t[p];
        if (dt > 0.f) {
            const double e = (double)depth[p] - (double)dt;
            ad += fabs(e);
            sd += e * e;
            cnt += 1.0;
        }
    }
    __shared__ double s[4][kMetricThreads / 32];
    double v[4] = {se, ad, cnt, sd};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) s[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0.0;
        for (int w = 0; w < kMetricThreads / 32; ++w) acc += s[threadIdx.x][w];
        out[threadIdx.x] = acc;
    }
}

}  // namespace

extern "C" gs_status gs_image_metrics(const float *rgb, const float *depth, const float *rgb_t, const float *depth_t,
                                      int64_t pixels, double *out, void *stream) {
    if (!rgb || !depth || !rgb_t || !depth_t || !out || pixels < 1) return GS_ERR_INVALID_ARG;
    k_image_metrics<<<1, kMetricThreads, 0, static_cast<cudaStream_t>(stream)>>>(rgb, depth, rgb_t, depth_t, pixels,
                                                                                   out);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
