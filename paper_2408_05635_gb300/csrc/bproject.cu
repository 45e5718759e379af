// bproject.cu -- chain rule from screen-space gradients to the Gaussian parameters and
// the camera pose, FP64 pose reduction, and the decoupled pose update.
//
// Forward quantities (recomputed): x_c = W m + t, M = W Rg diag(s), Sigma_c = M M^T,
// J = d pi_m / d x_c, N = J M, Sigma' = N N^T + eps I, conic Q = Sigma'^-1.
// Backward, with G = dL/dSigma' = -Q Gq Q (Gq the conic gradient as a symmetric
// matrix):  dN = 2 G N,  dJ = dN M^T,  dM = J^T dN,
//   dx_c = J^T d mu' + e_z d depth + (dJ chained through J(x_c)),
//   d m = W^T dx_c;  dB = W^T dM with B = Rg diag(s): dRg = dB diag(s),
//   d s_j = sum_i dB_ij Rg_ij, d log s = s d s; quaternion through Rg(q / |q|);
//   d logit = o (1 - o) d o.
// Pose, as two decoupled blocks (Sec. III-B): the rotation turns the camera about its
// own centre (x_c <- Exp(theta) x_c, i.e. W <- Exp(theta) W and t <- Exp(theta) t) and the
// translation shifts it (x_c <- x_c + t).  d t = dx_c and
// d theta = x_c x dx_c + axial(dM M^T) with axial(P) = (P21 - P12, P02 - P20, P10 - P01).
// The per-record 6-vectors are summed over the warp in FP32 (at most 32 terms) and over
// the cell's warps in double-float; k_finalize sums the view's cells in a fixed order
// (double-float)
// and, in tracking mode, applies the decoupled Adam step in FP64 (separate moments for
// theta and t; R <- Exp(-step_theta) R, t <- Exp(-step_theta) t - step_t).
#include "gs_internal.cuh"

namespace gsk {

// d loss / d (unit quaternion) from d loss / d Rg, entry by entry of quat_to_rot.
__device__ __forceinline__ void rot_grad_to_quat(float w, float x, float y, float z, const float dR[9], float dq[4]) {
    dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                   2.f * x * dR[8]);
    dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                   2.f * y * dR[8]);
    dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] + x * dR[6] +
                   y * dR[7]);
}

// cos(h) and sin(h) / h for |h| <= 0.1 by their Taylor series through h^8 (the first
// omitted terms, h^10 / 10! and h^10 / 11!, are below 3e-17): the half-angle of a pose
// step is ~1e-3 rad, where FP64 transcendentals are long dependent chains on this GPU.
__device__ __forceinline__ void cos_sinc_small(double h2, double &c, double &sc) {
    c = 1.0 + h2 * (-1.0 / 2 + h2 * (1.0 / 24 + h2 * (-1.0 / 720 + h2 * (1.0 / 40320))));
    sc = 1.0 + h2 * (-1.0 / 6 + h2 * (1.0 / 120 + h2 * (-1.0 / 5040 + h2 * (1.0 / 362880))));
}

// Decoupled Adam step of one view, FP64, writing the new pose and optimiser state to
// `pose_out` / `st_out` (and `res_out`, n x 8 with the loss last, if not NULL).  state:
// m_rot 3, v_rot 3, m_t 3, v_t 3, step count, beta1^k, beta2^k (running products, 0 before
// the first step), 1 unused.  FP64 instructions are slow here (a warp instruction takes
// the FP64 pipe for many cycles whatever its active lanes), so the work is laid out as few
// instructions: the six moment updates in one warp's lanes (one per pose coordinate),
// then the rotation step in warp 0 (lane i: quaternion component i) and the translation
// step in warp 1 (lane i: component i) at the same time, each warp computing the step's
// quaternion itself.  Every thread of the block calls it.
__device__ void adam_update(const double *pose, const double *st, const double *g, double loss, const Settings &S,
                            double *s_step, int tid, double *pose_out, double *st_out, double *res_out) {
    const double p1 = st[12] > 0.0 ? st[13] * S.beta1 : S.beta1;
    const double p2 = st[12] > 0.0 ? st[14] * S.beta2 : S.beta2;
    if (tid < 6) {
        const int im = tid < 3 ? tid : 6 + (tid - 3), iv = im + 3;
        const double m = S.beta1 * st[im] + (1.0 - S.beta1) * g[tid];
        const double v = S.beta2 * st[iv] + (1.0 - S.beta2) * g[tid] * g[tid];
        st_out[im] = m;
        st_out[iv] = v;
        const double lr = tid < 3 ? S.lr_rot : S.lr_trans;
        s_step[tid] = lr * (m / (1.0 - p1)) / (sqrt(v / (1.0 - p2)) + S.eps);
    } else if (tid == 32) {
        st_out[12] = st[12] + 1.0;
        st_out[13] = p1;
        st_out[14] = p2;
        st_out[15] = st[15];
    } else if (tid == 64 && res_out) {
        res_out[7] = loss;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    if (warp > 1) return;
    const double sx = s_step[0], sy = s_step[1], sz = s_step[2];
    const double th2 = sx * sx + sy * sy + sz * sz;
    const double h2 = 0.25 * th2;  // (theta / 2)^2
    double c, sinc;
    if (h2 <= 0.01) {
        cos_sinc_small(h2, c, sinc);
    } else {
        const double h = sqrt(h2);
        c = cos(h);
        sinc = sin(h) / h;
    }
    // quaternion of Exp(-step): (cos(theta/2), -step sin(theta/2) / theta), sin(h)/theta = sinc(h)/2
    const double a0 = c, a1 = -0.5 * sinc * sx, a2 = -0.5 * sinc * sy, a3 = -0.5 * sinc * sz;
    if (warp == 0) {
        // R <- Exp(-step) R: Hamilton product a (x) pose, component i = lane (0..3) as
        // a0 b_i + a1 x1 + a2 x2 + a3 x3 with signed, permuted components x of b
        const int i = lane & 3;
        const double b0 = pose[0], b1 = pose[1], b2 = pose[2], b3 = pose[3];
        const double bi = i == 0 ? b0 : (i == 1 ? b1 : (i == 2 ? b2 : b3));
        const double x1 = i == 0 ? -b1 : (i == 1 ? b0 : (i == 2 ? -b3 : b2));
        const double x2 = i == 0 ? -b2 : (i == 1 ? b3 : (i == 2 ? b0 : -b1));
        const double x3 = i == 0 ? -b3 : (i == 1 ? -b2 : (i == 2 ? b1 : b0));
        const double q = a0 * bi + a1 * x1 + a2 * x2 + a3 * x3;
        double n2 = q * q;
        n2 += __shfl_xor_sync(0xffffffffu, n2, 1);
        n2 += __shfl_xor_sync(0xffffffffu, n2, 2);
        const double qn = q * rsqrt(n2);
        if (lane < 4) {
            pose_out[lane] = qn;
            if (res_out) res_out[lane] = qn;
        }
    } else {
        // the camera turns about its own centre: t <- Exp(-step) t - step_t, component i =
        // lane (0..2), with Exp(-step) t = t + 2 a0 (a_v x t) + 2 a_v x (a_v x t) for the unit
        // quaternion a = (a0, a_v)
        const int i = lane < 3 ? lane : 0;
        const double t0 = pose[4], t1 = pose[5], t2 = pose[6];
        const double u0 = a2 * t2 - a3 * t1, u1 = a3 * t0 - a1 * t2, u2 = a1 * t1 - a2 * t0;
        const double w0 = a2 * u2 - a3 * u1, w1 = a3 * u0 - a1 * u2, w2 = a1 * u1 - a2 * u0;
        const double ti = i == 0 ? t0 : (i == 1 ? t1 : t2);
        const double ui = i == 0 ? u0 : (i == 1 ? u1 : u2);
        const double wi = i == 0 ? w0 : (i == 1 ? w1 : w2);
        const double tn = ti + 2.0 * (a0 * ui + wi) - s_step[3 + i];
        if (lane < 3) {
            pose_out[4 + lane] = tn;
            if (res_out) res_out[4 + lane] = tn;
        }
    }
}

// Butterfly reduce-scatter of 8 values over the warp (9 shuffles); afterwards lanes with
// (lane & 3) == 0 hold the full warp sum of value `idx`.
__device__ __forceinline__ float warp_reduce8(float (&v)[8], int lane, int &idx) {
    idx = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int mask = 16 >> s, w = 4 >> s;
        const bool up = (lane & mask) != 0;
#pragma unroll
        for (int k = 0; k < w; ++k) {
            const float send = up ? v[k] : v[k + w];
            const float keep = up ? v[k + w] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
        }
        if (up) idx += w;
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}

// One block per cell, one thread per record of the cell.  ISO: isotropic Gaussians (Eq. 1
// as written: one log-radius per Gaussian, no rotation), Sigma_c = s^2 I.
template <int DT, bool PARAMS, bool ISO>
__global__ void __launch_bounds__(kBlock, PARAMS ? 4 : 6) k_bproject(BprojLaunch L) {
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ float s_red[kWarps][8];
    const uint32_t cell = blockIdx.x;
    const uint32_t cnt = L.ws.cell_cnt[cell];
    const int view = (int)(cell / (uint32_t)L.d.nblk);
    float p6[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if ((uint32_t)tid < cnt) {
        const uint32_t rec = cell * kCell + (uint32_t)tid;
        const Rec rr = L.ws.rec[rec];
        const RecGrad gg = L.ws.rec_grad[rec];
        const uint32_t gv = __float_as_uint(rr.c.w);
        const int64_t i = (int64_t)((uint64_t)gv % (uint64_t)L.d.n);
        const ViewInfo vi = L.ws.views[view];
        float sRt[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) sRt[k] = __ldg(L.ws.view_rt + 12 * view + k);
        const float4 Bq = rr.b;  // conic the compositors used
        const float mx = __ldg(L.g.means + 3 * i), my = __ldg(L.g.means + 3 * i + 1), mz = __ldg(L.g.means + 3 * i + 2);
        const float x = cam_coord(sRt, 0, mx, my, mz);
        const float y = cam_coord(sRt, 1, mx, my, mz);
        const float z = cam_coord(sRt, 2, mx, my, mz);
        float w = 1.f, qx = 0.f, qy = 0.f, qz = 0.f, qinv = 1.f;
        float Rg[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
        float s[3];
        if constexpr (ISO) {
            s[0] = s[1] = s[2] = expf(ld_attr<DT>(L.g.log_scales, i));
        } else {
            const float q0 = ld_attr<DT>(L.g.quats, 4 * i), q1 = ld_attr<DT>(L.g.quats, 4 * i + 1);
            const float q2 = ld_attr<DT>(L.g.quats, 4 * i + 2), q3 = ld_attr<DT>(L.g.quats, 4 * i + 3);
            const float qn2 = q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3;
            qinv = rsqrtf(qn2);
            w = q0 * qinv;
            qx = q1 * qinv;
            qy = q2 * qinv;
            qz = q3 * qinv;
            quat_to_rot(w, qx, qy, qz, Rg);
            s[0] = expf(ld_attr<DT>(L.g.log_scales, 3 * i));
            s[1] = expf(ld_attr<DT>(L.g.log_scales, 3 * i + 1));
            s[2] = expf(ld_attr<DT>(L.g.log_scales, 3 * i + 2));
        }
        float Bm[9], M[9];  // B = Rg diag(s), M = W B
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Bm[3 * r + c] = Rg[3 * r + c] * s[c];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                M[3 * r + c] = sRt[3 * r] * Bm[c] + sRt[3 * r + 1] * Bm[3 + c] + sRt[3 * r + 2] * Bm[6 + c];
        const float iz = 1.f / z, iz2 = iz * iz;
        // J as the projection took it: tangent clamped to the view's limits
        const float txr = x * iz, tyr = y * iz;
        const float tx = fminf(fmaxf(txr, -vi.tan_lim_x), vi.tan_lim_x);
        const float ty = fminf(fmaxf(tyr, -vi.tan_lim_y), vi.tan_lim_y);
        const bool free_x = tx == txr, free_y = ty == tyr;
        const float J00 = vi.fx * iz, J02 = -vi.fx * tx * iz;
        const float J11 = vi.fy * iz, J12 = -vi.fy * ty * iz;
        float N0[3], N1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            N0[c] = J00 * M[c] + J02 * M[6 + c];
            N1[c] = J11 * M[3 + c] + J12 * M[6 + c];
        }
        // G = -Q Gq Q with Gq = [[da, db/2], [db/2, dc]] and Q = [[a, b], [b, c]]
        const float qa = Bq.x, qb = Bq.y, qc = Bq.z;
        const float ga = gg.g1.x, gb = 0.5f * gg.g1.y, gc = gg.g1.z;
        const float t00 = qa * ga + qb * gb, t01 = qa * gb + qb * gc;
        const float t10 = qb * ga + qc * gb, t11 = qb * gb + qc * gc;
        const float G00 = -(t00 * qa + t01 * qb), G01 = -(t00 * qb + t01 * qc), G11 = -(t10 * qb + t11 * qc);
        float dN0[3], dN1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dN0[c] = 2.f * (G00 * N0[c] + G01 * N1[c]);
            dN1[c] = 2.f * (G01 * N0[c] + G11 * N1[c]);
        }
        // dJ = dN M^T (only J00, J02, J11, J12 are variables); dM = J^T dN
        const float dJ00 = dN0[0] * M[0] + dN0[1] * M[1] + dN0[2] * M[2];
        const float dJ02 = dN0[0] * M[6] + dN0[1] * M[7] + dN0[2] * M[8];
        const float dJ11 = dN1[0] * M[3] + dN1[1] * M[4] + dN1[2] * M[5];
        const float dJ12 = dN1[0] * M[6] + dN1[1] * M[7] + dN1[2] * M[8];
        float dM[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dM[c] = J00 * dN0[c];
            dM[3 + c] = J11 * dN1[c];
            dM[6 + c] = J02 * dN0[c] + J12 * dN1[c];
        }
        const float dmu_x = gg.g0.x, dmu_y = gg.g0.y, dd = gg.g0.z;
        const float fx = vi.fx, fy = vi.fy;
        // d mu' / d x_c is the unclamped (f / z, -f x / z^2); J02 = -fx t_x / z passes
        // dJ02/dx = -fx / z^2 and dJ02/dz = fx (t_x + x / z) / z^2 where t_x is free, and
        // only dJ02/dz = fx t_x / z^2 where it is clamped (J12 likewise)
        const float dxc0 = dmu_x * J00 - (free_x ? dJ02 * fx * iz2 : 0.f);
        const float dxc1 = dmu_y * J11 - (free_y ? dJ12 * fy * iz2 : 0.f);
        const float dxc2 = -(dmu_x * fx * txr + dmu_y * fy * tyr) * iz + dd - dJ00 * fx * iz2 +
                           dJ02 * fx * iz2 * (tx + (free_x ? txr : 0.f)) - dJ11 * fy * iz2 +
                           dJ12 * fy * iz2 * (ty + (free_y ? tyr : 0.f));
        if (L.want_pose) {
            // translation, and rotation about the camera centre (mean and covariance parts)
            float P[9];  // dM M^T
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    P[3 * r + c] = dM[3 * r] * M[3 * c] + dM[3 * r + 1] * M[3 * c + 1] + dM[3 * r + 2] * M[3 * c + 2];
            p6[0] = y * dxc2 - z * dxc1 + (P[7] - P[5]);
            p6[1] = z * dxc0 - x * dxc2 + (P[2] - P[6]);
            p6[2] = x * dxc1 - y * dxc0 + (P[3] - P[1]);
            p6[3] = dxc0;
            p6[4] = dxc1;
            p6[5] = dxc2;
        }
        if constexpr (PARAMS) {
            const gs_gaussians_grad &G = L.grads;
            if (G.means) {
                atomicAdd(G.means + 3 * i, sRt[0] * dxc0 + sRt[3] * dxc1 + sRt[6] * dxc2);
                atomicAdd(G.means + 3 * i + 1, sRt[1] * dxc0 + sRt[4] * dxc1 + sRt[7] * dxc2);
                atomicAdd(G.means + 3 * i + 2, sRt[2] * dxc0 + sRt[5] * dxc1 + sRt[8] * dxc2);
            }
            if (G.quats || G.log_scales) {
                float dB[9];  // W^T dM
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        dB[3 * r + c] = sRt[r] * dM[c] + sRt[3 + r] * dM[3 + c] + sRt[6 + r] * dM[6 + c];
                if (G.log_scales) {
                    if constexpr (ISO) {
                        // one radius drives all three axes: d log s = s trace(W^T dM)
                        atomicAdd(G.log_scales + i, (dB[0] + dB[4] + dB[8]) * s[0]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float ds = dB[c] * Rg[c] + dB[3 + c] * Rg[3 + c] + dB[6 + c] * Rg[6 + c];
                            atomicAdd(G.log_scales + 3 * i + c, ds * s[c]);
                        }
                    }
                }
                if (!ISO && G.quats) {
                    float dRg[9];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) dRg[3 * r + c] = dB[3 * r + c] * s[c];
                    float dqn[4];
                    rot_grad_to_quat(w, qx, qy, qz, dRg, dqn);
                    const float pr = dqn[0] * w + dqn[1] * qx + dqn[2] * qy + dqn[3] * qz;
                    atomicAdd(G.quats + 4 * i, (dqn[0] - w * pr) * qinv);
                    atomicAdd(G.quats + 4 * i + 1, (dqn[1] - qx * pr) * qinv);
                    atomicAdd(G.quats + 4 * i + 2, (dqn[2] - qy * pr) * qinv);
                    atomicAdd(G.quats + 4 * i + 3, (dqn[3] - qz * pr) * qinv);
                }
            }
            if (G.opacity_logits) {
                const float o = rr.a.w;
                atomicAdd(G.opacity_logits + i, gg.g0.w * o * (1.f - o));
            }
            if (G.rgb) {
                atomicAdd(G.rgb + 3 * i, gg.g2.x);
                atomicAdd(G.rgb + 3 * i + 1, gg.g2.y);
                atomicAdd(G.rgb + 3 * i + 2, gg.g2.z);
            }
        }
    }
    if (!L.want_pose) return;  // uniform across the grid
    // cell sum: FP32 over the warp (at most 32 terms), then FP64 over the warps
    int slot;
    const float sum = warp_reduce8(p6, lane, slot);
    if ((lane & 3) == 0 && slot < 6) s_red[warp][slot] = sum;
    __syncthreads();
    if (tid < 6) {
        DF acc{0.f, 0.f};
        for (int w = 0; w < kWarps; ++w) acc = df_add(acc, DF{s_red[w][tid], 0.f});
        L.ws.pose_part[(size_t)cell * 6 + tid] = df_pack(acc);
    }
}

// One block per view: fixed-order double-float sums of the view's tile losses and cell
// pose partials, then (tracking) the decoupled Adam step in FP64.  The kernel is a chain
// of dependent steps, so every global load is issued as early as possible: the pose and
// the optimiser state first, then kFinUnroll partials per thread per round.  A cell's six
// partials are read as three 16-byte pairs; with a thread count divisible by three every
// thread always holds the same pair of components.  The block's partials are summed per
// component by one warp (strided columns, then a butterfly).
constexpr int kFinThreads = 384;
constexpr int kFinUnroll = 8;

__global__ void __launch_bounds__(kFinThreads) k_finalize(FinalizeLaunch L) {
    griddep_wait();  // the predecessor's results are visible from here on
    griddep_launch_dependents();
    const int v = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kPerComp = kFinThreads / 3;  // pose partial columns per component
    __shared__ float2 s_pose_acc[6][kPerComp];
    __shared__ float2 s_loss_acc[kFinThreads];
    __shared__ double s_g[7], s_step[6], s_pose[7], s_st[16];
    const bool adam = L.pose && L.poses;
    if (adam) {
        if (tid < 7)
            s_pose[tid] = L.poses[7 * v + tid];
        else if (tid >= 32 && tid < 48)
            s_st[tid - 32] = L.adam[16 * v + tid - 32];
    }
    DF lacc{0.f, 0.f}, pa{0.f, 0.f}, pb{0.f, 0.f};  // loss; components 2 (tid % 3), 2 (tid % 3) + 1
    if (L.loss_out || L.host_result) {
        const ViewInfo vi = L.ws.views[v];
        const uint32_t nt = (uint32_t)vi.tiles_x * (uint32_t)vi.tiles_y;
        const float2 *tl = L.ws.tile_loss + vi.tile_base;
        for (uint32_t b = 0; b < nt; b += kFinThreads * kFinUnroll) {
            float2 x[kFinUnroll];
#pragma unroll
            for (int k = 0; k < kFinUnroll; ++k) {
                const uint32_t t = b + (uint32_t)(k * kFinThreads + tid);
                x[k] = t < nt ? tl[t] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < kFinUnroll; ++k) lacc = df_add(lacc, df_load(x[k]));
        }
    }
    if (L.pose) {
        const size_t nq = (size_t)L.d.nblk * 3;  // 16-byte pairs of the view
        const float4 *pp = reinterpret_cast<const float4 *>(L.ws.pose_part + (size_t)v * (size_t)L.d.nblk * 6);
        for (size_t b = 0; b < nq; b += kFinThreads * kFinUnroll) {
            float4 x[kFinUnroll];
#pragma unroll
            for (int k = 0; k < kFinUnroll; ++k) {
                const size_t q = b + (size_t)(k * kFinThreads + tid);
                x[k] = q < nq ? pp[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < kFinUnroll; ++k) {
                pa = df_add(pa, DF{x[k].x, x[k].y});
                pb = df_add(pb, DF{x[k].z, x[k].w});
            }
        }
    }
    s_loss_acc[tid] = df_pack(lacc);
    s_pose_acc[2 * (tid % 3)][tid / 3] = df_pack(pa);
    s_pose_acc[2 * (tid % 3) + 1][tid / 3] = df_pack(pb);
    __syncthreads();
    if (warp < 7) {
        DF t{0.f, 0.f};
        if (warp < 6)
            for (int i = lane; i < kPerComp; i += 32) t = df_add(t, df_load(s_pose_acc[warp][i]));
        else
            for (int i = lane; i < kFinThreads; i += 32) t = df_add(t, df_load(s_loss_acc[i]));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t = df_add(t, df_shfl_xor(t, off));
        if (lane == 0) {
            const double g = (double)t.hi + (double)t.lo;
            s_g[warp] = g;
            if (warp == 6 && L.loss_out) L.loss_out[v] = g;
            if (warp < 6 && L.pose && L.pose_grad) L.pose_grad[6 * v + warp] = g;
        }
    }
    __syncthreads();
    if (!adam) return;
    // the new pose and state straight to their arrays (and into host memory: no copy after
    // the kernel)
    adam_update(s_pose, s_st, s_g, s_g[6], L.s, s_step, tid, L.poses + 7 * v, L.adam + 16 * v,
                L.host_result ? L.host_result + 8 * v : nullptr);
}

cudaError_t launch_finalize(const FinalizeLaunch &L, cudaStream_t st) {
    cudaError_t e = launch_dep(k_finalize, dim3(L.d.V), dim3(kFinThreads), st, L);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_bproject(const BprojLaunch &L, cudaStream_t st) {
    const uint32_t grid = (uint32_t)L.d.V * (uint32_t)L.d.nblk;
    const bool params = L.grads.means || L.grads.quats || L.grads.log_scales || L.grads.opacity_logits || L.grads.rgb;
    const bool iso = L.g.quats == nullptr;
    cudaError_t e;
#define GS_BPROJ(DT)                                                   \
    if (params && iso)                                                 \
        e = launch_dep(k_bproject<DT, true, true>, grid, dim3(kBlock), st, L);        \
    else if (params)                                                   \
        e = launch_dep(k_bproject<DT, true, false>, grid, dim3(kBlock), st, L);       \
    else if (iso)                                                      \
        e = launch_dep(k_bproject<DT, false, true>, grid, dim3(kBlock), st, L);       \
    else                                                               \
        e = launch_dep(k_bproject<DT, false, false>, grid, dim3(kBlock), st, L);
    switch (L.dtype) {
        case GS_F32: GS_BPROJ(GS_F32) break;
        case GS_BF16: GS_BPROJ(GS_BF16) break;
        case GS_F16: GS_BPROJ(GS_F16) break;
        default: return cudaErrorInvalidValue;
    }
#undef GS_BPROJ
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace gsk
