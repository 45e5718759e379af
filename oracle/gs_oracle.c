/*
 * gs_oracle.c -- plain FP64 CPU oracle for the differentiable 3D-Gaussian rasterizer
 * of "Visual SLAM with 3D Gaussian Primitives and Depth Priors Enabling Novel View
 * Synthesis" (arXiv 2408.05635).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it. The product path (the CUDA library)
 * neither links nor calls it, and it shares no code, header or constant with it.
 *
 * What it computes, step by step and in the paper's order:
 *   1. Projection of every Gaussian (Sec. II-A pinhole pi_m with the world->camera
 *      pose R_{c,w}, t_{c,w}; the anisotropic covariance Sigma = R s s^T R^T and the
 *      screen-space covariance Sigma' = J W Sigma W^T J^T written in the source of
 *      Sec. I).  The footprint of Gaussian i at pixel p is the 2-D form of Eq. 1:
 *      f_i(p) = o_i exp(-1/2 (p - mu'_i)^T Sigma'^-1 (p - mu'_i)).
 *   2. Per pixel, every surviving Gaussian in ascending (depth, index) order,
 *      composited front to back: Eq. 2 (colour), Eq. 3 (depth, d_i = camera-frame
 *      depth of the mean) and Eq. 4 (silhouette).
 *   3. The combined tracking loss of Sec. III-B (photometric + depth + visibility)
 *      plus the depth-prior regulariser (Sec. I contributions, Sec. V).
 *   4. Hand-derived gradients of that loss w.r.t. every Gaussian parameter and the
 *      camera pose, as two decoupled blocks: a rotation of the camera about its own
 *      centre (camera-frame points x_c <- Exp(theta) x_c) and a translation
 *      (x_c <- x_c + t).
 *   5. The decoupled rotation / translation update (Sec. III-B): one Adam state per
 *      block; R <- Exp(-step) R and t <- Exp(-step) t (the camera centre stays), then
 *      t <- t - step_t.
 *
 * Readings where the paper is silent (all passed in og_params, none hard-wired):
 *   alpha = min(alpha_max, f_i(p)); a Gaussian with alpha < alpha_min is skipped; the
 *   walk stops before the Gaussian whose inclusion would drop the transmittance below
 *   t_min; background is 0 for C, D and S; pixel (u, v) is sampled at integer (u, v);
 *   Gaussians with camera depth <= z_near are dropped; an optional dilation eps*I is
 *   added to Sigma'; the Jacobian J of Sigma' is taken at the mean's image-plane
 *   tangent (x_c / z, y_c / z) clamped to +-jac_clip times the half-extent of the view
 *   (W / 2 fx, H / 2 fy), as the 3DGS rasterizer the paper builds on (SplaTAM's) does:
 *   the local affine approximation is meaningless for a mean far outside the view, and
 *   unclamped it blows a Gaussian just beyond the near plane up into a footprint of
 *   thousands of pixels.  A clamped coordinate passes no gradient through J; the
 *   screen mean itself is never clamped.
 *
 * Two compositing modes give the same numbers by construction: brute force (every
 * pixel walks every surviving Gaussian) and culled (every pixel walks only the
 * Gaussians whose opacity-aware bounding box covers it; a Gaussian outside that box
 * has alpha < alpha_min there, so skipping it changes nothing).  A test checks the two
 * agree bit for bit.
 *
 * Depth order: the order of Eqs. 2-4 and the near-plane test are decided on an
 * exactly specified FP32 depth key (depth_key below), the precision of the GPU kernels,
 * so both implementations sort identically; all arithmetic stays FP64.
 *
 * Ambiguity mask: where FP32 and FP64 may legitimately take a different discrete
 * decision (alpha near alpha_min or alpha_max, transmittance near t_min, silhouette
 * near the loss threshold, an L1 residual near zero) the pixel is flagged so that
 * parity tests compare only unambiguous pixels.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Unit roundoff of IEEE binary32 (2^-24): the FP32 renderer's relative rounding. */
#define OG_FP32_ROUNDOFF 5.9604644775390625e-8

#define OG_OK 0
#define OG_ERR_ARG 1
#define OG_ERR_OOM 2

typedef struct {
    double fx, fy, cx, cy;
    int32_t width, height;
} og_camera;

typedef struct {
    double alpha_min, alpha_max, t_min, dilation, z_near, jac_clip, sil_thresh;
    double w_rgb, w_depth, w_vis, w_prior;
    double beta1, beta2, eps, lr_rot, lr_trans;
    double amb_alpha, amb_t, amb_sil, amb_resid, amb_effect;
    int32_t brute_force, n_threads;
} og_params;

typedef struct {
    int64_t n;
    const double *means;      /* n x 3, world frame */
    const double *quats;      /* n x 4, (w, x, y, z), need not be unit */
    const double *log_scales; /* n x 3 */
    const double *logits;     /* n, opacity o = sigmoid(logit) */
    const double *rgb;        /* n x 3 */
} og_scene;

typedef struct {
    int cand;          /* survives the near plane and has det(Sigma') > 0 */
    float zkey;        /* FP32 depth key that orders the Gaussians (see depth_key) */
    int onimage;       /* opacity-aware bounding box meets the image */
    double xc[3];      /* camera-frame mean */
    double mu[2];      /* pixel-space mean */
    double cov2[3];    /* Sigma' entries (A, B, C) = [[A, B], [B, C]] */
    double conic[3];   /* Sigma'^-1 entries (a, b, c) */
    double o;          /* opacity */
    double dmax2;      /* largest Mahalanobis^2 with o exp(-d2/2) >= alpha_min */
    double dmu;        /* bound of an FP32 renderer's screen-mean error from its camera transform */
    int x0, x1, y0, y1;/* inclusive pixel box, clamped to the image */
} og_proj;

typedef struct {
    int64_t g;
    double alpha, T, G;
    int clamped;
} og_contrib;

/* ------------------------------------------------------------------ small algebra */

/* Rotation matrix of a unit quaternion (w, x, y, z), row-major. */
static void quat_to_rot(const double q[4], double R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* d(loss)/d(unit quaternion) from d(loss)/dR, differentiating quat_to_rot entry by entry. */
static void rot_grad_to_quat(const double q[4], const double dR[9], double dq[4]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    dq[0] = -2 * z * dR[1] + 2 * y * dR[2] + 2 * z * dR[3] - 2 * x * dR[5] - 2 * y * dR[6] + 2 * x * dR[7];
    dq[1] = 2 * y * dR[1] + 2 * z * dR[2] + 2 * y * dR[3] - 4 * x * dR[4] - 2 * w * dR[5] + 2 * z * dR[6] +
            2 * w * dR[7] - 4 * x * dR[8];
    dq[2] = -4 * y * dR[0] + 2 * x * dR[1] + 2 * w * dR[2] + 2 * x * dR[3] + 2 * z * dR[5] - 2 * w * dR[6] +
            2 * z * dR[7] - 4 * y * dR[8];
    dq[3] = -4 * z * dR[0] - 2 * w * dR[1] + 2 * x * dR[2] + 2 * w * dR[3] - 4 * z * dR[4] + 2 * y * dR[5] +
            2 * x * dR[6] + 2 * y * dR[7];
}

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void mat3_transpose(const double A[9], double T[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * j + i] = A[3 * i + j];
}

static void pose_unpack(const double pose[7], double R[9], double t[3], double qn[4]) {
    double nq = sqrt(pose[0] * pose[0] + pose[1] * pose[1] + pose[2] * pose[2] + pose[3] * pose[3]);
    for (int k = 0; k < 4; ++k) qn[k] = pose[k] / nq;
    quat_to_rot(qn, R);
    t[0] = pose[4];
    t[1] = pose[5];
    t[2] = pose[6];
}

/* The front-to-back order of Eqs. 2-4 is a discrete decision taken by floating point,
 * so it is taken in the precision of the GPU kernels, on an exactly specified FP32 key:
 * the pose quaternion and translation are rounded to FP32, |q|^2 is summed left to
 * right, q is divided by the correctly rounded sqrt(|q|^2), the rotation entries are
 * formed with every FP32 operation rounded (no contraction), and the camera depth of
 * mean m is fmaf(R20, m0, fmaf(R21, m1, fmaf(R22, m2, t2))).  The near-plane test uses
 * the same key.  Everything else (mu', Sigma', the depth d_i of Eq. 3) stays FP64. */
static void pose_rot_f32(const double pose[7], float Rf[9], float tf[3]) {
    float w = (float)pose[0], x = (float)pose[1], y = (float)pose[2], z = (float)pose[3];
    const float nrm = sqrtf(((w * w + x * x) + y * y) + z * z);
    w = w / nrm;
    x = x / nrm;
    y = y / nrm;
    z = z / nrm;
    Rf[0] = 1.0f - 2.0f * (y * y + z * z);
    Rf[1] = 2.0f * (x * y - w * z);
    Rf[2] = 2.0f * (x * z + w * y);
    Rf[3] = 2.0f * (x * y + w * z);
    Rf[4] = 1.0f - 2.0f * (x * x + z * z);
    Rf[5] = 2.0f * (y * z - w * x);
    Rf[6] = 2.0f * (x * z - w * y);
    Rf[7] = 2.0f * (y * z + w * x);
    Rf[8] = 1.0f - 2.0f * (x * x + y * y);
    tf[0] = (float)pose[4];
    tf[1] = (float)pose[5];
    tf[2] = (float)pose[6];
}

static float depth_key(const float Rf[9], const float tf[3], const double m[3]) {
    const float m0 = (float)m[0], m1 = (float)m[1], m2 = (float)m[2];
    return fmaf(Rf[6], m0, fmaf(Rf[7], m1, fmaf(Rf[8], m2, tf[2])));
}

/* ------------------------------------------------------------------ step 1: projection */

/* Everything the backward needs again for one Gaussian, recomputed on demand. */
typedef struct {
    double qn[4], qnorm, Rg[9], s[3];
    double Sigma[9], Sigma_c[9], J[6];
    double xc[3];
    double tan_c[2];  /* image-plane tangent at which J is taken (clamped x_c / z, y_c / z) */
    int free_t[2];    /* 1 where that tangent is not clamped (J depends on x_c, y_c there) */
} og_geom;

static void geom_one(const og_scene *sc, int64_t i, const og_camera *cam, const double R[9],
                     const double t[3], double jac_clip, og_geom *g) {
    const double *m = sc->means + 3 * i;
    for (int r = 0; r < 3; ++r) g->xc[r] = R[3 * r] * m[0] + R[3 * r + 1] * m[1] + R[3 * r + 2] * m[2] + t[r];
    const double *q = sc->quats + 4 * i;
    g->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) g->qn[k] = q[k] / g->qnorm;
    quat_to_rot(g->qn, g->Rg);
    for (int k = 0; k < 3; ++k) g->s[k] = exp(sc->log_scales[3 * i + k]);
    /* Sigma = Rg diag(s^2) Rg^T */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += g->Rg[3 * a + k] * g->s[k] * g->s[k] * g->Rg[3 * b + k];
            g->Sigma[3 * a + b] = v;
        }
    /* Sigma_c = W Sigma W^T with W the camera rotation */
    double RS[9], Rt[9];
    mat3_mul(R, g->Sigma, RS);
    mat3_transpose(R, Rt);
    mat3_mul(RS, Rt, g->Sigma_c);
    /* Jacobian of pi_m at the camera-frame mean, its tangent clamped (jac_clip > 0) */
    const double z = g->xc[2];
    const double lim[2] = {jac_clip * 0.5 * cam->width / cam->fx, jac_clip * 0.5 * cam->height / cam->fy};
    for (int k = 0; k < 2; ++k) {
        const double tk = g->xc[k] / z;
        g->free_t[k] = !(jac_clip > 0.0) || fabs(tk) <= lim[k];
        g->tan_c[k] = g->free_t[k] ? tk : copysign(lim[k], tk);
    }
    g->J[0] = cam->fx / z;
    g->J[1] = 0.0;
    g->J[2] = -cam->fx * g->tan_c[0] / z;
    g->J[3] = 0.0;
    g->J[4] = cam->fy / z;
    g->J[5] = -cam->fy * g->tan_c[1] / z;
}

static void project_one(const og_scene *sc, int64_t i, const og_camera *cam, const double R[9], const double t[3],
                        const float Rf[9], const float tf[3], const og_params *p, og_proj *pr) {
    og_geom g;
    memset(pr, 0, sizeof(*pr));
    geom_one(sc, i, cam, R, t, p->jac_clip, &g);
    for (int k = 0; k < 3; ++k) pr->xc[k] = g.xc[k];
    const double z = g.xc[2];
    pr->zkey = depth_key(Rf, tf, sc->means + 3 * i);
    if (!(pr->zkey > (float)p->z_near) || !(g.qnorm > 0)) return;
    /* Sigma' = J Sigma_c J^T + dilation I */
    double JS[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += g.J[3 * r + k] * g.Sigma_c[3 * k + c];
            JS[3 * r + c] = v;
        }
    double S00 = 0, S01 = 0, S11 = 0;
    for (int k = 0; k < 3; ++k) {
        S00 += JS[k] * g.J[k];
        S01 += JS[k] * g.J[3 + k];
        S11 += JS[3 + k] * g.J[3 + k];
    }
    S00 += p->dilation;
    S11 += p->dilation;
    const double det = S00 * S11 - S01 * S01;
    if (!(det > 0)) return;
    pr->cov2[0] = S00;
    pr->cov2[1] = S01;
    pr->cov2[2] = S11;
    pr->conic[0] = S11 / det;
    pr->conic[1] = -S01 / det;
    pr->conic[2] = S00 / det;
    /* pi_m of Sec. II-A */
    pr->mu[0] = cam->fx * g.xc[0] / z + cam->cx;
    pr->mu[1] = cam->fy * g.xc[1] / z + cam->cy;
    /* An FP32 renderer applies the pose rounded to FP32: its camera-frame mean is off by
     * ~u (|x| + |t|) (twice that as the bound), nearly the same for neighbouring Gaussians,
     * which moves their screen means together by (f / z)(1 + |x_c / z| + |y_c / z|) times
     * that; the roundings of the product itself differ from Gaussian to Gaussian and
     * average out in the compositing. */
    {
        const double *m = sc->means + 3 * i;
        const double dxc = 2.0 * OG_FP32_ROUNDOFF * (sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) +
                                                     sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]));
        pr->dmu = fmax(cam->fx, cam->fy) / z * dxc * (1.0 + fabs(g.xc[0] / z) + fabs(g.xc[1] / z));
    }
    pr->o = 1.0 / (1.0 + exp(-sc->logits[i]));
    pr->cand = 1;
    /* opacity-aware support: o exp(-d2/2) >= alpha_min  <=>  d2 <= 2 ln(o / alpha_min) */
    if (p->alpha_min > 0) {
        if (pr->o < p->alpha_min) {
            pr->onimage = 0;
            return;
        }
        pr->dmax2 = 2.0 * log(pr->o / p->alpha_min);
        const double hx = sqrt(pr->dmax2 * S00), hy = sqrt(pr->dmax2 * S11);
        double fx0 = floor(pr->mu[0] - hx) - 1, fx1 = ceil(pr->mu[0] + hx) + 1;
        double fy0 = floor(pr->mu[1] - hy) - 1, fy1 = ceil(pr->mu[1] + hy) + 1;
        if (fx1 < 0 || fy1 < 0 || fx0 > cam->width - 1 || fy0 > cam->height - 1) {
            pr->onimage = 0;
            return;
        }
        pr->x0 = fx0 < 0 ? 0 : (int)fx0;
        pr->y0 = fy0 < 0 ? 0 : (int)fy0;
        pr->x1 = fx1 > cam->width - 1 ? cam->width - 1 : (int)fx1;
        pr->y1 = fy1 > cam->height - 1 ? cam->height - 1 : (int)fy1;
    } else {
        pr->dmax2 = INFINITY;
        pr->x0 = 0;
        pr->y0 = 0;
        pr->x1 = cam->width - 1;
        pr->y1 = cam->height - 1;
    }
    pr->onimage = 1;
}

/* ------------------------------------------------------------------ ordering */

typedef struct {
    float z;
    int64_t id;
} og_key;

static int key_cmp(const void *a, const void *b) {
    const og_key *x = (const og_key *)a, *y = (const og_key *)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Candidates in ascending (depth key, index) order. */
static int64_t sorted_candidates(const og_proj *P, int64_t n, int use_bbox, int64_t **out) {
    og_key *keys = (og_key *)malloc(sizeof(og_key) * (size_t)(n > 0 ? n : 1));
    if (!keys) return -1;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!P[i].cand) continue;
        if (use_bbox && !P[i].onimage) continue;
        keys[m].z = P[i].zkey;
        keys[m].id = i;
        ++m;
    }
    qsort(keys, (size_t)m, sizeof(og_key), key_cmp);
    int64_t *ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    if (!ids) {
        free(keys);
        return -1;
    }
    for (int64_t k = 0; k < m; ++k) ids[k] = keys[k].id;
    free(keys);
    *out = ids;
    return m;
}

/* Per-row lists (culled mode): row y holds, in sorted order, every candidate whose box covers y. */
typedef struct {
    int64_t *off; /* height + 1 */
    int64_t *ids;
} og_rows;

static int build_rows(const og_proj *P, const int64_t *order, int64_t m, int height, og_rows *rows) {
    rows->off = (int64_t *)calloc((size_t)height + 1, sizeof(int64_t));
    if (!rows->off) return OG_ERR_OOM;
    for (int64_t k = 0; k < m; ++k) {
        const og_proj *pr = &P[order[k]];
        for (int y = pr->y0; y <= pr->y1; ++y) rows->off[y + 1]++;
    }
    for (int y = 0; y < height; ++y) rows->off[y + 1] += rows->off[y];
    rows->ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rows->off[height] > 0 ? rows->off[height] : 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(height > 0 ? height : 1));
    if (!rows->ids || !cur) {
        free(rows->ids);
        free(cur);
        free(rows->off);
        return OG_ERR_OOM;
    }
    for (int y = 0; y < height; ++y) cur[y] = rows->off[y];
    for (int64_t k = 0; k < m; ++k) {
        const og_proj *pr = &P[order[k]];
        for (int y = pr->y0; y <= pr->y1; ++y) rows->ids[cur[y]++] = order[k];
    }
    free(cur);
    return OG_OK;
}

/* ------------------------------------------------------------------ step 2: Eqs. 2-4 */

/* Reasons a pixel is flagged ambiguous (bits of the mask). */
#define OG_AMB_ALPHA_MIN 1u /* an alpha within its margin of alpha_min, keeping or skipping it matters */
#define OG_AMB_ALPHA_MAX 2u /* an alpha within its margin of alpha_max (the clamp; gradients only) */
#define OG_AMB_T_MIN 4u     /* the transmittance reaches t_min within its margin */

/* One Gaussian at one pixel: its footprint G and alpha_raw = o G (Eq. 1, 2-D form), and
 * the relative error dexp with which an FP32 renderer can know alpha_raw there.  `noise`
 * is added to the exponent (0 except in the perturbed render that tests the mask).
 * |d exponent / d mu'| = |conic d| times the screen-mean error (its 24-bit rounding plus
 * dmu, the FP32 camera transform), and the quadratic form's terms are rounded once
 * each: a footprint evaluated thousands of pixels from its mean has an alpha known only
 * to ~1e-3, an ordinary one to ~1e-5. */
typedef struct {
    double G, araw, dexp;
} og_eval;

static void eval_gaussian(const og_proj *pr, int px, int py, const double noise[3], og_eval *e) {
    const double dx = (double)px - pr->mu[0] - noise[0], dy = (double)py - pr->mu[1] - noise[1];
    const double q = pr->conic[0] * dx * dx + 2.0 * pr->conic[1] * dx * dy + pr->conic[2] * dy * dy;
    e->G = exp(-0.5 * q + noise[2]);
    e->araw = pr->o * e->G;
    const double gx = pr->conic[0] * dx + pr->conic[1] * dy, gy = pr->conic[1] * dx + pr->conic[2] * dy;
    const double terms =
        fabs(pr->conic[0] * dx * dx) + 2.0 * fabs(pr->conic[1] * dx * dy) + fabs(pr->conic[2] * dy * dy);
    const double mu_mag = fmax(fabs(pr->mu[0]), fabs(pr->mu[1]));
    e->dexp = 4.0 * OG_FP32_ROUNDOFF * (sqrt(gx * gx + gy * gy) * mu_mag + terms) + sqrt(gx * gx + gy * gy) * pr->dmu;
}

/* The part of dexp that comes from the rounding of the screen mean and of the quadratic
 * form (the camera transform's part, dmu, moves the whole footprint instead). */
static double rounding_dexp(const og_proj *pr, int px, int py) {
    const double dx = (double)px - pr->mu[0], dy = (double)py - pr->mu[1];
    const double gx = pr->conic[0] * dx + pr->conic[1] * dy, gy = pr->conic[1] * dx + pr->conic[2] * dy;
    const double terms =
        fabs(pr->conic[0] * dx * dx) + 2.0 * fabs(pr->conic[1] * dx * dy) + fabs(pr->conic[2] * dy * dy);
    const double mu_mag = fmax(fabs(pr->mu[0]), fabs(pr->mu[1]));
    return 4.0 * OG_FP32_ROUNDOFF * (sqrt(gx * gx + gy * gy) * mu_mag + terms);
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the 64-bit finaliser applied to
 * seed + counter times the golden-ratio increment; a uniform in [-1, 1) from its top
 * 53 bits.  Used only by the perturbed render, which tests the ambiguity mask. */
static double splitmix_unit(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/* Exponent perturbation of the render that tests the mask: none when scale is 0. */
typedef struct {
    uint64_t seed;
    double scale;
    int64_t n;
} og_noise;

/* The perturbation of Gaussian g at one pixel: its screen mean moved by up to dmu (the
 * camera transform's error, one draw per Gaussian, the same at every pixel) and the
 * exponent of Eq. 1 by up to its rounding error (one draw per pixel and Gaussian). */
static void noise_at(const og_noise *nz, const og_proj *pr, int px, int py, int W, int64_t g, double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    if (!nz || nz->scale == 0.0) return;
    const uint64_t counter = ((uint64_t)py * (uint64_t)W + (uint64_t)px) * (uint64_t)nz->n + (uint64_t)g;
    out[2] = nz->scale * rounding_dexp(pr, px, py) * splitmix_unit(nz->seed, counter);
    const double ang = 3.14159265358979323846 * splitmix_unit(nz->seed ^ 0x5bd1e995u, 2u * (uint64_t)g);
    const double r = nz->scale * pr->dmu * splitmix_unit(nz->seed ^ 0x5bd1e995u, 2u * (uint64_t)g + 1u);
    out[0] = r * cos(ang);
    out[1] = r * sin(ang);
}

/* Relative margin of an alpha decision (alpha_min skip, alpha_max clamp) at one pixel:
 * the fixed floor amb_alpha or dexp, whichever is larger. */
static double alpha_margin(const og_params *p, const og_eval *e) { return fmax(p->amb_alpha, e->dexp); }

/* Is the transmittance Tn after a step within the margin of t_min (relative: the floor
 * amb_t or the carried error bound eT)? */
static int near_t_min(const og_params *p, double Tn, double eT) {
    return fabs(Tn - p->t_min) <= fmax(p->amb_t, eT) * p->t_min;
}

/* Composite one pixel front to back.  out5 = (C_r, C_g, C_b, D, S).  When `contrib` is
 * given, every Gaussian that contributed is recorded with its alpha, its incoming
 * transmittance T and its Gaussian factor G (alpha = min(alpha_max, o G)).  *amb gets
 * the OG_AMB_* reasons for which an FP32 renderer may take another discrete decision. */
static void composite_pixel(int px, int py, const int64_t *list, int64_t nlist, int use_bbox, const og_proj *P,
                            const og_scene *sc, const og_params *p, const og_noise *nz, int W, double out5[5],
                            double *t_final, og_contrib *contrib, int64_t *ncontrib, int *amb, double *diag2) {
    double T = 1.0, C0 = 0, C1 = 0, C2 = 0, D = 0, S = 0;
    double eT = 0.0; /* bound of the relative error of an FP32 renderer's T so far */
    int64_t nc = 0;
    int a = 0;
    if (diag2) diag2[0] = diag2[1] = 0.0;
    for (int64_t k = 0; k < nlist; ++k) {
        const int64_t gi = list[k];
        const og_proj *pr = &P[gi];
        if (use_bbox && (px < pr->x0 || px > pr->x1 || py < pr->y0 || py > pr->y1)) continue;
        og_eval e;
        double nzv[3];
        noise_at(nz, pr, px, py, W, gi, nzv);
        eval_gaussian(pr, px, py, nzv, &e);
        const double araw = e.araw;
        /* Relative margin of the alpha decisions: the fixed amb_alpha, or dexp, whichever is
         * larger.  Skipping or keeping an alpha ~ alpha_min Gaussian moves the pixel by at
         * most about 2 alpha_min T max(1, z): only a decision that can matter is ambiguous.
         * Either way it scales the transmittance of everything behind by 1 - alpha, which
         * an FP32 renderer may therefore hold off by alpha / (1 - alpha): a later t_min
         * decision inherits that uncertainty. */
        const double margin = alpha_margin(p, &e);
        const int near_min = araw > 0.0 && fabs(log(araw / p->alpha_min)) <= margin;
        if (near_min && 2.0 * p->alpha_min * T * fmax(1.0, fabs(pr->xc[2])) > p->amb_effect) a |= OG_AMB_ALPHA_MIN;
        if (near_min) eT += araw / (1.0 - araw);
        if (araw < p->alpha_min) continue;
        const int clamped = araw >= p->alpha_max;
        const double alpha = clamped ? p->alpha_max : araw;
        if (araw > 0.0 && fabs(log(araw / p->alpha_max)) <= margin) a |= OG_AMB_ALPHA_MAX;
        const double z = pr->xc[2];
        const double Tn = T * (1.0 - alpha);
        /* an alpha known to a relative dexp gives 1 - alpha to alpha dexp / (1 - alpha): the
         * product T = prod (1 - alpha_i) compounds it (a clamped alpha is exact) */
        if (!clamped) eT += alpha * e.dexp / (1.0 - alpha);
        if (near_t_min(p, Tn, eT)) a |= OG_AMB_T_MIN;
        if (Tn < p->t_min) {
            if (diag2) {
                diag2[0] = eT;
                diag2[1] = -log1p(-alpha);
            }
            break;
        }
        const double w = alpha * T;
        const double *c = sc->rgb + 3 * gi;
        C0 += c[0] * w;
        C1 += c[1] * w;
        C2 += c[2] * w;
        D += z * w;
        S += w;
        if (contrib) {
            contrib[nc].g = gi;
            contrib[nc].alpha = alpha;
            contrib[nc].T = T;
            contrib[nc].G = e.G;
            contrib[nc].clamped = clamped;
        }
        ++nc;
        T = Tn;
    }
    out5[0] = C0;
    out5[1] = C1;
    out5[2] = C2;
    out5[3] = D;
    out5[4] = S;
    *t_final = T;
    *ncontrib = nc;
    *amb = a;
}

/* Every outcome of one pixel that an FP32 renderer may legitimately produce: the walk of
 * composite_pixel, branching at each decision it would flag (an alpha_min decision that
 * matters: skip and keep; a t_min decision: stop and go on).  An alpha_max decision
 * needs no branch here: the clamp min(alpha_max, alpha) is continuous, so both sides of
 * it give the same maps.  Each finished walk appends (C_r, C_g, C_b, D, S, T) to alts;
 * *overflow is set once more than max_alt outcomes would be needed. */
typedef struct {
    const int64_t *list;
    int64_t nlist;
    int use_bbox, px, py, max_alt, W;
    const og_proj *P;
    const og_scene *sc;
    const og_params *p;
    double *alts;
    int nalt, overflow;
} og_branch;

static void branch_leaf(og_branch *b, const double st[6]) {
    if (b->nalt >= b->max_alt) {
        b->overflow = 1;
        return;
    }
    memcpy(b->alts + 6 * b->nalt, st, 6 * sizeof(double));
    b->nalt++;
}

/* st = (C_r, C_g, C_b, D, S, T); walks list entries k0.. with the transmittance-error
 * bound eT carried as in composite_pixel. */
static void branch_walk(og_branch *b, int64_t k0, const double st_in[6], double eT) {
    double st[6];
    memcpy(st, st_in, sizeof(st));
    const og_params *p = b->p;
    for (int64_t k = k0; k < b->nlist && !b->overflow; ++k) {
        const int64_t gi = b->list[k];
        const og_proj *pr = &b->P[gi];
        if (b->use_bbox && (b->px < pr->x0 || b->px > pr->x1 || b->py < pr->y0 || b->py > pr->y1)) continue;
        og_eval e;
        const double zero[3] = {0.0, 0.0, 0.0};
        eval_gaussian(pr, b->px, b->py, zero, &e);
        const double araw = e.araw, T = st[5];
        const double margin = alpha_margin(p, &e);
        const int near_min = araw > 0.0 && fabs(log(araw / p->alpha_min)) <= margin;
        const int matters = near_min && 2.0 * p->alpha_min * T * fmax(1.0, fabs(pr->xc[2])) > p->amb_effect;
        if (near_min) eT += araw / (1.0 - araw);
        int keep = araw >= p->alpha_min;
        if (matters) {
            /* the other outcome of this alpha_min decision, walked on its own */
            if (keep) {
                branch_walk(b, k + 1, st, eT);
            } else {
                const double alpha = fmin(araw, p->alpha_max), Tn = T * (1.0 - alpha);
                if (!(Tn < p->t_min)) {
                    double s2[6];
                    const double w = alpha * T, *c = b->sc->rgb + 3 * gi;
                    s2[0] = st[0] + c[0] * w;
                    s2[1] = st[1] + c[1] * w;
                    s2[2] = st[2] + c[2] * w;
                    s2[3] = st[3] + pr->xc[2] * w;
                    s2[4] = st[4] + w;
                    s2[5] = Tn;
                    branch_walk(b, k + 1, s2, eT + alpha * e.dexp / (1.0 - alpha));
                } else {
                    branch_leaf(b, st);
                }
            }
            if (b->overflow) return;
        }
        if (!keep) continue;
        const int clamped = araw >= p->alpha_max;
        const double alpha = clamped ? p->alpha_max : araw;
        const double Tn = T * (1.0 - alpha);
        if (!clamped) eT += alpha * e.dexp / (1.0 - alpha);
        const int near_t = near_t_min(p, Tn, eT);
        if (near_t) {
            /* one outcome stops here, the other takes this Gaussian and goes on (whichever
             * of the two the FP64 walk takes) */
            branch_leaf(b, st);
            if (b->overflow) return;
        } else if (Tn < p->t_min) {
            branch_leaf(b, st);
            return;
        }
        const double w = alpha * T, *c = b->sc->rgb + 3 * gi;
        st[0] += c[0] * w;
        st[1] += c[1] * w;
        st[2] += c[2] * w;
        st[3] += pr->xc[2] * w;
        st[4] += w;
        st[5] = Tn;
    }
    if (!b->overflow) branch_leaf(b, st);
}

typedef struct {
    og_proj *P;
    int64_t *order;
    int64_t m;
    og_rows rows;
    int use_bbox;
} og_frame;

static void frame_free(og_frame *f) {
    free(f->P);
    free(f->order);
    if (f->use_bbox) {
        free(f->rows.off);
        free(f->rows.ids);
    }
}

/* f32_pose: project with the pose an FP32 renderer applies (pose_rot_f32, then FP64
 * arithmetic), as the render that tests the ambiguity mask does. */
static int frame_setup(const og_scene *sc, const og_camera *cam, const double pose[7], const og_params *p,
                       int f32_pose, og_frame *f) {
    memset(f, 0, sizeof(*f));
    if (!sc || !cam || !pose || !p || sc->n < 0 || cam->width <= 0 || cam->height <= 0) return OG_ERR_ARG;
    double R[9], t[3], qn[4];
    float Rf[9], tf[3];
    pose_unpack(pose, R, t, qn);
    pose_rot_f32(pose, Rf, tf);
    if (f32_pose) {
        for (int k = 0; k < 9; ++k) R[k] = (double)Rf[k];
        for (int k = 0; k < 3; ++k) t[k] = (double)tf[k];
    }
    f->P = (og_proj *)malloc(sizeof(og_proj) * (size_t)(sc->n > 0 ? sc->n : 1));
    if (!f->P) return OG_ERR_OOM;
    for (int64_t i = 0; i < sc->n; ++i) project_one(sc, i, cam, R, t, Rf, tf, p, &f->P[i]);
    f->use_bbox = !p->brute_force;
    f->m = sorted_candidates(f->P, sc->n, f->use_bbox, &f->order);
    if (f->m < 0) {
        free(f->P);
        return OG_ERR_OOM;
    }
    if (f->use_bbox) {
        int st = build_rows(f->P, f->order, f->m, cam->height, &f->rows);
        if (st) {
            free(f->P);
            free(f->order);
            return st;
        }
    }
    return OG_OK;
}

static void frame_pixel_list(const og_frame *f, int py, const int64_t **list, int64_t *n) {
    if (f->use_bbox) {
        *list = f->rows.ids + f->rows.off[py];
        *n = f->rows.off[py + 1] - f->rows.off[py];
    } else {
        *list = f->order;
        *n = f->m;
    }
}

static void set_threads(const og_params *p) {
#ifdef _OPENMP
    if (p->n_threads > 0) omp_set_num_threads(p->n_threads);
#else
    (void)p;
#endif
}

/* Per Gaussian: 16 doubles = cand, mu_x, mu_y, z, A, B, C, a, b, c, o, dmax2, x0, x1, y0, y1
 * (cand = 1 for a Gaussian that survives the near plane, has det(Sigma') > 0 and whose
 * opacity-aware box meets the image). */
int og_project(const og_scene *sc, const og_camera *cam, const double pose[7], const og_params *p, double *out16) {
    if (!sc || !cam || !pose || !p || !out16) return OG_ERR_ARG;
    double R[9], t[3], qn[4];
    float Rf[9], tf[3];
    pose_unpack(pose, R, t, qn);
    pose_rot_f32(pose, Rf, tf);
    for (int64_t i = 0; i < sc->n; ++i) {
        og_proj pr;
        project_one(sc, i, cam, R, t, Rf, tf, p, &pr);
        double *o = out16 + 16 * i;
        o[0] = (pr.cand && pr.onimage) ? 1.0 : 0.0;
        o[1] = pr.mu[0];
        o[2] = pr.mu[1];
        o[3] = pr.xc[2];
        o[4] = pr.cov2[0];
        o[5] = pr.cov2[1];
        o[6] = pr.cov2[2];
        o[7] = pr.conic[0];
        o[8] = pr.conic[1];
        o[9] = pr.conic[2];
        o[10] = pr.o;
        o[11] = pr.dmax2;
        o[12] = pr.x0;
        o[13] = pr.x1;
        o[14] = pr.y0;
        o[15] = pr.y1;
    }
    return OG_OK;
}

/* Full image, planar: rgb is 3 x H x W, the others H x W.  Any output may be NULL. */
int og_render(const og_scene *sc, const og_camera *cam, const double pose[7], const og_params *p, double *rgb,
              double *depth, double *sil, double *t_final, int32_t *n_contrib, uint8_t *amb) {
    og_frame f;
    int st = frame_setup(sc, cam, pose, p, 0, &f);
    if (st) return st;
    const int W = cam->width, H = cam->height;
    const int64_t HW = (int64_t)W * H;
    set_threads(p);
#pragma omp parallel for schedule(dynamic, 1)
    for (int py = 0; py < H; ++py) {
        const int64_t *list;
        int64_t nl;
        frame_pixel_list(&f, py, &list, &nl);
        for (int px = 0; px < W; ++px) {
            double o5[5], tf;
            int64_t nc;
            int a;
            composite_pixel(px, py, list, nl, f.use_bbox, f.P, sc, p, NULL, W, o5, &tf, NULL, &nc, &a, NULL);
            const int64_t pix = (int64_t)py * W + px;
            if (rgb) {
                rgb[pix] = o5[0];
                rgb[HW + pix] = o5[1];
                rgb[2 * HW + pix] = o5[2];
            }
            if (depth) depth[pix] = o5[3];
            if (sil) sil[pix] = o5[4];
            if (t_final) t_final[pix] = tf;
            if (n_contrib) n_contrib[pix] = (int32_t)nc;
            if (amb) amb[pix] = (uint8_t)a;
        }
    }
    frame_free(&f);
    return OG_OK;
}

/* Selected pixels only (index = y * W + x).  out5 is npix x 5 = (C_r, C_g, C_b, D, S). */
int og_render_pixels(const og_scene *sc, const og_camera *cam, const double pose[7], const og_params *p,
                     const int64_t *pix, int64_t npix, double *out5, double *t_final, uint8_t *amb) {
    if (!pix || npix < 0 || !out5) return OG_ERR_ARG;
    og_frame f;
    int st = frame_setup(sc, cam, pose, p, 0, &f);
    if (st) return st;
    const int W = cam->width;
    set_threads(p);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < npix; ++k) {
        const int px = (int)(pix[k] % W), py = (int)(pix[k] / W);
        const int64_t *list;
        int64_t nl;
        frame_pixel_list(&f, py, &list, &nl);
        double tf;
        int64_t nc;
        int a;
        composite_pixel(px, py, list, nl, f.use_bbox, f.P, sc, p, NULL, W, out5 + 5 * k, &tf, NULL, &nc, &a, NULL);
        if (t_final) t_final[k] = tf;
        if (amb) amb[k] = (uint8_t)a;
    }
    frame_free(&f);
    return OG_OK;
}

/* The render an FP32 renderer could produce under the error model behind the ambiguity
 * mask, for testing that mask: every screen mean moves by scale times up to dmu (the
 * modelled error of an FP32 camera transform, the pose's rounding included) in a
 * direction drawn per Gaussian, and every (pixel, Gaussian) exponent of Eq. 1 by scale
 * times up to its modelled rounding error, the draws SplitMix64 uniforms from (seed,
 * pixel, Gaussian).  With f32_pose the projection also applies the pose rounded to FP32
 * as the GPU kernels do.  Outputs as og_render (any may be NULL). */
int og_render_perturbed(const og_scene *sc, const og_camera *cam, const double pose[7], const og_params *p,
                        uint64_t seed, double scale, int32_t f32_pose, double *rgb, double *depth, double *sil,
                        double *t_final) {
    og_frame f;
    int st = frame_setup(sc, cam, pose, p, f32_pose, &f);
    if (st) return st;
    const int W = cam->width, H = cam->height;
    const int64_t HW = (int64_t)W * H;
    const og_noise nz = {seed, scale, sc->n};
    set_threads(p);
#pragma omp parallel for schedule(dynamic, 1)
    for (int py = 0; py < H; ++py) {
        const int64_t *list;
        int64_t nl;
        frame_pixel_list(&f, py, &list, &nl);
        for (int px = 0; px < W; ++px) {
            double o5[5], tf;
            int64_t nc;
            int a;
            composite_pixel(px, py, list, nl, f.use_bbox, f.P, sc, p, &nz, W, o5, &tf, NULL, &nc, &a, NULL);
            const int64_t pix = (int64_t)py * W + px;
            if (rgb) {
                rgb[pix] = o5[0];
                rgb[HW + pix] = o5[1];
                rgb[2 * HW + pix] = o5[2];
            }
            if (depth) depth[pix] = o5[3];
            if (sil) sil[pix] = o5[4];
            if (t_final) t_final[pix] = tf;
        }
    }
    frame_free(&f);
    return OG_OK;
}

/* Per pixel, for checking the share of pixels the t_min margin flags: at the step where
 * the walk stops on t_min, the transmittance-error bound eT it carried and the step's
 * size -ln(1 - alpha) in log transmittance (both 0 for a pixel whose walk does not stop). */
int og_render_tstats(const og_scene *sc, const og_camera *cam, const double pose[7], const og_params *p,
                     double *eT_stop, double *step_stop) {
    if (!eT_stop || !step_stop) return OG_ERR_ARG;
    og_frame f;
    int st = frame_setup(sc, cam, pose, p, 0, &f);
    if (st) return st;
    const int W = cam->width, H = cam->height;
    set_threads(p);
#pragma omp parallel for schedule(dynamic, 1)
    for (int py = 0; py < H; ++py) {
        const int64_t *list;
        int64_t nl;
        frame_pixel_list(&f, py, &list, &nl);
        for (int px = 0; px < W; ++px) {
            double o5[5], tf, d2[2];
            int64_t nc;
            int a;
            composite_pixel(px, py, list, nl, f.use_bbox, f.P, sc, p, NULL, W, o5, &tf, NULL, &nc, &a, d2);
            const int64_t pix = (int64_t)py * W + px;
            eT_stop[pix] = d2[0];
            step_stop[pix] = d2[1];
        }
    }
    frame_free(&f);
    return OG_OK;
}

/* Every outcome an FP32 renderer may produce at the selected pixels (index y * W + x):
 * the front-to-back walk of Eqs. 2-4 branched at each decision the ambiguity mask flags
 * (see branch_walk).  alts is npix x max_alt x 6 = (C_r, C_g, C_b, D, S, T) per outcome;
 * n_alt[k] is the number of outcomes of pixel k, or -1 when it would take more than
 * max_alt. */
int og_render_alternatives(const og_scene *sc, const og_camera *cam, const double pose[7], const og_params *p,
                           const int64_t *pix, int64_t npix, int32_t max_alt, int32_t *n_alt, double *alts) {
    if (!pix || npix < 0 || max_alt < 1 || !n_alt || !alts) return OG_ERR_ARG;
    og_frame f;
    int st = frame_setup(sc, cam, pose, p, 0, &f);
    if (st) return st;
    const int W = cam->width;
    set_threads(p);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < npix; ++k) {
        og_branch b;
        memset(&b, 0, sizeof(b));
        b.px = (int)(pix[k] % W);
        b.py = (int)(pix[k] / W);
        frame_pixel_list(&f, b.py, &b.list, &b.nlist);
        b.use_bbox = f.use_bbox;
        b.max_alt = max_alt;
        b.W = W;
        b.P = f.P;
        b.sc = sc;
        b.p = p;
        b.alts = alts + (size_t)k * (size_t)max_alt * 6;
        const double st0[6] = {0, 0, 0, 0, 0, 1.0};
        branch_walk(&b, 0, st0, 0.0);
        n_alt[k] = b.overflow ? -1 : b.nalt;
    }
    frame_free(&f);
    return OG_OK;
}

/* Per Gaussian: the FP32 depth key that orders Eqs. 2-4 (depth_key) and the FP64
 * camera-frame depth of its mean, for pinning the key against the exact order. */
int og_depth_keys(const og_scene *sc, const double pose[7], float *keys, double *z64) {
    if (!sc || !pose || !keys || !z64) return OG_ERR_ARG;
    double R[9], t[3], qn[4];
    float Rf[9], tf[3];
    pose_unpack(pose, R, t, qn);
    pose_rot_f32(pose, Rf, tf);
    for (int64_t i = 0; i < sc->n; ++i) {
        const double *m = sc->means + 3 * i;
        keys[i] = depth_key(Rf, tf, m);
        z64[i] = R[6] * m[0] + R[7] * m[1] + R[8] * m[2] + t[2];
    }
    return OG_OK;
}

/* ------------------------------------------------------------------ step 3: the loss */

static double sgn(double x) { return (x > 0) - (x < 0); }

/* L = w_rgb sum_M |C - C*|_1 + w_depth sum_M |D - D*| + w_vis sum_{D*>0} (1 - S)
 *   + w_prior sum_{M, prior>0} |D - prior|,   M = {S > sil_thresh and D* > 0}.
 * The mask is a constant (no gradient through it).  Upstream gradients of L w.r.t.
 * the rendered maps are written when the pointers are non-NULL; amb_grad flags pixels
 * whose mask or L1 sign may differ between FP32 and FP64. */
int og_loss(const og_camera *cam, const og_params *p, const double *rgb, const double *depth, const double *sil,
            const double *rgb_t, const double *depth_t, const double *prior, double *loss, double *d_rgb,
            double *d_depth, double *d_sil, uint8_t *amb_grad) {
    if (!cam || !p || !rgb || !depth || !sil || !rgb_t || !depth_t || !loss) return OG_ERR_ARG;
    const int64_t HW = (int64_t)cam->width * cam->height;
    double L = 0;
    for (int64_t i = 0; i < HW; ++i) {
        const double S = sil[i], D = depth[i], Dt = depth_t[i];
        const int valid = Dt > 0;
        const int M = valid && S > p->sil_thresh;
        const int pv = prior && prior[i] > 0;
        int a = valid && fabs(S - p->sil_thresh) <= p->amb_sil;
        double g[3] = {0, 0, 0}, gD = 0, gS = 0;
        if (M) {
            for (int c = 0; c < 3; ++c) {
                const double r = rgb[c * HW + i] - rgb_t[c * HW + i];
                L += p->w_rgb * fabs(r);
                g[c] = p->w_rgb * sgn(r);
                if (fabs(r) <= p->amb_resid) a = 1;
            }
            const double rd = D - Dt;
            L += p->w_depth * fabs(rd);
            gD += p->w_depth * sgn(rd);
            if (fabs(rd) <= p->amb_resid) a = 1;
            if (pv) {
                const double rp = D - prior[i];
                L += p->w_prior * fabs(rp);
                gD += p->w_prior * sgn(rp);
                if (fabs(rp) <= p->amb_resid) a = 1;
            }
        }
        if (valid) {
            L += p->w_vis * (1.0 - S);
            gS = -p->w_vis;
        }
        if (d_rgb)
            for (int c = 0; c < 3; ++c) d_rgb[c * HW + i] = g[c];
        if (d_depth) d_depth[i] = gD;
        if (d_sil) d_sil[i] = gS;
        if (amb_grad) amb_grad[i] = (uint8_t)a;
    }
    *loss = L;
    return OG_OK;
}

/* ------------------------------------------------------------------ step 4: gradients */

/* Per-Gaussian screen-space gradient layout (10 doubles):
 * 0,1 d mu'_x, d mu'_y; 2,3,4 d conic (a, b, c) with b the single off-diagonal
 * parameter; 5 d opacity; 6,7,8 d rgb; 9 d depth (camera-frame z used in Eq. 3). */
enum { G_MX = 0, G_MY, G_CA, G_CB, G_CC, G_O, G_R, G_G, G_B, G_Z, G_N };

/* Reverse walk of one pixel.  With B_ch the colour of everything behind Gaussian i
 * (B_ch <- alpha_i v_ch + (1 - alpha_i) B_ch, starting from the zero background),
 * dL/dalpha_i = T_i sum_ch g_ch (v_ch,i - B_ch), channels v = (r, g, b, depth, 1). */
static void backward_pixel(int px, int py, const og_contrib *cb, int64_t nc, const og_proj *P, const og_scene *sc,
                           const double g5[5], double *acc /* n x G_N */) {
    double B[5] = {0, 0, 0, 0, 0};
    for (int64_t k = nc - 1; k >= 0; --k) {
        const og_contrib *c = &cb[k];
        const og_proj *pr = &P[c->g];
        const double *col = sc->rgb + 3 * c->g;
        const double v[5] = {col[0], col[1], col[2], pr->xc[2], 1.0};
        double dalpha = 0;
        for (int ch = 0; ch < 5; ++ch) dalpha += g5[ch] * (v[ch] - B[ch]);
        dalpha *= c->T;
        double *a = acc + (size_t)G_N * (size_t)c->g;
        const double w = c->alpha * c->T;
        a[G_R] += w * g5[0];
        a[G_G] += w * g5[1];
        a[G_B] += w * g5[2];
        a[G_Z] += w * g5[3];
        if (!c->clamped) {
            /* alpha = o G, G = exp(power), power = -1/2 (a dx^2 + 2 b dx dy + c dy^2) */
            a[G_O] += dalpha * c->G;
            const double dpow = dalpha * c->alpha;
            const double dx = (double)px - pr->mu[0], dy = (double)py - pr->mu[1];
            a[G_MX] += dpow * (pr->conic[0] * dx + pr->conic[1] * dy);
            a[G_MY] += dpow * (pr->conic[1] * dx + pr->conic[2] * dy);
            a[G_CA] += dpow * (-0.5 * dx * dx);
            a[G_CB] += dpow * (-dx * dy);
            a[G_CC] += dpow * (-0.5 * dy * dy);
        }
        for (int ch = 0; ch < 5; ++ch) B[ch] = c->alpha * v[ch] + (1.0 - c->alpha) * B[ch];
    }
}

/* Chain one Gaussian's screen-space gradient to its parameters and to the pose.
 * grads14 = (means 3, quats 4, log_scales 3, logit 1, rgb 3).  pose6 += (d theta, d t)
 * for x_c <- Exp(theta) x_c (rotation about the camera centre) and x_c <- x_c + t. */
static void chain_one(const og_scene *sc, int64_t i, const og_camera *cam, const double R[9], const double t[3],
                      const og_params *p, const double *a, double *g14, double pose6[6]) {
    og_geom g;
    geom_one(sc, i, cam, R, t, p->jac_clip, &g);
    const double z = g.xc[2], x = g.xc[0], y = g.xc[1];
    /* Sigma' and its inverse (same formulas as the projection) */
    double JS[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += g.J[3 * r + k] * g.Sigma_c[3 * k + c];
            JS[3 * r + c] = v;
        }
    double S00 = p->dilation, S01 = 0, S11 = p->dilation;
    for (int k = 0; k < 3; ++k) {
        S00 += JS[k] * g.J[k];
        S01 += JS[k] * g.J[3 + k];
        S11 += JS[3 + k] * g.J[3 + k];
    }
    const double det = S00 * S11 - S01 * S01;
    const double Q[4] = {S11 / det, -S01 / det, -S01 / det, S00 / det};
    /* d conic as a symmetric matrix: the off-diagonal parameter b appears twice */
    const double Gq[4] = {a[G_CA], 0.5 * a[G_CB], 0.5 * a[G_CB], a[G_CC]};
    /* d Sigma' = -Q Gq Q  (derivative of a matrix inverse) */
    double QG[4], Gs[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) QG[2 * r + c] = Q[2 * r] * Gq[c] + Q[2 * r + 1] * Gq[2 + c];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) Gs[2 * r + c] = -(QG[2 * r] * Q[c] + QG[2 * r + 1] * Q[2 + c]);
    /* Sigma' = J Sigma_c J^T:  d Sigma_c = J^T Gs J,  d J = 2 Gs J Sigma_c */
    double Gc[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double v = 0;
            for (int u = 0; u < 2; ++u)
                for (int w = 0; w < 2; ++w) v += g.J[3 * u + r] * Gs[2 * u + w] * g.J[3 * w + c];
            Gc[3 * r + c] = v;
        }
    double dJ[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double v = 0;
            for (int u = 0; u < 2; ++u) v += Gs[2 * r + u] * JS[3 * u + c];
            dJ[3 * r + c] = 2.0 * v;
        }
    /* camera-frame mean: through pi_m (d mu' = (f / z, -f x / z^2) d x_c, never clamped),
     * the depth channel and J itself: J02 = -fx tan_x / z with tan_x = x / z where free,
     * so dJ02/dx = -fx / z^2 and dJ02/dz = fx tan_x / z^2 + fx x / z^3 there, and
     * dJ02/dx = 0, dJ02/dz = fx tan_x / z^2 where clamped (J12 likewise) */
    const double fx = cam->fx, fy = cam->fy;
    double dxc[3];
    dxc[0] = fx / z * a[G_MX];
    dxc[1] = fy / z * a[G_MY];
    dxc[2] = -fx * x / (z * z) * a[G_MX] - fy * y / (z * z) * a[G_MY] + a[G_Z];
    if (g.free_t[0]) dxc[0] += dJ[2] * (-fx / (z * z));
    if (g.free_t[1]) dxc[1] += dJ[5] * (-fy / (z * z));
    dxc[2] += dJ[0] * (-fx / (z * z)) + dJ[2] * (fx * g.tan_c[0] / (z * z) + (g.free_t[0] ? fx * x / (z * z * z) : 0.0)) +
              dJ[4] * (-fy / (z * z)) + dJ[5] * (fy * g.tan_c[1] / (z * z) + (g.free_t[1] ? fy * y / (z * z * z) : 0.0));
    /* x_c = W m + t */
    double dm[3];
    for (int c = 0; c < 3; ++c) dm[c] = R[c] * dxc[0] + R[3 + c] * dxc[1] + R[6 + c] * dxc[2];
    /* Sigma_c = W Sigma W^T: d Sigma = W^T Gc W */
    double Wt[9], WtG[9], dSig[9];
    mat3_transpose(R, Wt);
    mat3_mul(Wt, Gc, WtG);
    mat3_mul(WtG, R, dSig);
    /* Sigma = Rg D Rg^T with D = diag(s^2): d Rg = 2 dSig Rg D, d s_j = 2 s_j (Rg^T dSig Rg)_jj */
    double dRg[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += dSig[3 * r + k] * g.Rg[3 * k + c];
            dRg[3 * r + c] = 2.0 * v * g.s[c] * g.s[c];
        }
    double dls[3];
    for (int j = 0; j < 3; ++j) {
        double v = 0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) v += g.Rg[3 * r + j] * dSig[3 * r + c] * g.Rg[3 * c + j];
        const double ds = 2.0 * g.s[j] * v;
        dls[j] = ds * g.s[j];
    }
    double dqn[4];
    rot_grad_to_quat(g.qn, dRg, dqn);
    /* q_hat = q / |q| */
    const double proj = dqn[0] * g.qn[0] + dqn[1] * g.qn[1] + dqn[2] * g.qn[2] + dqn[3] * g.qn[3];
    double dq[4];
    for (int k = 0; k < 4; ++k) dq[k] = (dqn[k] - g.qn[k] * proj) / g.qnorm;
    const double o = 1.0 / (1.0 + exp(-sc->logits[i]));
    if (g14) {
        g14[0] = dm[0];
        g14[1] = dm[1];
        g14[2] = dm[2];
        for (int k = 0; k < 4; ++k) g14[3 + k] = dq[k];
        for (int k = 0; k < 3; ++k) g14[7 + k] = dls[k];
        g14[10] = a[G_O] * o * (1.0 - o);
        g14[11] = a[G_R];
        g14[12] = a[G_G];
        g14[13] = a[G_B];
    }
    if (pose6) {
        /* translation: x_c moves one-for-one with t */
        pose6[3] += dxc[0];
        pose6[4] += dxc[1];
        pose6[5] += dxc[2];
        /* rotation about the camera centre, mean part: x_c -> Exp(theta) x_c, d x_c = theta x x_c */
        const double *xc = g.xc;
        pose6[0] += xc[1] * dxc[2] - xc[2] * dxc[1];
        pose6[1] += xc[2] * dxc[0] - xc[0] * dxc[2];
        pose6[2] += xc[0] * dxc[1] - xc[1] * dxc[0];
        /* rotation, covariance part: Sigma_c -> Sigma_c + [th]x Sigma_c - Sigma_c [th]x gives
         * dL = tr((Sigma_c Gc - Gc Sigma_c)[th]x) = -2 m . th with [m]x = Sigma_c Gc - Gc Sigma_c */
        double SG[9], GS[9];
        mat3_mul(g.Sigma_c, Gc, SG);
        mat3_mul(Gc, g.Sigma_c, GS);
        double M[9];
        for (int k = 0; k < 9; ++k) M[k] = SG[k] - GS[k];
        pose6[0] += -2.0 * M[7];
        pose6[1] += -2.0 * M[2];
        pose6[2] += -2.0 * M[3];
    }
}

/* Gradients of sum_p (d_rgb . C + d_depth D + d_sil S) w.r.t. every parameter and the
 * pose, for given upstream maps (planar, like og_render's outputs).  grads14 is n x 14,
 * grads10 is n x 10 (screen-space layout above), pose6 = (d theta, d t) for the two
 * decoupled blocks of chain_one; any may be NULL. */
int og_backward(const og_scene *sc, const og_camera *cam, const double pose[7], const og_params *p,
                const double *d_rgb, const double *d_depth, const double *d_sil, double *grads14, double *grads10,
                double *pose6) {
    if (!d_rgb || !d_depth || !d_sil) return OG_ERR_ARG;
    og_frame f;
    int st = frame_setup(sc, cam, pose, p, 0, &f);
    if (st) return st;
    const int W = cam->width, H = cam->height;
    const int64_t HW = (int64_t)W * H;
    const int64_t n = sc->n;
    set_threads(p);
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nthr * (size_t)(n > 0 ? n : 1) * G_N, sizeof(double));
    if (!acc) {
        frame_free(&f);
        return OG_ERR_OOM;
    }
    int oom = 0;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *myacc = acc + (size_t)tid * (size_t)(n > 0 ? n : 1) * G_N;
        og_contrib *cb = (og_contrib *)malloc(sizeof(og_contrib) * (size_t)(f.m > 0 ? f.m : 1));
        if (!cb) {
#pragma omp atomic write
            oom = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int py = 0; py < H; ++py) {
            if (!cb) continue;
            const int64_t *list;
            int64_t nl;
            frame_pixel_list(&f, py, &list, &nl);
            for (int px = 0; px < W; ++px) {
                const int64_t pix = (int64_t)py * W + px;
                const double g5[5] = {d_rgb[pix], d_rgb[HW + pix], d_rgb[2 * HW + pix], d_depth[pix], d_sil[pix]};
                if (g5[0] == 0 && g5[1] == 0 && g5[2] == 0 && g5[3] == 0 && g5[4] == 0) continue;
                double o5[5], tf;
                int64_t nc;
                int a;
                composite_pixel(px, py, list, nl, f.use_bbox, f.P, sc, p, NULL, W, o5, &tf, cb, &nc, &a, NULL);
                backward_pixel(px, py, cb, nc, f.P, sc, g5, myacc);
            }
        }
        free(cb);
    }
    if (oom) {
        free(acc);
        frame_free(&f);
        return OG_ERR_OOM;
    }
    /* sum the per-thread buffers in thread order */
    for (int th = 1; th < nthr; ++th) {
        const double *src = acc + (size_t)th * (size_t)n * G_N;
        for (int64_t k = 0; k < n * G_N; ++k) acc[k] += src[k];
    }
    if (grads10) memcpy(grads10, acc, sizeof(double) * (size_t)n * G_N);
    double R[9], t[3], qn[4];
    pose_unpack(pose, R, t, qn);
    double p6[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        const og_proj *pr = &f.P[i];
        double *g14 = grads14 ? grads14 + 14 * i : NULL;
        if (!pr->cand) {
            if (g14) memset(g14, 0, sizeof(double) * 14);
            continue;
        }
        chain_one(sc, i, cam, R, t, p, acc + (size_t)G_N * i, g14, pose6 ? p6 : NULL);
    }
    if (pose6) memcpy(pose6, p6, sizeof(p6));
    free(acc);
    frame_free(&f);
    return OG_OK;
}

/* ------------------------------------------------------------------ step 5: pose update */

/* Hamilton product a (x) b. */
static void quat_mul(const double a[4], const double b[4], double c[4]) {
    c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* Decoupled rotation / translation step.  state (16 doubles) = m_rot 3, v_rot 3, m_t 3,
 * v_t 3, step count, 3 unused.  Each block runs its own bias-corrected Adam; the rotation
 * step turns the camera about its centre (R <- Exp(-d) R with the quaternion
 * renormalised, t <- Exp(-d) t) and the translation step moves it (t <- t - d_t). */
int og_adam_step(double pose[7], double state[16], const double g6[6], const og_params *p) {
    if (!pose || !state || !g6 || !p) return OG_ERR_ARG;
    state[12] += 1.0;
    const double k = state[12];
    const double bc1 = 1.0 - pow(p->beta1, k), bc2 = 1.0 - pow(p->beta2, k);
    double step[6];
    for (int j = 0; j < 6; ++j) {
        double *m = &state[j < 3 ? j : 6 + (j - 3)];
        double *v = &state[j < 3 ? 3 + j : 9 + (j - 3)];
        *m = p->beta1 * *m + (1.0 - p->beta1) * g6[j];
        *v = p->beta2 * *v + (1.0 - p->beta2) * g6[j] * g6[j];
        const double mh = *m / bc1, vh = *v / bc2;
        const double lr = j < 3 ? p->lr_rot : p->lr_trans;
        step[j] = lr * mh / (sqrt(vh) + p->eps);
    }
    /* rotation: quaternion of Exp(-step_rot), composed on the left */
    const double th = sqrt(step[0] * step[0] + step[1] * step[1] + step[2] * step[2]);
    double dq[4] = {1, 0, 0, 0};
    if (th > 0) {
        const double s = sin(0.5 * th) / th;
        dq[0] = cos(0.5 * th);
        dq[1] = -step[0] * s;
        dq[2] = -step[1] * s;
        dq[3] = -step[2] * s;
    }
    double q[4] = {pose[0], pose[1], pose[2], pose[3]}, qn[4];
    quat_mul(dq, q, qn);
    const double nq = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
    for (int j = 0; j < 4; ++j) pose[j] = qn[j] / nq;
    /* the camera turns about its own centre: t follows the rotation, then moves */
    double Rd[9], tr[3];
    quat_to_rot(dq, Rd);
    for (int j = 0; j < 3; ++j) tr[j] = Rd[3 * j] * pose[4] + Rd[3 * j + 1] * pose[5] + Rd[3 * j + 2] * pose[6];
    for (int j = 0; j < 3; ++j) pose[4 + j] = tr[j] - step[3 + j];
    return OG_OK;
}

int og_num_threads(const og_params *p) {
    set_threads(p);
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
