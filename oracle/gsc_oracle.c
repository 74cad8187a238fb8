/*
 * GSCache oracle: a plain, slow, obviously-correct CPU restatement of the hot
 * path of "GSCache: Real-Time Radiance Caching for Volume Path Tracing using
 * 3D Gaussian Splatting" (Bauer, Wu, Gadirov, Ma).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant table with the CUDA path; both sides were written
 * separately from the paper and the readings listed in the design notes.
 *
 * Precision: FP64 throughout, except
 *   - the tracer's FP32 mirror mode (trace_body.inc with REAL = float), which
 *     exists so that the GPU tracer can be compared bit for bit;
 *   - the rasterizer's view depth, the sort key of the compositing order and
 *     the near-plane test: a decision the kernel takes in FP32, so the oracle
 *     takes it in FP32 too (same operation order, no contraction).
 *
 * Contents and the passages they follow:
 *   philox4x32_10       Salmon et al., SC'11 (counter-based RNG; the paper is
 *                       silent on its RNG)
 *   orc_trace           Sec. 3.1 (Eq. 1), 3.2, 3.3 (Algorithm 1), 3.4 (Eq. 2),
 *                       3.5; trace_body.inc.  tr_mode selects the reading of
 *                       Algorithm 1's Tr_out (0 cumulative, 1 per call)
 *   orc_init_points     Sec. 3.2 "Cache Initialization": delta-tracked point
 *                       sampling (trace_body.inc); orc_knn3_mean and
 *                       orc_init_scales: the k-NN scale of Eq. 3
 *   orc_transmittance   delta tracking (Sec. 3.2) vs ratio tracking
 *   orc_project         3D Gaussian splatting projection, Sec. 3.1 / Sec. 3.6
 *                       (SH degree 0)
 *   orc_render          front-to-back alpha compositing of all Gaussians per
 *                       pixel (Sec. 3.1)
 *   orc_render_backward analytic gradient of orc_render (the "inverse
 *                       splatting step", Sec. 3.5); orc_render_backward_ex
 *                       adds per Gaussian the summed absolute (pixel, term)
 *                       contributions and their count, orc_project_backward
 *                       its last step alone (2D record -> packed gradient)
 *                       and orc_grad_abs_map that step on absolute values:
 *                       the magnitudes that bound an FP32 evaluation's
 *                       rounding
 *   orc_render_leaves,  orc_render / orc_render_backward taken every way
 *   orc_render_backward_bounds   the decisions within MARGIN_REL of a
 *                       threshold can go (the results and gradient bounds a
 *                       lower-precision implementation may reach)
 *   orc_loss_hdr        Sec. 3.6 "Loss", Eq. after Noise2Noise
 *   orc_loss_l1ssim     0.8 L1 + 0.2 (1 - SSIM), Wang et al. 2004 (not in the
 *                       paper; the 1M-Gaussian differentiation workload)
 *   orc_adamw           Sec. 3.6 "Regularization" (AdamW, Loshchilov & Hutter)
 *   orc_lr_scale        Eq. 4
 *
 * The cache-coupled branch of the tracer (Algorithm 1 with C > 0 and cache
 * images) is pinned by the C -> infinity identity and by closed forms in a
 * homogeneous medium with constant cache images: C -> 0+, one roulette
 * survival then an escape from a dense half-space, and no roulette from
 * Tr = 0.9 up; the per-call reading of Tr_out by its exact relation to the
 * cumulative one when only the third vertex's weight differs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TRACK_MAX_STEPS (1 << 20)
#define TRACE_MAX_LEVELS 16
#define INIT_STREAM 0xffffffffu /* third Philox counter word of the initialisation rays */
#define ORC_MAX_SPHERES 4       /* spherical area lights */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Ten rounds; round r uses key + r * (W0, W1).   */

static void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    philox4x32_10(c, key[0], key[1]);
    memcpy(out, c, sizeof c);
}

/* stream for one path sample: key = seed, counter = (pixel, sample, frame,
   block); each block yields four words consumed in order */
typedef struct {
    uint32_t c0, c1, c2, block, k0, k1;
    uint32_t buf[4];
    int avail;
} rng_t;

static void rng_init(rng_t* r, uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t frame) {
    r->c0 = pixel; r->c1 = sample; r->c2 = frame; r->block = 0;
    r->k0 = (uint32_t)seed; r->k1 = (uint32_t)(seed >> 32);
    r->avail = 0;
}

static uint32_t rng_next(rng_t* r) {
    if (r->avail == 0) {
        uint32_t c[4] = {r->c0, r->c1, r->c2, r->block};
        r->block += 1;
        philox4x32_10(c, r->k0, r->k1);
        memcpy(r->buf, c, sizeof c);
        r->avail = 4;
    }
    uint32_t v = r->buf[4 - r->avail];
    r->avail -= 1;
    return v;
}

/* ------------------------------------------------------------------------ */
/* FP32 elementary functions of the mirror mode.                             */
/* ln: x = 2^e m with m in [sqrt(1/2), sqrt(2)], ln m = 2 atanh(s),          */
/*     s = (m - 1)/(m + 1), atanh by its Taylor series to s^11.              */
/* sincos(2 pi u): quadrant split, theta in [-pi/4, pi/4], Taylor series of  */
/*     sin to theta^9 and cos to theta^10, angle addition with pi/4.         */

static float ln_f32(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    int e = (int)((b >> 23) & 0xffu) - 127;
    uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mb, 4);
    if (m > 1.41421356f) { m = m * 0.5f; e = e + 1; }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = 0.181818182f;
    p = 0.222222222f + s2 * p;
    p = 0.285714286f + s2 * p;
    p = 0.4f + s2 * p;
    p = 0.666666667f + s2 * p;
    p = 2.0f + s2 * p;
    return (float)e * 0.693147181f + s * p;
}

static void sincos2pi_f32(float u, float* sn_out, float* cs_out) {
    float v = u * 4.0f;
    int q = (int)v;
    float f = v - (float)q;
    float th = (f - 0.5f) * 1.57079633f;
    float t2 = th * th;
    float a = 1.0f - t2 * 0.0138888889f;
    a = 1.0f - (t2 * 0.0238095238f) * a;
    a = 1.0f - (t2 * 0.05f) * a;
    a = 1.0f - (t2 * 0.166666667f) * a;
    float sn = th * a;
    float b = 1.0f - t2 * 0.0111111111f;
    b = 1.0f - (t2 * 0.0178571429f) * b;
    b = 1.0f - (t2 * 0.0333333333f) * b;
    b = 1.0f - (t2 * 0.0833333333f) * b;
    float cs = 1.0f - (t2 * 0.5f) * b;
    float cp = (cs - sn) * 0.707106781f;
    float sp = (sn + cs) * 0.707106781f;
    switch (q) {
        case 0: *cs_out = cp; *sn_out = sp; break;
        case 1: *cs_out = -sp; *sn_out = cp; break;
        case 2: *cs_out = -cp; *sn_out = -sp; break;
        default: *cs_out = sp; *sn_out = -cp; break;
    }
}

void orc_ln_f32(const float* x, float* y, int64_t n) {
    for (int64_t i = 0; i < n; ++i) y[i] = ln_f32(x[i]);
}

void orc_sincos2pi_f32(const float* u, float* s, float* c, int64_t n) {
    for (int64_t i = 0; i < n; ++i) sincos2pi_f32(u[i], &s[i], &c[i]);
}

static void sincos2pi_f64(double u, double* s, double* c) {
    *s = sin(6.283185307179586476925 * u);
    *c = cos(6.283185307179586476925 * u);
}

/* ------------------------------------------------------------------------ */
/* tracer, two instantiations                                               */

#define REAL double
#define SUFFIX _d
#define LN(x) log(x)
#define SQRT(x) sqrt(x)
#define SINCOS2PI(u, s, c) sincos2pi_f64((u), (s), (c))
#include "trace_body.inc"
#undef REAL
#undef SUFFIX
#undef LN
#undef SQRT
#undef SINCOS2PI

#define REAL float
#define SUFFIX _f
#define LN(x) ln_f32(x)
#define SQRT(x) sqrtf(x)
#define SINCOS2PI(u, s, c) sincos2pi_f32((u), (s), (c))
#include "trace_body.inc"
#undef REAL
#undef SUFFIX
#undef LN
#undef SQRT
#undef SINCOS2PI

/*
 * Path-traced image and K intermediate path buffers (Sec. 3.5) over a pixel
 * window.  precision = 32 (FP32 mirror) or 64.  cam = R[9], t[3], pos[3],
 * fx, fy, cx, cy.  vol_f = {density_max, sigma_max, albedo}.  light = ldir[3],
 * lrad[3], env[3].  spheres: n_spheres x 7 floats (centre, radius, radiance)
 * of spherical area lights outside the box.  cache: K x 3 x H x W
 * full-frame images or NULL.
 * lengths (optional): per (pixel, sample) path length.
 */
int orc_trace(int precision, const float* grid, int nx, int ny, int nz, const float* vol_f, int tf_n,
              const float* tf_pos, const float* tf_rgba, const float* light, int n_spheres,
              const float* spheres, const float* cam, int W, int H,
              int spp, int max_bounces, int K, uint64_t seed, uint32_t frame, float C, float eps, int tr_mode,
              const float* cache, int x0, int y0, int w, int h, double* targets, double* image,
              int32_t* lengths, int nthreads) {
    if (nx < 2 || ny < 2 || nz < 2 || tf_n < 1 || tf_n > 16 || K < 0 || K > TRACE_MAX_LEVELS || spp < 1 ||
        n_spheres < 0 || n_spheres > ORC_MAX_SPHERES)
        return 1;
    if (precision == 32) {
        vol_t_f v;
        cam_t_f c;
        vol_setup_f(&v, grid, nx, ny, nz, vol_f[0], vol_f[1], vol_f[2], tf_n, tf_pos, tf_rgba, light, light + 3,
                    light + 6);
        vol_spheres_f(&v, n_spheres, spheres);
        cam_setup_f(&c, cam, W, H);
        trace_window_f(&v, &c, spp, max_bounces, K, seed, frame, C, eps, tr_mode, cache, x0, y0, w, h, targets,
                       image, lengths, nthreads);
    } else {
        vol_t_d v;
        cam_t_d c;
        vol_setup_d(&v, grid, nx, ny, nz, vol_f[0], vol_f[1], vol_f[2], tf_n, tf_pos, tf_rgba, light, light + 3,
                    light + 6);
        vol_spheres_d(&v, n_spheres, spheres);
        cam_setup_d(&c, cam, W, H);
        trace_window_d(&v, &c, spp, max_bounces, K, seed, frame, C, eps, tr_mode, cache, x0, y0, w, h, targets,
                       image, lengths, nthreads);
    }
    return 0;
}

/*
 * n transmittance estimates along one ray from `origin` in direction `dir`
 * (FP64): mode 0 = delta tracking (1 if the ray leaves without a real
 * collision, else 0), mode 1 = ratio tracking.  Estimate k uses the Philox
 * stream (k, 0, 0).
 */
void orc_transmittance(int mode, const float* grid, int nx, int ny, int nz, const float* vol_f, int tf_n,
                       const float* tf_pos, const float* tf_rgba, const double* origin, const double* dir,
                       int64_t n, uint64_t seed, double* out, int nthreads) {
    vol_t_d v;
    float zero3[3] = {0, 0, 0}, up[3] = {0, 0, 1};
    vol_setup_d(&v, grid, nx, ny, nz, vol_f[0], vol_f[1], vol_f[2], tf_n, tf_pos, tf_rgba, up, zero3, zero3);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t k = 0; k < n; ++k) {
        rng_t r;
        rng_init(&r, seed, (uint32_t)k, 0u, 0u);
        if (mode == 0) {
            double x[3];
            out[k] = free_flight_d(&v, &r, origin, dir, x) ? 0.0 : 1.0;
        } else {
            out[k] = ratio_T_d(&v, &r, origin, dir);
        }
    }
}

/* density and sigma_t at points (FP64), for closed-form checks */
void orc_sigma_t(const float* grid, int nx, int ny, int nz, const float* vol_f, int tf_n, const float* tf_pos,
                 const float* tf_rgba, const double* pts, int64_t n, double* out) {
    vol_t_d v;
    float zero3[3] = {0, 0, 0}, up[3] = {0, 0, 1};
    vol_setup_d(&v, grid, nx, ny, nz, vol_f[0], vol_f[1], vol_f[2], tf_n, tf_pos, tf_rgba, up, zero3, zero3);
    for (int64_t k = 0; k < n; ++k) out[k] = sigma_t_d(&v, pts + 3 * k);
}

/* ------------------------------------------------------------------------ */
/* Cache initialisation (Sec. 3.2 "Cache Initialization", Eq. 3).            */

/*
 * Point sampling for the points idx[0..n) (NULL: 0..n-1), precision 32 (FP32
 * mirror) or 64.  pos, alb: n x 3; attempts: n (0 = no collision found).
 */
void orc_init_points(int precision, const float* grid, int nx, int ny, int nz, const float* vol_f, int tf_n,
                     const float* tf_pos, const float* tf_rgba, int64_t n, const int64_t* idx, uint64_t seed,
                     int max_attempts, double* pos, double* alb, int32_t* attempts, int nthreads) {
    float zero3[3] = {0, 0, 0}, up[3] = {0, 0, 1};
    if (precision == 32) {
        vol_t_f v;
        vol_setup_f(&v, grid, nx, ny, nz, vol_f[0], vol_f[1], vol_f[2], tf_n, tf_pos, tf_rgba, up, zero3, zero3);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
        for (int64_t k = 0; k < n; ++k) {
            float x[3] = {0, 0, 0}, a[3] = {0, 0, 0};
            attempts[k] = init_point_f(&v, seed, (uint32_t)(idx ? idx[k] : k), max_attempts, x, a);
            for (int c = 0; c < 3; ++c) { pos[3 * k + c] = x[c]; alb[3 * k + c] = a[c]; }
        }
    } else {
        vol_t_d v;
        vol_setup_d(&v, grid, nx, ny, nz, vol_f[0], vol_f[1], vol_f[2], tf_n, tf_pos, tf_rgba, up, zero3, zero3);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
        for (int64_t k = 0; k < n; ++k) {
            double x[3] = {0, 0, 0}, a[3] = {0, 0, 0};
            attempts[k] = init_point_d(&v, seed, (uint32_t)(idx ? idx[k] : k), max_attempts, x, a);
            for (int c = 0; c < 3; ++c) { pos[3 * k + c] = x[c]; alb[3 * k + c] = a[c]; }
        }
    }
}

/*
 * Mean distance to the three nearest other points (Eq. 3's (1/3) sum_j d_ij),
 * by brute force in FP64: for query q[k] (an index into pts, M x 3) over all
 * M points but itself.  Fewer than three other points: the mean of those.
 */
void orc_knn3_mean(const double* pts, int64_t M, const int64_t* q, int64_t Q, double* out, int nthreads) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t k = 0; k < Q; ++k) {
        int64_t i = q ? q[k] : k;
        double b[3] = {INFINITY, INFINITY, INFINITY};
        for (int64_t j = 0; j < M; ++j) {
            if (j == i) continue;
            double dx = pts[3 * j] - pts[3 * i], dy = pts[3 * j + 1] - pts[3 * i + 1], dz = pts[3 * j + 2] - pts[3 * i + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (d < b[2]) {
                if (d < b[1]) {
                    b[2] = b[1];
                    if (d < b[0]) { b[1] = b[0]; b[0] = d; } else b[1] = d;
                } else {
                    b[2] = d;
                }
            }
        }
        int m = M - 1 < 3 ? (int)(M - 1) : 3;
        double acc = 0;
        for (int t = 0; t < m; ++t) acc += b[t];
        out[k] = m > 0 ? acc / m : 0.0;
    }
}

/*
 * Eq. 3: s_i = min(mu + 2 sigma, mbar_i) / 2 over the M mean 3-NN distances
 * mbar (mu, sigma: their mean and population standard deviation).
 */
void orc_init_scales(const double* mbar, int64_t M, double* s, double* mu_out, double* sigma_out) {
    double mu = 0, var = 0;
    for (int64_t i = 0; i < M; ++i) mu += mbar[i];
    mu /= (double)(M > 0 ? M : 1);
    for (int64_t i = 0; i < M; ++i) var += (mbar[i] - mu) * (mbar[i] - mu);
    var /= (double)(M > 0 ? M : 1);
    double cap = mu + 2.0 * sqrt(var);
    for (int64_t i = 0; i < M; ++i) s[i] = (mbar[i] < cap ? mbar[i] : cap) / 2.0;
    if (mu_out) *mu_out = mu;
    if (sigma_out) *sigma_out = sqrt(var);
}

/* ------------------------------------------------------------------------ */
/* 3D Gaussian splatting rasterizer (FP64).                                  */
/*                                                                           */
/* Packed parameters per Gaussian (16 float): mean[0:3], opacity logit[3],  */
/* log-scale[4:7], pad, quaternion (w,x,y,z)[8:12], RGB[12:15], pad.         */
/* cam: R[9] (rows: right, down, forward), t[3], pos[3], fx, fy, cx, cy.     */
/* cfg: alpha_max, alpha_min, T_min, near, dilation.                         */

typedef struct {
    double mx, my;          /* projected mean, pixel units */
    double a, b, c;         /* conic: inverse of the 2D covariance */
    double op;              /* sigmoid(opacity logit) */
    double col[3];          /* max(rgb, 0) */
    double lthr;            /* ln(alpha_min / opacity): power below it cannot reach alpha_min */
    float depth;            /* FP32 view depth (sort key) */
    int visible;
} proj_t;

typedef struct {
    double R[9], t[3], fx, fy, cx, cy;
    float Rf[9], tf[3];
} rcam_t;

static void rcam_setup(rcam_t* c, const float* cam) {
    for (int k = 0; k < 9; ++k) { c->R[k] = cam[k]; c->Rf[k] = cam[k]; }
    for (int k = 0; k < 3; ++k) { c->t[k] = cam[9 + k]; c->tf[k] = cam[9 + k]; }
    c->fx = cam[15]; c->fy = cam[16]; c->cx = cam[17]; c->cy = cam[18];
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* rotation matrix of the unit quaternion (w, x, y, z), row-major */
static void quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* FP32 view depth, operation order ((r20 x + r21 y) + r22 z) + t2 */
static float view_depth_f32(const rcam_t* c, const float* m) {
    float p0 = c->Rf[6] * m[0];
    float p1 = c->Rf[7] * m[1];
    float p2 = c->Rf[8] * m[2];
    float s = p0 + p1;
    s = s + p2;
    return s + c->tf[2];
}

/* intermediate quantities of one projection, kept for the backward pass */
typedef struct {
    double qn[4], qnorm, Rq[9], s[3], M[9], Sig[9], t[3], J[6], Tm[6], A, B, Cc, det;
} proj_aux_t;

static void project_one(const float* p, const rcam_t* c, const double* cfg, proj_t* out, proj_aux_t* aux) {
    proj_aux_t local;
    proj_aux_t* x = aux ? aux : &local;
    out->visible = 0;
    out->depth = view_depth_f32(c, p);
    if (!(out->depth > (float)cfg[3])) return;
    double q[4] = {p[8], p[9], p[10], p[11]};
    x->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) x->qn[k] = q[k] / x->qnorm;
    quat_to_rot(x->qn, x->Rq);
    for (int k = 0; k < 3; ++k) x->s[k] = exp((double)p[4 + k]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) x->M[3 * i + j] = x->Rq[3 * i + j] * x->s[j];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += x->M[3 * i + j] * x->M[3 * k + j];
            x->Sig[3 * i + k] = acc;
        }
    for (int m = 0; m < 3; ++m)
        x->t[m] = c->R[3 * m] * p[0] + c->R[3 * m + 1] * p[1] + c->R[3 * m + 2] * p[2] + c->t[m];
    double tx = x->t[0], ty = x->t[1], tz = x->t[2];
    x->J[0] = c->fx / tz; x->J[1] = 0;            x->J[2] = -c->fx * tx / (tz * tz);
    x->J[3] = 0;          x->J[4] = c->fy / tz;   x->J[5] = -c->fy * ty / (tz * tz);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int m = 0; m < 3; ++m) acc += x->J[3 * r + m] * c->R[3 * m + k];
            x->Tm[3 * r + k] = acc;
        }
    double S2[4];
    for (int r = 0; r < 2; ++r)
        for (int q2 = 0; q2 < 2; ++q2) {
            double acc = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) acc += x->Tm[3 * r + i] * x->Sig[3 * i + j] * x->Tm[3 * q2 + j];
            S2[2 * r + q2] = acc;
        }
    x->A = S2[0] + cfg[4];
    x->B = S2[1];
    x->Cc = S2[3] + cfg[4];
    x->det = x->A * x->Cc - x->B * x->B;
    if (!(x->det > 0)) return;
    out->a = x->Cc / x->det;
    out->b = -x->B / x->det;
    out->c = x->A / x->det;
    out->mx = c->fx * tx / tz + c->cx;
    out->my = c->fy * ty / tz + c->cy;
    out->op = sigmoid((double)p[3]);
    out->lthr = log(cfg[1] / out->op);
    for (int k = 0; k < 3; ++k) out->col[k] = p[12 + k] > 0.0f ? (double)p[12 + k] : 0.0;
    out->visible = 1;
}

/* per-Gaussian projection: mx, my, a, b, c, opacity, r, g, b, depth, visible */
void orc_project(int64_t N, const float* params, const float* cam, const double* cfg, double* out) {
    rcam_t c;
    rcam_setup(&c, cam);
    for (int64_t g = 0; g < N; ++g) {
        proj_t pr;
        memset(&pr, 0, sizeof pr);
        project_one(params + 16 * g, &c, cfg, &pr, NULL);
        double* o = out + 11 * g;
        o[0] = pr.mx; o[1] = pr.my; o[2] = pr.a; o[3] = pr.b; o[4] = pr.c; o[5] = pr.op;
        o[6] = pr.col[0]; o[7] = pr.col[1]; o[8] = pr.col[2]; o[9] = pr.depth; o[10] = pr.visible;
    }
}

typedef struct {
    float depth;
    int64_t idx;
} order_t;

static int order_cmp(const void* pa, const void* pb) {
    const order_t* a = (const order_t*)pa;
    const order_t* b = (const order_t*)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* project all Gaussians, return the visible ones sorted by (depth, index) */
static int64_t project_sorted(int64_t N, const float* params, const rcam_t* c, const double* cfg, proj_t* pr,
                              int64_t* order, int nthreads) {
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t g = 0; g < N; ++g) project_one(params + 16 * g, c, cfg, &pr[g], NULL);
    order_t* tmp = (order_t*)malloc(sizeof(order_t) * (size_t)(N > 0 ? N : 1));
    int64_t V = 0;
    for (int64_t g = 0; g < N; ++g)
        if (pr[g].visible) { tmp[V].depth = pr[g].depth; tmp[V].idx = g; ++V; }
    qsort(tmp, (size_t)V, sizeof(order_t), order_cmp);
    for (int64_t k = 0; k < V; ++k) order[k] = tmp[k].idx;
    free(tmp);
    return V;
}

static int near_rel(double x, double thr, double rel) { return fabs(x - thr) <= rel * fabs(thr); }

#define MARGIN_REL 2e-4

typedef struct {
    int64_t g;
    double alpha, T, G, dx, dy;
    int clamped;
} term_t;

/*
 * Walk one pixel front to back over the depth-ordered visible Gaussians.
 * The plain definition: alpha = min(alpha_max, sigmoid(o) exp(-d^T conic d / 2)),
 * terms with alpha < alpha_min are dropped, the walk stops before a term
 * whose T (1 - alpha) < T_min, C = sum c alpha T.  Returns the number of
 * composited terms; `terms` (optional, capacity cap) receives them.
 * *marginal is set if a threshold decision lay within MARGIN_REL of its
 * threshold (the FP32 kernel may decide it the other way).
 */
static int64_t walk_pixel(const proj_t* pr, const int64_t* order, int64_t V, const double* cfg, double px,
                          double py, double C[3], double* T_final, int* marginal, term_t* terms, int64_t cap,
                          int grad_margins) {
    double amax = cfg[0], amin = cfg[1], tmin = cfg[2];
    double T = 1.0;
    int64_t n = 0;
    C[0] = C[1] = C[2] = 0.0;
    *marginal = 0;
    for (int64_t k = 0; k < V; ++k) {
        const proj_t* p = &pr[order[k]];
        double dx = px - p->mx, dy = py - p->my;
        double power = -0.5 * (p->a * dx * dx + p->c * dy * dy) - p->b * dx * dy;
        /* cheap reject far below the alpha_min threshold, before exp */
        if (power < p->lthr - 1e-3) continue;
        double G = exp(power);
        double araw = p->op * G;
        if (near_rel(araw, amin, MARGIN_REL)) *marginal = 1;
        if (grad_margins && near_rel(araw, amax, MARGIN_REL)) *marginal = 1;
        double alpha = araw < amax ? araw : amax;
        if (alpha < amin) continue;
        double Tn = T * (1.0 - alpha);
        if (near_rel(Tn, tmin, MARGIN_REL)) *marginal = 1;
        if (Tn < tmin) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += p->col[ch] * alpha * T;
        if (terms && n < cap) {
            term_t* t = &terms[n];
            t->g = order[k]; t->alpha = alpha; t->T = T; t->G = G; t->dx = dx; t->dy = dy;
            t->clamped = araw >= amax;
        }
        ++n;
        T = Tn;
    }
    *T_final = T;
    return n;
}

/*
 * Forward render of the pixel window [x0, x0 + w) x [y0, y0 + h) of a W x H
 * camera.  Pixel (i, j) is sampled at its centre (i + 0.5, j + 0.5);
 * background 0.  image: 3 x h x w; marginal, ncontrib: h x w (optional).
 * grad_margins != 0 also flags pixels with a term near the alpha_max clamp
 * (where the gradient, not the image, jumps).
 */
int orc_render(int64_t N, const float* params, const float* cam, const double* cfg, int x0, int y0, int w, int h,
               double* image, uint8_t* marginal, int32_t* ncontrib, double* T_final, int grad_margins,
               int nthreads) {
    rcam_t c;
    rcam_setup(&c, cam);
    proj_t* pr = (proj_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(proj_t));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!pr || !order) { free(pr); free(order); return 2; }
    int64_t V = project_sorted(N, params, &c, cfg, pr, order, nthreads);
    long WH = (long)w * h;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int jj = 0; jj < h; ++jj) {
        for (int ii = 0; ii < w; ++ii) {
            double C[3], T;
            int marg;
            int64_t n = walk_pixel(pr, order, V, cfg, x0 + ii + 0.5, y0 + jj + 0.5, C, &T, &marg, NULL, 0,
                                   grad_margins);
            long p = (long)jj * w + ii;
            for (int ch = 0; ch < 3; ++ch) image[ch * WH + p] = C[ch];
            if (marginal) marginal[p] = (uint8_t)marg;
            if (ncontrib) ncontrib[p] = (int32_t)n;
            if (T_final) T_final[p] = T;
        }
    }
    free(pr);
    free(order);
    return 0;
}

/*
 * Backward of a project step, from 2D gradients to the packed parameter
 * gradient (chain rule through conic = inverse(J W Sigma W^T J^T + dil I),
 * Sigma = R(q/|q|) diag(exp(ls))^2 R^T, the pinhole projection of the mean).
 * g2: dL/d{mx, my, a, b, c, opacity logit, r, g, b}.  grad: 16 floats (+=).
 */
static void project_backward_one(const float* p, const rcam_t* c, const double* cfg, const double* g2,
                                 double* grad) {
    proj_t pr;
    proj_aux_t x;
    project_one(p, c, cfg, &pr, &x);
    if (!pr.visible) return;
    double A = x.A, B = x.B, Cc = x.Cc, det2 = x.det * x.det;
    double ga = g2[2], gb = g2[3], gc = g2[4];
    /* d conic / d (A, B, Cc) of a = Cc/det, b = -B/det, c = A/det */
    double dA = (ga * (-Cc * Cc) + gb * (B * Cc) + gc * (-B * B)) / det2;
    double dB = (ga * (2 * B * Cc) + gb * (-(A * Cc + B * B)) + gc * (2 * A * B)) / det2;
    double dC = (ga * (-B * B) + gb * (A * B) + gc * (-A * A)) / det2;
    /* A = Tm0 Sig Tm0^T, B = Tm0 Sig Tm1^T, Cc = Tm1 Sig Tm1^T */
    const double* Tm0 = x.Tm;
    const double* Tm1 = x.Tm + 3;
    double G[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            G[3 * i + j] = dA * Tm0[i] * Tm0[j] + dB * Tm0[i] * Tm1[j] + dC * Tm1[i] * Tm1[j];
    double ST0[3], ST1[3];
    for (int k = 0; k < 3; ++k) {
        ST0[k] = x.Sig[3 * k] * Tm0[0] + x.Sig[3 * k + 1] * Tm0[1] + x.Sig[3 * k + 2] * Tm0[2];
        ST1[k] = x.Sig[3 * k] * Tm1[0] + x.Sig[3 * k + 1] * Tm1[1] + x.Sig[3 * k + 2] * Tm1[2];
    }
    double dTm[6];
    for (int k = 0; k < 3; ++k) {
        dTm[k] = 2 * dA * ST0[k] + dB * ST1[k];
        dTm[3 + k] = dB * ST0[k] + 2 * dC * ST1[k];
    }
    /* Tm = J R_w */
    double dJ[6];
    for (int r = 0; r < 2; ++r)
        for (int m = 0; m < 3; ++m) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += dTm[3 * r + k] * c->R[3 * m + k];
            dJ[3 * r + m] = acc;
        }
    double tx = x.t[0], ty = x.t[1], tz = x.t[2];
    double tz2 = tz * tz, tz3 = tz2 * tz;
    double dt[3] = {0, 0, 0};
    dt[0] += dJ[2] * (-c->fx / tz2);
    dt[1] += dJ[5] * (-c->fy / tz2);
    dt[2] += dJ[0] * (-c->fx / tz2) + dJ[2] * (2 * c->fx * tx / tz3) + dJ[4] * (-c->fy / tz2) +
             dJ[5] * (2 * c->fy * ty / tz3);
    /* mean2D = (fx tx / tz + cx, fy ty / tz + cy) */
    dt[0] += g2[0] * c->fx / tz;
    dt[2] += g2[0] * (-c->fx * tx / tz2);
    dt[1] += g2[1] * c->fy / tz;
    dt[2] += g2[1] * (-c->fy * ty / tz2);
    /* t = R_w mean + t_w */
    for (int k = 0; k < 3; ++k) grad[k] += c->R[k] * dt[0] + c->R[3 + k] * dt[1] + c->R[6 + k] * dt[2];
    /* Sigma = M M^T, M = R_q diag(s): dL/dM = (G + G^T) M */
    double dM[9];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += (G[3 * k + j] + G[3 * j + k]) * x.M[3 * j + l];
            dM[3 * k + l] = acc;
        }
    double dR[9];
    for (int l = 0; l < 3; ++l) {
        double ds = 0;
        for (int k = 0; k < 3; ++k) {
            ds += dM[3 * k + l] * x.Rq[3 * k + l];
            dR[3 * k + l] = dM[3 * k + l] * x.s[l];
        }
        grad[4 + l] += ds * x.s[l];
    }
    /* rotation matrix of the normalised quaternion */
    double w = x.qn[0], qx = x.qn[1], qy = x.qn[2], qz = x.qn[3];
    double dq[4];
    dq[0] = 2 * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
    dq[1] = 2 * (qy * dR[1] + qz * dR[2] + qy * dR[3] - w * dR[5] + qz * dR[6] + w * dR[7]) -
            4 * qx * (dR[4] + dR[8]);
    dq[2] = 2 * (qx * dR[1] + w * dR[2] + qx * dR[3] + qz * dR[5] - w * dR[6] + qz * dR[7]) -
            4 * qy * (dR[0] + dR[8]);
    dq[3] = 2 * (-w * dR[1] + qx * dR[2] + w * dR[3] + qy * dR[5] + qx * dR[6] + qy * dR[7]) -
            4 * qz * (dR[0] + dR[4]);
    double dot = w * dq[0] + qx * dq[1] + qy * dq[2] + qz * dq[3];
    for (int k = 0; k < 4; ++k) grad[8 + k] += (dq[k] - x.qn[k] * dot) / x.qnorm;
    grad[3] += g2[5];
    for (int k = 0; k < 3; ++k) grad[12 + k] += g2[6 + k];
}

/*
 * Gradient of the window render w.r.t. the packed parameters, given
 * dL/dimage (3 x h x w).  grads: N x 16 (+=).  g2d (optional): N x 9 2D
 * gradients dL/d{mx, my, a, b, c, opacity logit, r, g, b} (+=).
 *
 * The 2D gradient of a Gaussian is a sum over (pixel, term) contributions.
 * For the error analysis of an FP32 implementation, abs2d (optional, N x 9)
 * receives the sum of their absolute values and nterm (optional, N) their
 * number; neither changes the gradient.
 */
int orc_render_backward_ex(int64_t N, const float* params, const float* cam, const double* cfg, int x0, int y0,
                           int w, int h, const double* dL_dimage, double* grads, double* g2d, double* abs2d,
                           int64_t* nterm, int nthreads);

int orc_render_backward(int64_t N, const float* params, const float* cam, const double* cfg, int x0, int y0, int w,
                        int h, const double* dL_dimage, double* grads, double* g2d, int nthreads) {
    return orc_render_backward_ex(N, params, cam, cfg, x0, y0, w, h, dL_dimage, grads, g2d, NULL, NULL, nthreads);
}

int orc_render_backward_ex(int64_t N, const float* params, const float* cam, const double* cfg, int x0, int y0,
                           int w, int h, const double* dL_dimage, double* grads, double* g2d, double* abs2d,
                           int64_t* nterm, int nthreads) {
    rcam_t c;
    rcam_setup(&c, cam);
    proj_t* pr = (proj_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(proj_t));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    double* acc = (double*)calloc((size_t)(N > 0 ? N : 1) * 9, sizeof(double));
    if (!pr || !order || !acc) { free(pr); free(order); free(acc); return 2; }
    int64_t V = project_sorted(N, params, &c, cfg, pr, order, nthreads);
    long WH = (long)w * h;
#pragma omp parallel num_threads(nthreads)
    {
        int64_t cap = 4096;
        term_t* terms = (term_t*)malloc(sizeof(term_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
        for (int jj = 0; jj < h; ++jj) {
            for (int ii = 0; ii < w; ++ii) {
                long p = (long)jj * w + ii;
                double gC[3] = {dL_dimage[p], dL_dimage[WH + p], dL_dimage[2 * WH + p]};
                if (gC[0] == 0 && gC[1] == 0 && gC[2] == 0) continue;
                double C[3], T;
                int marg;
                int64_t n = walk_pixel(pr, order, V, cfg, x0 + ii + 0.5, y0 + jj + 0.5, C, &T, &marg, terms, cap, 1);
                if (n > cap) {
                    cap = n;
                    terms = (term_t*)realloc(terms, sizeof(term_t) * (size_t)cap);
                    n = walk_pixel(pr, order, V, cfg, x0 + ii + 0.5, y0 + jj + 0.5, C, &T, &marg, terms, cap, 1);
                }
                double S[3] = {0, 0, 0};
                for (int64_t k = n - 1; k >= 0; --k) {
                    const term_t* t = &terms[k];
                    const proj_t* q = &pr[t->g];
                    const float* pp = params + 16 * t->g;
                    double* a9 = acc + 9 * t->g;
                    double dalpha = 0;
                    if (nterm) {
#pragma omp atomic
                        nterm[t->g] += 1;
                    }
                    for (int ch = 0; ch < 3; ++ch) {
                        if (pp[12 + ch] > 0.0f) {
#pragma omp atomic
                            a9[6 + ch] += t->alpha * t->T * gC[ch];
                            if (abs2d) {
#pragma omp atomic
                                abs2d[9 * t->g + 6 + ch] += fabs(t->alpha * t->T * gC[ch]);
                            }
                        }
                        dalpha += gC[ch] * (q->col[ch] * t->T - S[ch] / (1.0 - t->alpha));
                        S[ch] += q->col[ch] * t->alpha * t->T;
                    }
                    if (t->clamped) continue;
                    double dop = dalpha * t->G * q->op * (1.0 - q->op);
                    double dpow = dalpha * t->alpha;
                    double v[5];
                    v[0] = dpow * (q->a * t->dx + q->b * t->dy);
                    v[1] = dpow * (q->b * t->dx + q->c * t->dy);
                    v[2] = dpow * (-0.5 * t->dx * t->dx);
                    v[3] = dpow * (-t->dx * t->dy);
                    v[4] = dpow * (-0.5 * t->dy * t->dy);
                    for (int k5 = 0; k5 < 5; ++k5) {
#pragma omp atomic
                        a9[k5] += v[k5];
                        if (abs2d) {
#pragma omp atomic
                            abs2d[9 * t->g + k5] += fabs(v[k5]);
                        }
                    }
#pragma omp atomic
                    a9[5] += dop;
                    if (abs2d) {
#pragma omp atomic
                        abs2d[9 * t->g + 5] += fabs(dop);
                    }
                }
            }
        }
        free(terms);
    }
    if (g2d)
        for (int64_t g = 0; g < 9 * N; ++g) g2d[g] += acc[g];
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t g = 0; g < N; ++g) {
        const double* a9 = acc + 9 * g;
        int any = 0;
        for (int k = 0; k < 9; ++k) any |= a9[k] != 0;
        if (any) project_backward_one(params + 16 * g, &c, cfg, a9, grads + 16 * g);
    }
    free(pr);
    free(order);
    free(acc);
    return 0;
}

/*
 * Magnitude of the projection backward (project_backward_one) for a record
 * of magnitudes m >= 0: the same operations with every operand replaced by
 * its absolute value and every difference by a sum.  It bounds |J a| for any
 * record |a| <= m (J the record-to-packed-gradient Jacobian), and it bounds
 * the intermediate values too, so that u times it (times the number of
 * operations on the way) bounds the rounding of a low-precision evaluation,
 * including the cancellation of the quaternion gradient's radial part.
 * out: N x 16 (overwritten); Gaussians with a zero m row get zeros.
 */
static void project_backward_mag(const float* p, const rcam_t* c, const double* cfg, const double* m,
                                 double* grad) {
    proj_t pr;
    proj_aux_t x;
    project_one(p, c, cfg, &pr, &x);
    if (!pr.visible) return;
    const double A = fabs(x.A), B = fabs(x.B), Cc = fabs(x.Cc), det2 = x.det * x.det;
    const double ga = m[2], gb = m[3], gc = m[4];
    const double dA = (ga * Cc * Cc + gb * B * Cc + gc * B * B) / det2;
    const double dB = (ga * 2 * B * Cc + gb * (A * Cc + B * B) + gc * 2 * A * B) / det2;
    const double dC = (ga * B * B + gb * A * B + gc * A * A) / det2;
    double T0[3], T1[3], Sg[9], G[9];
    for (int k = 0; k < 3; ++k) { T0[k] = fabs(x.Tm[k]); T1[k] = fabs(x.Tm[3 + k]); }
    for (int k = 0; k < 9; ++k) Sg[k] = fabs(x.Sig[k]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G[3 * i + j] = dA * T0[i] * T0[j] + dB * T0[i] * T1[j] + dC * T1[i] * T1[j];
    double ST0[3], ST1[3];
    for (int k = 0; k < 3; ++k) {
        ST0[k] = Sg[3 * k] * T0[0] + Sg[3 * k + 1] * T0[1] + Sg[3 * k + 2] * T0[2];
        ST1[k] = Sg[3 * k] * T1[0] + Sg[3 * k + 1] * T1[1] + Sg[3 * k + 2] * T1[2];
    }
    double dTm[6];
    for (int k = 0; k < 3; ++k) {
        dTm[k] = 2 * dA * ST0[k] + dB * ST1[k];
        dTm[3 + k] = dB * ST0[k] + 2 * dC * ST1[k];
    }
    double dJ[6];
    for (int r = 0; r < 2; ++r)
        for (int mm = 0; mm < 3; ++mm) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += dTm[3 * r + k] * fabs(c->R[3 * mm + k]);
            dJ[3 * r + mm] = acc;
        }
    const double tx = fabs(x.t[0]), ty = fabs(x.t[1]), tz = fabs(x.t[2]);
    const double tz2 = tz * tz, tz3 = tz2 * tz, fx = fabs(c->fx), fy = fabs(c->fy);
    double dt[3] = {0, 0, 0};
    dt[0] += dJ[2] * fx / tz2 + m[0] * fx / tz;
    dt[1] += dJ[5] * fy / tz2 + m[1] * fy / tz;
    dt[2] += dJ[0] * fx / tz2 + dJ[2] * 2 * fx * tx / tz3 + dJ[4] * fy / tz2 + dJ[5] * 2 * fy * ty / tz3 +
             m[0] * fx * tx / tz2 + m[1] * fy * ty / tz2;
    for (int k = 0; k < 3; ++k)
        grad[k] += fabs(c->R[k]) * dt[0] + fabs(c->R[3 + k]) * dt[1] + fabs(c->R[6 + k]) * dt[2];
    double dM[9];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += (G[3 * k + j] + G[3 * j + k]) * fabs(x.M[3 * j + l]);
            dM[3 * k + l] = acc;
        }
    double dR[9];
    for (int l = 0; l < 3; ++l) {
        double ds = 0;
        for (int k = 0; k < 3; ++k) {
            ds += dM[3 * k + l] * fabs(x.Rq[3 * k + l]);
            dR[3 * k + l] = dM[3 * k + l] * x.s[l];
        }
        grad[4 + l] += ds * x.s[l];
    }
    const double w = fabs(x.qn[0]), qx = fabs(x.qn[1]), qy = fabs(x.qn[2]), qz = fabs(x.qn[3]);
    double dq[4];
    dq[0] = 2 * (qz * dR[1] + qy * dR[2] + qz * dR[3] + qx * dR[5] + qy * dR[6] + qx * dR[7]);
    dq[1] = 2 * (qy * dR[1] + qz * dR[2] + qy * dR[3] + w * dR[5] + qz * dR[6] + w * dR[7]) + 4 * qx * (dR[4] + dR[8]);
    dq[2] = 2 * (qx * dR[1] + w * dR[2] + qx * dR[3] + qz * dR[5] + w * dR[6] + qz * dR[7]) + 4 * qy * (dR[0] + dR[8]);
    dq[3] = 2 * (w * dR[1] + qx * dR[2] + w * dR[3] + qy * dR[5] + qx * dR[6] + qy * dR[7]) + 4 * qz * (dR[0] + dR[4]);
    const double dot = w * dq[0] + qx * dq[1] + qy * dq[2] + qz * dq[3];
    const double qa[4] = {w, qx, qy, qz};
    for (int k = 0; k < 4; ++k) grad[8 + k] += (dq[k] + qa[k] * dot) / x.qnorm;
    grad[3] += m[5];
    for (int k = 0; k < 3; ++k) grad[12 + k] += m[6 + k];
}

void orc_grad_abs_map(int64_t N, const float* params, const float* cam, const double* cfg, const double* abs2d,
                      double* out, int nthreads) {
    rcam_t c;
    rcam_setup(&c, cam);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t g = 0; g < N; ++g) {
        double* o = out + 16 * g;
        for (int k = 0; k < 16; ++k) o[k] = 0.0;
        const double* m = abs2d + 9 * g;
        int any = 0;
        for (int k = 0; k < 9; ++k) any |= m[k] != 0.0;
        if (any) project_backward_mag(params + 16 * g, &c, cfg, m, o);
    }
}

/* ------------------------------------------------------------------------ */
/* marginal decisions: every way a lower-precision walk may take them       */

/*
 * The compositing decisions of a pixel (alpha >= alpha_min, T (1 - alpha) <
 * T_min, and for gradients the alpha_max clamp) are taken in FP64 here.  An
 * FP32 implementation evaluates alpha and T with relative errors far below
 * MARGIN_REL, so it can take a decision the other way only where the FP64
 * value lies within MARGIN_REL of its threshold.  walk_from follows the plain
 * definition and, at every such marginal decision, both ways: each complete
 * walk (a "leaf") is a result such an implementation may produce.  The
 * leaves of a pixel are capped at max_leaves (the pixel is then flagged).
 */
typedef struct {
    const proj_t* pr;
    const int64_t* order;
    int64_t V;
    const double* cfg;
    double px, py;
    int grad;        /* also branch on the alpha_max clamp */
    term_t* terms;   /* the composited terms of the walk in progress */
    int64_t cap;
    int nleaves, max_leaves, overflow;
    void (*leaf)(void* ud, const double C[3], const term_t* terms, int64_t n);
    void* ud;
} walk_ctx;

static void emit_leaf(walk_ctx* w, const double C[3], int64_t n) {
    if (++w->nleaves > w->max_leaves) {
        w->overflow = 1;
        return;
    }
    w->leaf(w->ud, C, w->terms, n);
}

static void walk_from(walk_ctx* w, int64_t k, double T, const double C[3], int64_t n);

/* composite term k with the given alpha and clamp state and walk on; or stop
 * before it (T_min), or both when that decision is marginal */
static void take_term(walk_ctx* w, int64_t k, double T, const double C[3], int64_t n, double alpha, double G,
                      double dx, double dy, int clamped) {
    if (w->overflow) return;
    const double tmin = w->cfg[2];
    const double Tn = T * (1.0 - alpha);
    const int near = near_rel(Tn, tmin, MARGIN_REL);
    if (Tn < tmin || near) emit_leaf(w, C, n);
    if (Tn < tmin && !near) return;
    if (n >= w->cap) {
        w->overflow = 1;
        return;
    }
    const proj_t* p = &w->pr[w->order[k]];
    term_t* t = &w->terms[n];
    t->g = w->order[k]; t->alpha = alpha; t->T = T; t->G = G; t->dx = dx; t->dy = dy; t->clamped = clamped;
    double C2[3];
    for (int ch = 0; ch < 3; ++ch) C2[ch] = C[ch] + p->col[ch] * alpha * T;
    walk_from(w, k + 1, Tn, C2, n + 1);
}

/* term k taken, with its clamp as FP64 decides it and, for gradients, also
 * the other way when araw is within the margin of alpha_max */
static void take_alts(walk_ctx* w, int64_t k, double T, const double C[3], int64_t n, double araw, double G,
                      double dx, double dy) {
    const double amax = w->cfg[0];
    const int clamped = araw >= amax;
    take_term(w, k, T, C, n, clamped ? amax : araw, G, dx, dy, clamped);
    if (w->grad && near_rel(araw, amax, MARGIN_REL)) take_term(w, k, T, C, n, clamped ? araw : amax, G, dx, dy, !clamped);
}

static void walk_from(walk_ctx* w, int64_t k, double T, const double C[3], int64_t n) {
    const double amax = w->cfg[0], amin = w->cfg[1];
    for (; k < w->V; ++k) {
        if (w->overflow) return;
        const proj_t* p = &w->pr[w->order[k]];
        const double dx = w->px - p->mx, dy = w->py - p->my;
        const double power = -0.5 * (p->a * dx * dx + p->c * dy * dy) - p->b * dx * dy;
        if (power < p->lthr - 1e-3) continue;
        const double G = exp(power), araw = p->op * G;
        const double alpha = araw < amax ? araw : amax;
        const int marg = near_rel(araw, amin, MARGIN_REL);
        if (!(alpha >= amin)) {
            if (marg) take_alts(w, k, T, C, n, araw, G, dx, dy);  /* FP64 drops it, FP32 may take it */
            continue;
        }
        if (marg) walk_from(w, k + 1, T, C, n);  /* FP64 takes it, FP32 may drop it */
        take_alts(w, k, T, C, n, araw, G, dx, dy);
        return;
    }
    emit_leaf(w, C, n);
}

typedef struct {
    double* out;  /* max_leaves x 3 colours of the pixel */
    int i;
} leaf_colours;

static void leaf_colour(void* ud, const double C[3], const term_t* terms, int64_t n) {
    (void)terms; (void)n;
    leaf_colours* lc = (leaf_colours*)ud;
    for (int ch = 0; ch < 3; ++ch) lc->out[3 * lc->i + ch] = C[ch];
    lc->i++;
}

/*
 * Every result of the window's pixels an implementation may produce by taking
 * marginal decisions either way: leaves (h x w x max_leaves x 3, pixel-major)
 * and their number per pixel in nleaves (h x w; -1: more than max_leaves).
 * Without marginal decisions a pixel has one leaf, orc_render's value.
 */
int orc_render_leaves(int64_t N, const float* params, const float* cam, const double* cfg, int x0, int y0, int w,
                      int h, int max_leaves, double* leaves, int32_t* nleaves, int nthreads) {
    rcam_t c;
    rcam_setup(&c, cam);
    proj_t* pr = (proj_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(proj_t));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!pr || !order) { free(pr); free(order); return 2; }
    const int64_t V = project_sorted(N, params, &c, cfg, pr, order, nthreads);
    int bad = 0;
#pragma omp parallel num_threads(nthreads)
    {
        const int64_t cap = 1 << 16;
        term_t* terms = (term_t*)malloc(sizeof(term_t) * (size_t)cap);
        if (!terms) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int jj = 0; jj < h; ++jj) {
            for (int ii = 0; ii < w; ++ii) {
                if (!terms) continue;
                const long p = (long)jj * w + ii;
                leaf_colours lc = {leaves + (size_t)p * max_leaves * 3, 0};
                walk_ctx wc = {pr, order, V, cfg, x0 + ii + 0.5, y0 + jj + 0.5, 0, terms, cap, 0, max_leaves, 0,
                               leaf_colour, &lc};
                const double C0[3] = {0, 0, 0};
                walk_from(&wc, 0, 1.0, C0, 0);
                nleaves[p] = wc.overflow ? -1 : wc.nleaves;
            }
        }
        free(terms);
    }
    free(pr);
    free(order);
    return bad ? 2 : 0;
}

/* 2D gradient contributions (9 per term, the record of orc_render_backward)
 * of one walk's terms for the pixel gradient gC */
static void walk_terms_backward(const proj_t* pr, const float* params, const term_t* terms, int64_t n,
                                const double gC[3], double* v9) {
    double S[3] = {0, 0, 0};
    for (int64_t k = n - 1; k >= 0; --k) {
        const term_t* t = &terms[k];
        const proj_t* q = &pr[t->g];
        const float* pp = params + 16 * t->g;
        double* v = v9 + 9 * k;
        double dalpha = 0;
        for (int ch = 0; ch < 3; ++ch) {
            v[6 + ch] = pp[12 + ch] > 0.0f ? t->alpha * t->T * gC[ch] : 0.0;
            dalpha += gC[ch] * (q->col[ch] * t->T - S[ch] / (1.0 - t->alpha));
            S[ch] += q->col[ch] * t->alpha * t->T;
        }
        for (int j = 0; j < 6; ++j) v[j] = 0.0;
        if (t->clamped) continue;
        const double dpow = dalpha * t->alpha;
        v[0] = dpow * (q->a * t->dx + q->b * t->dy);
        v[1] = dpow * (q->b * t->dx + q->c * t->dy);
        v[2] = dpow * (-0.5 * t->dx * t->dx);
        v[3] = dpow * (-t->dx * t->dy);
        v[4] = dpow * (-0.5 * t->dy * t->dy);
        v[5] = dalpha * t->G * q->op * (1.0 - q->op);
    }
}

typedef struct {
    int64_t g;
    int leaf;
    double v[9];
} leaf_row;

typedef struct {
    const proj_t* pr;
    const float* params;
    double gC[3];
    leaf_row* rows;
    int64_t nrows, caprows;
    double* v9;  /* scratch: 9 per term */
    int64_t capv;
    int leaf, failed;
} leaf_grads;

static void leaf_grad(void* ud, const double C[3], const term_t* terms, int64_t n) {
    (void)C;
    leaf_grads* lg = (leaf_grads*)ud;
    if (n > lg->capv) {
        double* v = (double*)realloc(lg->v9, sizeof(double) * 9 * (size_t)n);
        if (!v) { lg->failed = 1; return; }
        lg->v9 = v;
        lg->capv = n;
    }
    if (lg->nrows + n > lg->caprows) {
        int64_t c = (lg->nrows + n) * 2;
        leaf_row* r = (leaf_row*)realloc(lg->rows, sizeof(leaf_row) * (size_t)c);
        if (!r) { lg->failed = 1; return; }
        lg->rows = r;
        lg->caprows = c;
    }
    walk_terms_backward(lg->pr, lg->params, terms, n, lg->gC, lg->v9);
    for (int64_t k = 0; k < n; ++k) {
        leaf_row* r = &lg->rows[lg->nrows++];
        r->g = terms[k].g;
        r->leaf = lg->leaf;
        for (int j = 0; j < 9; ++j) r->v[j] = lg->v9[9 * k + j];
    }
    lg->leaf++;
}

static int row_cmp(const void* pa, const void* pb) {
    const leaf_row* a = (const leaf_row*)pa;
    const leaf_row* b = (const leaf_row*)pb;
    return (a->g > b->g) - (a->g < b->g);
}

/*
 * Bounds of the 2D gradient record over every way the window's marginal
 * decisions may be taken: per Gaussian (N x 9, +=), lo2d and hi2d sum over
 * the pixels the smallest and largest contribution among the pixel's leaves
 * (0 where a leaf does not composite the Gaussian); abs2d the largest
 * absolute contribution and nterm the number of contributing pixels (for the
 * rounding bound of an FP32 sum, as in orc_render_backward_ex).  nleaves
 * (h x w): leaves per pixel, -1 beyond max_leaves.  An implementation that
 * takes each pixel's decisions one of these ways has its record, in exact
 * arithmetic, in [lo2d, hi2d].
 */
int orc_render_backward_bounds(int64_t N, const float* params, const float* cam, const double* cfg, int x0, int y0,
                               int w, int h, const double* dL_dimage, int max_leaves, double* lo2d, double* hi2d,
                               double* abs2d, int64_t* nterm, int32_t* nleaves, int nthreads) {
    rcam_t c;
    rcam_setup(&c, cam);
    proj_t* pr = (proj_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(proj_t));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!pr || !order) { free(pr); free(order); return 2; }
    const int64_t V = project_sorted(N, params, &c, cfg, pr, order, nthreads);
    const long WH = (long)w * h;
    int bad = 0;
#pragma omp parallel num_threads(nthreads)
    {
        const int64_t cap = 1 << 16;
        term_t* terms = (term_t*)malloc(sizeof(term_t) * (size_t)cap);
        leaf_grads lg = {pr, params, {0, 0, 0}, NULL, 0, 0, NULL, 0, 0, 0};
#pragma omp for schedule(dynamic, 1)
        for (int jj = 0; jj < h; ++jj) {
            for (int ii = 0; ii < w; ++ii) {
                const long p = (long)jj * w + ii;
                nleaves[p] = 0;
                const double gC[3] = {dL_dimage[p], dL_dimage[WH + p], dL_dimage[2 * WH + p]};
                if (!terms || (gC[0] == 0 && gC[1] == 0 && gC[2] == 0)) continue;
                lg.gC[0] = gC[0]; lg.gC[1] = gC[1]; lg.gC[2] = gC[2];
                lg.nrows = 0;
                lg.leaf = 0;
                walk_ctx wc = {pr, order, V, cfg, x0 + ii + 0.5, y0 + jj + 0.5, 1, terms, cap, 0, max_leaves, 0,
                               leaf_grad, &lg};
                const double C0[3] = {0, 0, 0};
                walk_from(&wc, 0, 1.0, C0, 0);
                if (wc.overflow || lg.failed) {
                    nleaves[p] = -1;
                    continue;
                }
                nleaves[p] = wc.nleaves;
                const int L = wc.nleaves;
                if (L > 1) qsort(lg.rows, (size_t)lg.nrows, sizeof(leaf_row), row_cmp);
                for (int64_t r0 = 0; r0 < lg.nrows;) {
                    int64_t r1 = r0 + 1;
                    while (r1 < lg.nrows && lg.rows[r1].g == lg.rows[r0].g) ++r1;
                    const int64_t g = lg.rows[r0].g;
                    const int in_all = (int)(r1 - r0) == L;
                    for (int j = 0; j < 9; ++j) {
                        double lo = in_all ? lg.rows[r0].v[j] : 0.0, hi = lo, mag = 0.0;
                        for (int64_t r = r0; r < r1; ++r) {
                            const double x = lg.rows[r].v[j];
                            lo = x < lo ? x : lo;
                            hi = x > hi ? x : hi;
                            mag = fabs(x) > mag ? fabs(x) : mag;
                        }
#pragma omp atomic
                        lo2d[9 * g + j] += lo;
#pragma omp atomic
                        hi2d[9 * g + j] += hi;
                        if (abs2d) {
#pragma omp atomic
                            abs2d[9 * g + j] += mag;
                        }
                    }
                    if (nterm) {
#pragma omp atomic
                        nterm[g] += 1;
                    }
                    r0 = r1;
                }
            }
        }
        if (lg.failed || !terms) {
#pragma omp atomic write
            bad = 1;
        }
        free(lg.rows);
        free(lg.v9);
        free(terms);
    }
    free(pr);
    free(order);
    return bad ? 2 : 0;
}

/* the packed parameter gradient of 2D records g2d (N x 9), as the last step
 * of orc_render_backward: grads (N x 16) += project_backward(g2d) */
void orc_project_backward(int64_t N, const float* params, const float* cam, const double* cfg, const double* g2d,
                          double* grads, int nthreads) {
    rcam_t c;
    rcam_setup(&c, cam);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t g = 0; g < N; ++g) {
        const double* a9 = g2d + 9 * g;
        int any = 0;
        for (int k = 0; k < 9; ++k) any |= a9[k] != 0;
        if (any) project_backward_one(params + 16 * g, &c, cfg, a9, grads + 16 * g);
    }
}

/* ------------------------------------------------------------------------ */
/* frozen decisions: finite differences of the backward at scale             */

/*
 * The analytic backward differentiates the render with every threshold
 * decision held fixed: which terms a pixel composites, in which order, where
 * it stops, and which alphas sit at the alpha_max clamp.  A central
 * difference of the plain render itself crosses some decision somewhere once
 * a Gaussian covers thousands of pixels, so the large-scale pin differences
 * the render with those decisions frozen instead.
 *
 * orc_render_lists: for every pixel of the window, the ordered composited
 * Gaussians and their clamp state, written at offsets[p] (offsets: h w + 1
 * prefix sums of the per-pixel term counts that orc_render reports).
 * Returns 0, or 3 if a pixel's term count disagrees with its offsets.
 */
int orc_render_lists(int64_t N, const float* params, const float* cam, const double* cfg, int x0, int y0, int w,
                     int h, const int64_t* offsets, int64_t* list_g, uint8_t* list_clamped, int nthreads) {
    rcam_t c;
    rcam_setup(&c, cam);
    proj_t* pr = (proj_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(proj_t));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!pr || !order) { free(pr); free(order); return 2; }
    int64_t V = project_sorted(N, params, &c, cfg, pr, order, nthreads);
    int bad = 0;
#pragma omp parallel num_threads(nthreads)
    {
        int64_t cap = 4096;
        term_t* terms = (term_t*)malloc(sizeof(term_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
        for (int jj = 0; jj < h; ++jj) {
            for (int ii = 0; ii < w; ++ii) {
                long p = (long)jj * w + ii;
                int64_t want = offsets[p + 1] - offsets[p];
                if (want > cap) {
                    cap = want;
                    terms = (term_t*)realloc(terms, sizeof(term_t) * (size_t)cap);
                }
                double C[3], T;
                int marg;
                int64_t n = walk_pixel(pr, order, V, cfg, x0 + ii + 0.5, y0 + jj + 0.5, C, &T, &marg, terms, cap, 1);
                if (n != want) {
#pragma omp atomic write
                    bad = 1;
                    continue;
                }
                for (int64_t k = 0; k < n; ++k) {
                    list_g[offsets[p] + k] = terms[k].g;
                    list_clamped[offsets[p] + k] = (uint8_t)terms[k].clamped;
                }
            }
        }
        free(terms);
    }
    free(pr);
    free(order);
    return bad ? 3 : 0;
}

/* colour of one pixel over its frozen list; Gaussian `gsub` (or -1) uses
 * the projection *sub instead of its own */
static void frozen_pixel(const proj_t* pr, const int64_t* lg, const uint8_t* lc, int64_t n, const double* cfg,
                         double px, double py, int64_t gsub, const proj_t* sub, double C[3]) {
    double T = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const proj_t* p = lg[k] == gsub ? sub : &pr[lg[k]];
        double dx = px - p->mx, dy = py - p->my;
        double power = -0.5 * (p->a * dx * dx + p->c * dy * dy) - p->b * dx * dy;
        double alpha = lc[k] ? cfg[0] : p->op * exp(power);
        for (int ch = 0; ch < 3; ++ch) C[ch] += p->col[ch] * alpha * T;
        T *= 1.0 - alpha;
    }
}

/*
 * Central differences of F(theta) = sum over the window of v . C(theta)
 * (v: 3 x h x w), decisions frozen as recorded by orc_render_lists: for
 * each requested (Gaussian fd_g[i], packed slot fd_slot[i]) the parameter
 * is stepped to the FP32 values nearest theta +- hstep, and out[i] =
 * (F+ - F-) / (actual step).  Only pixels whose list holds the Gaussian
 * change, so only those are evaluated.  The gradient of F is what the
 * backward computes when handed v as dL/dimage.
 */
int orc_frozen_fd(int64_t N, const float* params, const float* cam, const double* cfg, int x0, int y0, int w, int h,
                  const int64_t* offsets, const int64_t* list_g, const uint8_t* list_clamped, const double* v,
                  int32_t n_fd, const int64_t* fd_g, const int32_t* fd_slot, double hstep, double* out,
                  int nthreads) {
    rcam_t c;
    rcam_setup(&c, cam);
    proj_t* pr = (proj_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(proj_t));
    if (!pr) return 2;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t g = 0; g < N; ++g) project_one(params + 16 * g, &c, cfg, &pr[g], NULL);
    long WH = (long)w * h;
    for (int32_t i = 0; i < n_fd; ++i) {
        int64_t g = fd_g[i];
        float pp[16], pm[16];
        memcpy(pp, params + 16 * g, sizeof pp);
        memcpy(pm, params + 16 * g, sizeof pm);
        pp[fd_slot[i]] = (float)((double)pp[fd_slot[i]] + hstep);
        pm[fd_slot[i]] = (float)((double)pm[fd_slot[i]] - hstep);
        double step = (double)pp[fd_slot[i]] - (double)pm[fd_slot[i]];
        proj_t plus, minus;
        memset(&plus, 0, sizeof plus);
        memset(&minus, 0, sizeof minus);
        project_one(pp, &c, cfg, &plus, NULL);
        project_one(pm, &c, cfg, &minus, NULL);
        double acc = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : acc) num_threads(nthreads)
        for (long p = 0; p < WH; ++p) {
            int64_t o = offsets[p], n = offsets[p + 1] - offsets[p];
            int has = 0;
            for (int64_t k = 0; k < n && !has; ++k) has = list_g[o + k] == g;
            if (!has) continue;
            double px = x0 + (p % w) + 0.5, py = y0 + (p / w) + 0.5, Cp[3], Cm[3];
            frozen_pixel(pr, list_g + o, list_clamped + o, n, cfg, px, py, g, &plus, Cp);
            frozen_pixel(pr, list_g + o, list_clamped + o, n, cfg, px, py, g, &minus, Cm);
            for (int ch = 0; ch < 3; ++ch) acc += v[ch * WH + p] * (Cp[ch] - Cm[ch]);
        }
        out[i] = acc / step;
    }
    free(pr);
    return 0;
}

/*
 * The frozen-decision render itself (for the check that it reproduces
 * orc_render at the recorded parameters).  image: 3 x h x w.
 */
int orc_render_frozen(int64_t N, const float* params, const float* cam, const double* cfg, int x0, int y0, int w,
                      int h, const int64_t* offsets, const int64_t* list_g, const uint8_t* list_clamped,
                      double* image, int nthreads) {
    rcam_t c;
    rcam_setup(&c, cam);
    proj_t* pr = (proj_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(proj_t));
    if (!pr) return 2;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t g = 0; g < N; ++g) project_one(params + 16 * g, &c, cfg, &pr[g], NULL);
    long WH = (long)w * h;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (long p = 0; p < WH; ++p) {
        double C[3];
        frozen_pixel(pr, list_g + offsets[p], list_clamped + offsets[p], offsets[p + 1] - offsets[p], cfg,
                     x0 + (p % w) + 0.5, y0 + (p / w) + 0.5, -1, NULL, C);
        for (int ch = 0; ch < 3; ++ch) image[ch * WH + p] = C[ch];
    }
    free(pr);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* losses                                                                    */

/*
 * HDR loss of Sec. 3.6: mean over the k = C h w crop elements of
 * (x - y)^2 / (y + 0.01)^2 with x the (noisy) target and y the prediction.
 * full_grad = 0 treats the denominator as a constant (stop-gradient),
 * 1 differentiates it too.  crop = {x0, y0, w, h} or NULL (whole image);
 * dL_dpred is zero outside the crop.
 */
double orc_loss_hdr(const float* pred, const float* target, int C, int H, int W, const int* crop, int full_grad,
                    double* dL_dpred) {
    int x0 = 0, y0 = 0, w = W, h = H;
    if (crop) { x0 = crop[0]; y0 = crop[1]; w = crop[2]; h = crop[3]; }
    double k = (double)C * w * h, loss = 0;
    if (dL_dpred) memset(dL_dpred, 0, sizeof(double) * (size_t)C * H * W);
    for (int ch = 0; ch < C; ++ch)
        for (int j = y0; j < y0 + h; ++j)
            for (int i = x0; i < x0 + w; ++i) {
                long p = ((long)ch * H + j) * W + i;
                double y = pred[p], x = target[p], den = y + 0.01;
                loss += (x - y) * (x - y) / (den * den);
                if (dL_dpred) {
                    double g = 2.0 * (y - x) / (den * den);
                    if (full_grad) g -= 2.0 * (x - y) * (x - y) / (den * den * den);
                    dL_dpred[p] = g / k;
                }
            }
    return loss / k;
}

/* 11-tap Gaussian window, sigma 1.5, normalised to sum 1 */
static void ssim_window(double wnd[11]) {
    double s = 0;
    for (int i = 0; i < 11; ++i) { wnd[i] = exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)); s += wnd[i]; }
    for (int i = 0; i < 11; ++i) wnd[i] /= s;
}

/* zero-padded 'same' 2D filtering with the separable window (it is symmetric,
   so correlation and convolution coincide) */
static void filter2(const double* in, double* out, int h, int w, const double wnd[11]) {
    double* tmp = (double*)calloc((size_t)h * w, sizeof(double));
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            double acc = 0;
            for (int k = -5; k <= 5; ++k) {
                int ii = i + k;
                if (ii >= 0 && ii < w) acc += wnd[k + 5] * in[(long)j * w + ii];
            }
            tmp[(long)j * w + i] = acc;
        }
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            double acc = 0;
            for (int k = -5; k <= 5; ++k) {
                int jj = j + k;
                if (jj >= 0 && jj < h) acc += wnd[k + 5] * tmp[(long)jj * w + i];
            }
            out[(long)j * w + i] = acc;
        }
    free(tmp);
}

/*
 * 0.8 L1 + 0.2 (1 - SSIM) over the crop (treated as its own zero-padded
 * image), SSIM of Wang et al. 2004 per channel with an 11x11 Gaussian
 * window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, mean over channels and
 * pixels.  ssim_map (optional): C x h x w.
 */
double orc_loss_l1ssim(const float* pred, const float* target, int C, int H, int W, const int* crop,
                       double* dL_dpred, double* ssim_map) {
    int x0 = 0, y0 = 0, w = W, h = H;
    if (crop) { x0 = crop[0]; y0 = crop[1]; w = crop[2]; h = crop[3]; }
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double wnd[11];
    ssim_window(wnd);
    long n = (long)w * h;
    double k = (double)C * n;
    double l1 = 0, ssim_sum = 0;
    if (dL_dpred) memset(dL_dpred, 0, sizeof(double) * (size_t)C * H * W);
    double* buf = (double*)malloc(sizeof(double) * (size_t)n * 13);
    double *x = buf, *y = buf + n, *xx = buf + 2 * n, *yy = buf + 3 * n, *xy = buf + 4 * n;
    double *mx = buf + 5 * n, *my = buf + 6 * n, *exx = buf + 7 * n, *eyy = buf + 8 * n, *exy = buf + 9 * n;
    double *gmu = buf + 10 * n, *gxx = buf + 11 * n, *gxy = buf + 12 * n;
    for (int ch = 0; ch < C; ++ch) {
        for (int j = 0; j < h; ++j)
            for (int i = 0; i < w; ++i) {
                long p = ((long)ch * H + (y0 + j)) * W + (x0 + i), q = (long)j * w + i;
                x[q] = pred[p]; y[q] = target[p];
                xx[q] = x[q] * x[q]; yy[q] = y[q] * y[q]; xy[q] = x[q] * y[q];
                double d = x[q] - y[q];
                l1 += fabs(d);
                if (dL_dpred) dL_dpred[p] = 0.8 * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / k;
            }
        filter2(x, mx, h, w, wnd);
        filter2(y, my, h, w, wnd);
        filter2(xx, exx, h, w, wnd);
        filter2(yy, eyy, h, w, wnd);
        filter2(xy, exy, h, w, wnd);
        for (long q = 0; q < n; ++q) {
            double sxx = exx[q] - mx[q] * mx[q], syy = eyy[q] - my[q] * my[q], sxy = exy[q] - mx[q] * my[q];
            double A1 = 2 * mx[q] * my[q] + C1, A2 = 2 * sxy + C2;
            double B1 = mx[q] * mx[q] + my[q] * my[q] + C1, B2 = sxx + syy + C2;
            double s = (A1 * A2) / (B1 * B2);
            ssim_sum += s;
            if (ssim_map) ssim_map[(long)ch * n + q] = s;
            /* partials of s w.r.t. mu_x, E[x^2], E[xy] (mu_y, E[y^2] are constants) */
            double dA1 = 2 * my[q], dA2 = -2 * my[q], dB1 = 2 * mx[q], dB2 = -2 * mx[q];
            gmu[q] = (dA1 * A2 + A1 * dA2) / (B1 * B2) - s * (dB1 * B2 + B1 * dB2) / (B1 * B2);
            gxx[q] = -s / B2;
            gxy[q] = 2 * A1 / (B1 * B2);
        }
        if (dL_dpred) {
            /* d mean(s) / d x_q = (w * gmu)(q) + 2 x_q (w * gxx)(q) + y_q (w * gxy)(q), over n */
            filter2(gmu, mx, h, w, wnd);
            filter2(gxx, exx, h, w, wnd);
            filter2(gxy, exy, h, w, wnd);
            for (int j = 0; j < h; ++j)
                for (int i = 0; i < w; ++i) {
                    long p = ((long)ch * H + (y0 + j)) * W + (x0 + i), q = (long)j * w + i;
                    double ds = mx[q] + 2 * x[q] * exx[q] + y[q] * exy[q];
                    dL_dpred[p] += -0.2 * ds / k;
                }
        }
    }
    free(buf);
    return 0.8 * l1 / k + 0.2 * (1.0 - ssim_sum / k);
}

/* ------------------------------------------------------------------------ */
/* AdamW (Sec. 3.6 "Regularization"; Loshchilov & Hutter's decoupled decay)  */
/* per element e of slot e % 16: lr_e = lr[slot] * lr_scale;                */
/* m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;                               */
/* p -= lr_e (m / (1-b1^t) / (sqrt(v / (1-b2^t)) + eps) + wd p); g = 0.      */
/* Slots with lr 0 are left untouched (no decay).                           */

void orc_adamw(int64_t n, double* p, double* g, double* m, double* v, const double* lr, double lr_scale,
               double b1, double b2, double eps, double wd, int step) {
    double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
    for (int64_t e = 0; e < n; ++e) {
        double lre = lr[e % 16] * lr_scale;
        if (lre != 0.0) {
            m[e] = b1 * m[e] + (1.0 - b1) * g[e];
            v[e] = b2 * v[e] + (1.0 - b2) * g[e] * g[e];
            double mh = m[e] / bc1, vh = v[e] / bc2;
            p[e] -= lre * (mh / (sqrt(vh) + eps) + wd * p[e]);
        }
        g[e] = 0.0;
    }
}

/* Eq. 4: eta_t = eta_0 / (1 + ln t), t >= 1 frames of a static viewport */
double orc_lr_scale(int t) { return 1.0 / (1.0 + log((double)(t < 1 ? 1 : t))); }

/* cache memory of Table 3: 14 FP32 attributes per Gaussian */
int64_t orc_cache_bytes(int64_t n) { return n * 14 * 4; }
