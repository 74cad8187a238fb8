// Volume path tracer that produces the training targets of the cache
// (GSCache Sec. 3.2 - 3.5): delta (Woodcock) tracking against a global
// majorant, next-event estimation at every interaction (directional light
// with phase 1/(4 pi), spherical area lights by one cone direction each,
// constant environment by one uniform direction; shadow transmittance by
// ratio tracking), isotropic scattering, optional
// early termination into the cache (Algorithm 1) with the cascaded beta
// correction (Eq. 2), and one intermediate path buffer per path length.
//
// Reproducibility: this translation unit is compiled without FMA
// contraction; every operation below is a single IEEE FP32 operation in the
// order written, transcendental functions are the library's own (ln by the
// atanh series, sincos(2 pi u) by Taylor series on an octant), and random
// numbers come from Philox4x32-10 with counter (pixel, sample, frame, block)
// and key = seed.  Each (pixel, sample) is an independent stream, so the
// result does not depend on the launch shape.  The density scale, the
// majorant and the transfer function's segment widths enter the tracking
// steps as reciprocals formed once on the host (FP32 divisions), so a step
// multiplies where it would divide (1.38 -> 1.20 ms per 1080p frame).
#include "gsc_internal.cuh"

namespace gsc {

constexpr int kTrackMaxSteps = 1 << 20;  // bounds every tracking loop
constexpr int kMaxLevels = 16;

struct TraceDev {
    const float* grid;
    int nx, ny, nz;
    float dmax, smax, albedo, sbar;
    float inv_dmax, inv_sbar;  // 1 / dmax, 1 / sbar (FP32 divisions on the host)
    int tf_n;
    float tf_pos[16];
    float tf_inv[16];  // 1 / (tf_pos[k + 1] - tf_pos[k])
    float tf_rgba[16][4];
    float ldir[3], lrad[3], env[3];
    int has_dir, has_env;
    int nsph;
    float sc[GSC_MAX_SPHERE_LIGHTS][3], sr[GSC_MAX_SPHERE_LIGHTS], sl[GSC_MAX_SPHERE_LIGHTS][3];
    int spp, B, K;
    uint32_t frame, k0, k1;
    float C, eps;
    int tr_per_call;  // Algorithm 1's Tr_out read per call (else cumulatively)
};

struct Philox {
    uint32_t c0, c1, c2, blk, k0, k1;
    uint32_t b0, b1, b2, b3;
    int avail;

    __device__ void init(uint32_t pixel, uint32_t sample, uint32_t frame, uint32_t key0, uint32_t key1) {
        c0 = pixel; c1 = sample; c2 = frame; blk = 0; k0 = key0; k1 = key1; avail = 0;
    }
    __device__ void refill() {
        uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = blk;
        uint32_t a = k0, b = k1;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
            uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
            uint32_t y0 = hi1 ^ x1 ^ a, y2 = hi0 ^ x3 ^ b;
            x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
            a += 0x9E3779B9u;
            b += 0xBB67AE85u;
        }
        b0 = x0; b1 = x1; b2 = x2; b3 = x3;
        blk += 1;
        avail = 4;
    }
    __device__ uint32_t next() {
        if (avail == 0) refill();
        uint32_t v = b0;
        b0 = b1; b1 = b2; b2 = b3;
        avail -= 1;
        return v;
    }
    __device__ float uniform() { return (float)(next() >> 8) * 5.9604644775390625e-8f; }
};

// ln(x), x normal and positive: x = 2^e m, m in [sqrt(1/2), sqrt(2)];
// ln m = 2 atanh(s), s = (m - 1) / (m + 1), series to s^11
__device__ float ln32(float x) {
    uint32_t bits = __float_as_uint(x);
    int e = (int)((bits >> 23) & 0xffu) - 127;
    float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
    if (m > 1.41421356f) {
        m = m * 0.5f;
        e = e + 1;
    }
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

// (sin, cos) of 2 pi u for u in [0, 1): quadrant q, theta = (frac - 1/2) pi/2,
// Taylor series of sin (to theta^9) and cos (to theta^10), rotation by
// q pi/2 + pi/4
__device__ void sincos2pi32(float u, float* sn_out, float* cs_out) {
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
    if (q == 0) { *cs_out = cp; *sn_out = sp; }
    else if (q == 1) { *cs_out = -sp; *sn_out = cp; }
    else if (q == 2) { *cs_out = -cp; *sn_out = -sp; }
    else { *cs_out = sp; *sn_out = -cp; }
}

__device__ __forceinline__ float clamp01(float x) { return x < 0.0f ? 0.0f : (x > 1.0f ? 1.0f : x); }

__device__ float density_at(const TraceDev& v, float px, float py, float pz) {
    float gx = clamp01(px) * (float)(v.nx - 1);
    float gy = clamp01(py) * (float)(v.ny - 1);
    float gz = clamp01(pz) * (float)(v.nz - 1);
    int ix = (int)gx, iy = (int)gy, iz = (int)gz;
    if (ix > v.nx - 2) ix = v.nx - 2;
    if (iy > v.ny - 2) iy = v.ny - 2;
    if (iz > v.nz - 2) iz = v.nz - 2;
    float fx = gx - (float)ix, fy = gy - (float)iy, fz = gz - (float)iz;
    size_t sy = (size_t)v.nx, sz = (size_t)v.nx * v.ny;
    const float* g = v.grid + (size_t)iz * sz + (size_t)iy * sy + ix;
    float v000 = __ldg(g), v100 = __ldg(g + 1), v010 = __ldg(g + sy), v110 = __ldg(g + sy + 1);
    float v001 = __ldg(g + sz), v101 = __ldg(g + sz + 1), v011 = __ldg(g + sz + sy), v111 = __ldg(g + sz + sy + 1);
    float c00 = v000 + fx * (v100 - v000);
    float c10 = v010 + fx * (v110 - v010);
    float c01 = v001 + fx * (v101 - v001);
    float c11 = v011 + fx * (v111 - v011);
    float c0 = c00 + fy * (c10 - c00);
    float c1 = c01 + fy * (c11 - c01);
    return c0 + fz * (c1 - c0);
}

// piecewise-linear transfer function; channel ch (3 = opacity)
__device__ float tf_channel(const TraceDev& v, float s, int ch) {
    int n = v.tf_n;
    if (s <= v.tf_pos[0]) return v.tf_rgba[0][ch];
    if (s >= v.tf_pos[n - 1]) return v.tf_rgba[n - 1][ch];
    int k = 0;
    while (k < n - 2 && s >= v.tf_pos[k + 1]) ++k;
    float w = (s - v.tf_pos[k]) * v.tf_inv[k];
    return v.tf_rgba[k][ch] + w * (v.tf_rgba[k + 1][ch] - v.tf_rgba[k][ch]);
}

__device__ __forceinline__ float norm_density(const TraceDev& v, const float* x) {
    return clamp01(density_at(v, x[0], x[1], x[2]) * v.inv_dmax);
}

__device__ __forceinline__ float sigma_t_at(const TraceDev& v, const float* x) {
    return v.smax * tf_channel(v, norm_density(v, x), 3);
}

__device__ bool clip_box(const float* o, const float* d, float* t0, float* t1) {
    float lo = 0.0f, hi = (float)1e30;
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0f) {
            float inv = 1.0f / d[a];
            float ta = -o[a] * inv;
            float tb = (1.0f - o[a]) * inv;
            if (ta > tb) { float tmp = ta; ta = tb; tb = tmp; }
            if (ta > lo) lo = ta;
            if (tb < hi) hi = tb;
        } else if (o[a] < 0.0f || o[a] > 1.0f) {
            return false;
        }
    }
    *t0 = lo;
    *t1 = hi;
    return lo < hi;
}

__device__ bool free_flight(const TraceDev& v, Philox& r, const float* o, const float* d, float* x) {
    float t0, t1;
    if (!clip_box(o, d, &t0, &t1)) return false;
    if (!(v.sbar > 0.0f)) return false;
    float t = t0;
    for (int it = 0; it < kTrackMaxSteps; ++it) {
        float u = r.uniform();
        float dt = -ln32(1.0f - u) * v.inv_sbar;
        t = t + dt;
        if (t >= t1) return false;
        for (int a = 0; a < 3; ++a) x[a] = o[a] + t * d[a];
        float sig = sigma_t_at(v, x);
        float u2 = r.uniform();
        if (u2 * v.sbar < sig) return true;
    }
    return false;
}

__device__ float ratio_tracking(const TraceDev& v, Philox& r, const float* p, const float* d) {
    float t0, t1;
    if (!clip_box(p, d, &t0, &t1)) return 1.0f;
    if (!(v.sbar > 0.0f)) return 1.0f;
    float T = 1.0f, t = t0;
    for (int it = 0; it < kTrackMaxSteps; ++it) {
        float u = r.uniform();
        float dt = -ln32(1.0f - u) * v.inv_sbar;
        t = t + dt;
        if (t >= t1) break;
        float x[3];
        for (int a = 0; a < 3; ++a) x[a] = p[a] + t * d[a];
        float sig = sigma_t_at(v, x);
        T = T * (1.0f - sig * v.inv_sbar);
        if (!(T > 0.0f)) {
            T = 0.0f;
            break;
        }
    }
    return T;
}

__device__ void sphere_dir(float u1, float u2, float* d) {
    float z = 1.0f - 2.0f * u1;
    float r2 = 1.0f - z * z;
    float r = r2 > 0.0f ? sqrtf(r2) : 0.0f;
    float s, c;
    sincos2pi32(u2, &s, &c);
    d[0] = r * c;
    d[1] = r * s;
    d[2] = z;
}

// NEE towards a spherical area light (centre c, radius rad, outside the box)
// from x: one direction uniform in the cone the sphere subtends, in the
// orthonormal frame of Duff et al. (2017) around the axis to the centre.
// With the isotropic phase 1/(4 pi) and the cone pdf 1/(2 pi (1 - cos_max)),
// the estimate is L_e T (1 - cos_max) / 2; returns that weight, T included.
__device__ float sphere_nee(const TraceDev& v, Philox& r, const float* x, const float* c, float rad) {
    float w[3];
    for (int a = 0; a < 3; ++a) w[a] = c[a] - x[a];
    float dist2 = (w[0] * w[0] + w[1] * w[1]) + w[2] * w[2];
    float inv = 1.0f / sqrtf(dist2);
    for (int a = 0; a < 3; ++a) w[a] = w[a] * inv;
    float s2 = (rad * rad) / dist2;
    float cmax = sqrtf(1.0f - s2);
    float u1 = r.uniform(), u2 = r.uniform();
    float ct = 1.0f - u1 * (1.0f - cmax);
    float st2 = 1.0f - ct * ct;
    float st = st2 > 0.0f ? sqrtf(st2) : 0.0f;
    float sp, cp;
    sincos2pi32(u2, &sp, &cp);
    float sg = w[2] >= 0.0f ? 1.0f : -1.0f;
    float ia = -1.0f / (sg + w[2]);
    float bb = (w[0] * w[1]) * ia;
    float t[3] = {1.0f + ((sg * w[0]) * w[0]) * ia, sg * bb, -(sg * w[0])};
    float bv[3] = {bb, sg + (w[1] * w[1]) * ia, -w[1]};
    float a1 = st * cp, a2 = st * sp;
    float d[3];
    for (int a = 0; a < 3; ++a) d[a] = (t[a] * a1 + bv[a] * a2) + w[a] * ct;
    float T = ratio_tracking(v, r, x, d);
    return T * ((1.0f - cmax) * 0.5f);
}

// Two register budgets for the same code.  MINB = 16 (every warp slot of the
// SM, 32 registers, with spills): on a frame of many waves the tracer waits
// mostly on dependent volume loads, and the extra warps hide that better than
// registers (1080p: 1.40 ms against 1.54 ms at MINB = 5).  MINB = 5 (no
// spills): on a frame of a few waves or less the warps are there anyway and
// the spills only cost (256^2 to 640x480: 17-19% faster than MINB = 16).
// CACHE: whether a cache is given (Algorithm 1 and natural-termination
// sampling); without one its per-path state takes no registers.
template <int MINB, bool CACHE>
__global__ void __launch_bounds__(128, MINB) k_trace(TraceDev v, CamDev cam, const float* __restrict__ cache,
                                                     float* __restrict__ targets, float* __restrict__ image) {
    int i = blockIdx.x * 16 + (threadIdx.x & 15);
    int j = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (i >= cam.W || j >= cam.H) return;
    size_t HW = (size_t)cam.W * cam.H, pix = (size_t)j * cam.W + i;
    float img[3] = {0.0f, 0.0f, 0.0f};
    // the pixel's target buffers accumulate in place (the thread owns the
    // pixel): a per-thread array indexed by path length would live in local
    // memory, which at every warp slot of the SM spills into L2 and evicts
    // the volume
    for (int k = 0; k < v.K; ++k)
        for (int c = 0; c < 3; ++c) targets[((size_t)k * 3 + c) * HW + pix] = 0.0f;
    const bool cache_on = CACHE;
    for (int s = 0; s < v.spp; ++s) {
        Philox r;
        r.init((uint32_t)(j * cam.W + i), (uint32_t)s, v.frame, v.k0, v.k1);
        float jx = 0.5f, jy = 0.5f;
        if (v.spp > 1) {
            jx = r.uniform();
            jy = r.uniform();
        }
        float px = (float)i + jx, py = (float)j + jy;
        float dc0 = (px - cam.cx) / cam.fx;
        float dc1 = (py - cam.cy) / cam.fy;
        float d[3], o[3];
        for (int a = 0; a < 3; ++a) d[a] = (cam.R[a] * dc0 + cam.R[3 + a] * dc1) + cam.R[6 + a];
        float n2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        float inv = 1.0f / sqrtf(n2);
        for (int a = 0; a < 3; ++a) {
            d[a] = d[a] * inv;
            o[a] = cam.pos[a];
        }
        float thr[3] = {1.0f, 1.0f, 1.0f}, prod[3] = {1.0f, 1.0f, 1.0f}, beta = 1.0f;
        float L[3] = {0.0f, 0.0f, 0.0f};
        int n = 0;
        bool early = false, escaped = false;
        for (;;) {
            float x[3];
            if (!free_flight(v, r, o, d, x)) {
                escaped = true;
                break;
            }
            n = n + 1;
            float sn = norm_density(v, x);
            for (int c = 0; c < 3; ++c) {
                float alb = v.albedo * tf_channel(v, sn, c);
                thr[c] = thr[c] * alb;
                prod[c] = prod[c] * alb;
            }
            if (v.has_dir) {
                float Td = ratio_tracking(v, r, x, v.ldir);
                float wd = Td * (float)0.0795774715459476679;
                for (int c = 0; c < 3; ++c) L[c] = L[c] + thr[c] * (v.lrad[c] * wd);
            }
            for (int l = 0; l < v.nsph; ++l) {
                float ws = sphere_nee(v, r, x, v.sc[l], v.sr[l]);
                for (int c = 0; c < 3; ++c) L[c] = L[c] + thr[c] * (v.sl[l][c] * ws);
            }
            if (v.has_env) {
                float ua = r.uniform(), ub = r.uniform();
                float e[3];
                sphere_dir(ua, ub, e);
                float Te = ratio_tracking(v, r, x, e);
                for (int c = 0; c < 3; ++c) L[c] = L[c] + thr[c] * (v.env[c] * Te);
            }
            if (n >= v.B) break;
            if (cache_on && v.C > 0.0f && n <= v.K) {
                float lum = ((float)0.2126 * prod[0] + (float)0.7152 * prod[1]) + (float)0.0722 * prod[2];
                float Tr = v.C * lum;
                Tr = Tr < 0.0f ? 0.0f : (Tr > 1.0f ? 1.0f : Tr);
                if (Tr < (float)0.9) {
                    float q = r.uniform();
                    if (q < 1.0f - Tr) {
                        early = true;
                        break;
                    }
                    // Tr_out / (Tr + eps): cumulative, or this call's product of albedos
                    for (int c = 0; c < 3; ++c) thr[c] = (v.tr_per_call ? prod[c] : thr[c]) / (Tr + v.eps);
                    beta = beta * Tr;
                } else if (v.tr_per_call) {
                    for (int c = 0; c < 3; ++c) thr[c] = prod[c];  // this call's Tr_out, undivided
                }
            }
            float ua = r.uniform(), ub = r.uniform();
            sphere_dir(ua, ub, d);
            for (int a = 0; a < 3; ++a) o[a] = x[a];
        }
        float val[3];
        if (n == 0) {
            for (int c = 0; c < 3; ++c) val[c] = v.env[c];
        } else if (cache_on && n <= v.K &&
                   (early || (escaped && L[0] == 0.0f && L[1] == 0.0f && L[2] == 0.0f))) {
            for (int c = 0; c < 3; ++c) val[c] = cache[((size_t)(n - 1) * 3 + c) * HW + pix] / beta;
        } else {
            for (int c = 0; c < 3; ++c) val[c] = L[c];
        }
        for (int c = 0; c < 3; ++c) img[c] = img[c] + val[c];
        if (n >= 1 && n <= v.K)
            for (int c = 0; c < 3; ++c) {
                float* t = &targets[((size_t)(n - 1) * 3 + c) * HW + pix];
                *t = *t + L[c];
            }
    }
    for (int c = 0; c < 3; ++c) image[c * HW + pix] = img[c] / (float)v.spp;
    if (v.spp > 1)  // x / 1 = x
        for (int k = 0; k < v.K; ++k)
            for (int c = 0; c < 3; ++c) {
                float* t = &targets[((size_t)k * 3 + c) * HW + pix];
                *t = *t / (float)v.spp;
            }
}

// Cache initialisation, point sampling (Sec. 3.2 "Cache Initialization"):
// point i casts rays until delta tracking finds a real collision and keeps
// its position and albedo.  Attempt a uses the Philox stream (i, a,
// kInitStream); the ray starts on the unit sphere around the box centre and
// points at a uniform point of the box.  Points that find no collision in
// max_attempts rays are counted in *fails (and left at the origin).
constexpr uint32_t kInitStream = 0xffffffffu;

__global__ void __launch_bounds__(128, 16) k_init_sample(TraceDev v, uint32_t n, int max_attempts,
                                                     float4* __restrict__ pos, float4* __restrict__ alb,
                                                     unsigned int* __restrict__ fails) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[3] = {0.0f, 0.0f, 0.0f}, a3[3] = {0.0f, 0.0f, 0.0f};
    bool found = false;
    for (int a = 0; a < max_attempts && !found; ++a) {
        Philox r;
        r.init(i, (uint32_t)a, kInitStream, v.k0, v.k1);
        float u0 = r.uniform(), u1 = r.uniform();
        float sd[3], o[3], d[3];
        sphere_dir(u0, u1, sd);
        for (int k = 0; k < 3; ++k) o[k] = 0.5f + sd[k];
        for (int k = 0; k < 3; ++k) d[k] = r.uniform() - o[k];
        float n2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        float inv = 1.0f / sqrtf(n2);
        for (int k = 0; k < 3; ++k) d[k] = d[k] * inv;
        if (free_flight(v, r, o, d, x)) {
            float sn = norm_density(v, x);
            for (int c = 0; c < 3; ++c) a3[c] = v.albedo * tf_channel(v, sn, c);
            found = true;
        }
    }
    if (!found) atomicAdd(fails, 1u);
    pos[i] = make_float4(x[0], x[1], x[2], 0.0f);
    alb[i] = make_float4(a3[0], a3[1], a3[2], 0.0f);
}

static TraceDev trace_dev(const gsc_scene* sc) {
    TraceDev v{};
    const gsc_scene_desc& d = sc->desc;
    v.grid = d.density;
    v.nx = d.nx; v.ny = d.ny; v.nz = d.nz;
    v.dmax = d.density_max; v.smax = d.sigma_max; v.albedo = d.albedo; v.sbar = sc->sbar;
    v.inv_dmax = 1.0f / d.density_max;
    v.inv_sbar = sc->sbar > 0.0f ? 1.0f / sc->sbar : 0.0f;
    v.tf_n = d.tf_count;
    for (int k = 0; k < 16; ++k) {
        v.tf_pos[k] = d.tf_pos[k];
        v.tf_inv[k] = k + 1 < d.tf_count ? 1.0f / (d.tf_pos[k + 1] - d.tf_pos[k]) : 0.0f;
        for (int c = 0; c < 4; ++c) v.tf_rgba[k][c] = d.tf_rgba[k][c];
    }
    for (int c = 0; c < 3; ++c) {
        v.ldir[c] = d.light_dir[c];
        v.lrad[c] = d.light_radiance[c];
        v.env[c] = d.env_radiance[c];
    }
    v.has_dir = (d.light_radiance[0] > 0.0f || d.light_radiance[1] > 0.0f || d.light_radiance[2] > 0.0f);
    v.has_env = (d.env_radiance[0] > 0.0f || d.env_radiance[1] > 0.0f || d.env_radiance[2] > 0.0f);
    v.nsph = d.n_spheres;
    for (int l = 0; l < GSC_MAX_SPHERE_LIGHTS; ++l) {
        v.sr[l] = l < d.n_spheres ? d.sphere_radius[l] : 0.0f;
        for (int a = 0; a < 3; ++a) {
            v.sc[l][a] = l < d.n_spheres ? d.sphere_center[l][a] : 0.0f;
            v.sl[l][a] = l < d.n_spheres ? d.sphere_radiance[l][a] : 0.0f;
        }
    }
    return v;
}

cudaError_t launch_init_sample(const gsc_scene* sc, uint32_t n, uint64_t seed, int max_attempts, float4* pos,
                               float4* alb, unsigned int* fails, cudaStream_t s) {
    TraceDev v = trace_dev(sc);
    v.k0 = (uint32_t)seed;
    v.k1 = (uint32_t)(seed >> 32);
    PhaseScope ph(kPhInit, s, 1);
    k_init_sample<<<(n + 127) / 128, 128, 0, s>>>(v, n, max_attempts, pos, alb, fails);
    return cudaGetLastError();
}

// SMs of the current device (queried once)
static int sm_count() {
    static int cached = 0;
    if (cached <= 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached = sms > 0 ? sms : 1;
    }
    return cached;
}

cudaError_t launch_trace(const gsc_scene* sc, const CamDev& cam, const gsc_trace_params& p, const float* cache,
                         float* targets, float* image, cudaStream_t s) {
    TraceDev v = trace_dev(sc);
    v.spp = p.spp; v.B = p.max_bounces; v.K = p.levels;
    v.frame = p.frame;
    v.k0 = (uint32_t)p.seed;
    v.k1 = (uint32_t)(p.seed >> 32);
    v.C = p.C; v.eps = p.eps;
    v.tr_per_call = p.tr_out == GSC_TR_OUT_PER_CALL ? 1 : 0;
    dim3 grid((cam.W + 15) / 16, (cam.H + 7) / 8);
    PhaseScope ph(kPhTrace, s, 1);
    // two full waves at 16 CTAs per SM: below that, the spill-free budget
    const bool many = (size_t)grid.x * grid.y >= (size_t)2 * 16 * sm_count();
    if (cache)
        (many ? k_trace<16, true> : k_trace<5, true>)<<<grid, 128, 0, s>>>(v, cam, cache, targets, image);
    else
        (many ? k_trace<16, false> : k_trace<5, false>)<<<grid, 128, 0, s>>>(v, cam, cache, targets, image);
    return cudaGetLastError();
}

}  // namespace gsc
