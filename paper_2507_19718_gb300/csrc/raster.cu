// Tile-based Gaussian splatting of one cache level and its gradient
// (Sec. 3.1 / 3.5 of GSCache, which renders each level with the 3D Gaussian
// splatting rasterizer at SH degree 0, Sec. 3.6).
//
// Forward:  k_project  -> depth radix sort (one sweep) -> scan of bin counts -> k_emit
//           (a pair per bin of the tile rectangle; a bin the falloff bound
//           cannot reach gets a key past every bin)
//           -> stable radix sort of the (bin, Gaussian) pairs by bin
//           -> bin ranges and tile order (k_tile_order; k_ranges first when
//           the pair sort took more than one pass; with feedback from the
//           last gradient launch k_tile_cost, k_tile_class before and
//           k_tile_scatter after it) -> k_render (each tile filters its
//           bin's list)
// Backward: the same binning (no per-pixel state is kept from the forward),
//           k_render_bwd (forward re-walk for the final T and the last
//           composited entry, then back to front), k_project_bwd.
// Training step: the same binning, k_render_bwd with the HDR loss folded in,
//           k_project_bwd_step (parameter gradients + AdamW; its first
//           blocks sum the views' losses).
//
// The compositing decisions (alpha >= alpha_min, T (1 - alpha) < T_min) are
// computed by one inline function with explicitly rounded operations, so the
// forward and the backward take them identically.  A Gaussian is binned into
// every tile its alpha >= alpha_min support can reach (the bounding box of
// that ellipse, then the exact bound per bin and per tile), which makes
// every pixel's ordered list independent of the tile shape: images are
// bit-identical for any tile size.
#include <math.h>

#include "gsc_internal.cuh"

namespace gsc {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// reciprocal to about one ulp, enough for the gradient arithmetic (never
// for a compositing decision)
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// FP32 view depth with a fixed operation order ((r20 x + r21 y) + r22 z) + t2;
// it is the sort key and the near-plane test.
__device__ __forceinline__ float view_depth(const CamDev& c, float x, float y, float z) {
    float s = __fadd_rn(__fmul_rn(c.R[6], x), __fmul_rn(c.R[7], y));
    s = __fadd_rn(s, __fmul_rn(c.R[8], z));
    return __fadd_rn(s, c.t[2]);
}

// log2 of the Gaussian falloff at pixel-centre offset (dx, dy), fixed rounding:
// p = fma(fma(qc, dy, qb dx), dy, (qa dx) dx), Horner in dy.  The dx terms are
// shared by the pixels of one column, so they are split off.
__device__ __forceinline__ float falloff_col(float4 r0, float dx, float& wx) {
    wx = __fmul_rn(r0.w, dx);
    return __fmul_rn(__fmul_rn(r0.z, dx), dx);
}
__device__ __forceinline__ float falloff_row(float xx, float wx, float qc, float dy) {
    return __fmaf_rn(__fmaf_rn(qc, dy, wx), dy, xx);
}

// transmittance behind a composited entry, T (1 - alpha) as T - T alpha with
// one rounding
__device__ __forceinline__ float transmit(float T, float alpha) { return __fmaf_rn(-T, alpha, T); }

struct Proj {
    float qn[4], qinv;
    float Rq[9], s[3], M[9];
    float Sig[9];
    float t[3];
    float Tm[6];
    float A, B, C;
    float a, b, c;  // conic
};

// Projection of one Gaussian (EWA splatting, pinhole Jacobian at the camera
// space mean, dilation added to the 2D covariance).  False if culled.
__device__ __forceinline__ bool project_core(float4 p0, float4 p1, float4 p2, const CamDev& cam,
                                             const RasterDev& rc, Proj& x) {
    float depth = view_depth(cam, p0.x, p0.y, p0.z);
    if (!(depth > rc.near_plane)) return false;
    float qn2 = p2.x * p2.x + p2.y * p2.y + p2.z * p2.z + p2.w * p2.w;
    if (!(qn2 > 0.f)) return false;
    float qlen = sqrtf(qn2);
    x.qinv = 1.f / qlen;
    float w = p2.x * x.qinv, qx = p2.y * x.qinv, qy = p2.z * x.qinv, qz = p2.w * x.qinv;
    x.qn[0] = w; x.qn[1] = qx; x.qn[2] = qy; x.qn[3] = qz;
    x.Rq[0] = 1.f - 2.f * (qy * qy + qz * qz);
    x.Rq[1] = 2.f * (qx * qy - w * qz);
    x.Rq[2] = 2.f * (qx * qz + w * qy);
    x.Rq[3] = 2.f * (qx * qy + w * qz);
    x.Rq[4] = 1.f - 2.f * (qx * qx + qz * qz);
    x.Rq[5] = 2.f * (qy * qz - w * qx);
    x.Rq[6] = 2.f * (qx * qz - w * qy);
    x.Rq[7] = 2.f * (qy * qz + w * qx);
    x.Rq[8] = 1.f - 2.f * (qx * qx + qy * qy);
    x.s[0] = expf(p1.x); x.s[1] = expf(p1.y); x.s[2] = expf(p1.z);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) x.M[3 * i + j] = x.Rq[3 * i + j] * x.s[j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = i; k < 3; ++k) {
            float v = x.M[3 * i] * x.M[3 * k] + x.M[3 * i + 1] * x.M[3 * k + 1] + x.M[3 * i + 2] * x.M[3 * k + 2];
            x.Sig[3 * i + k] = v;
            x.Sig[3 * k + i] = v;
        }
    const float* R = cam.R;
    x.t[0] = R[0] * p0.x + R[1] * p0.y + R[2] * p0.z + cam.t[0];
    x.t[1] = R[3] * p0.x + R[4] * p0.y + R[5] * p0.z + cam.t[1];
    x.t[2] = depth;
    float iz = 1.f / depth;
    float J00 = cam.fx * iz, J02 = -cam.fx * x.t[0] * iz * iz;
    float J11 = cam.fy * iz, J12 = -cam.fy * x.t[1] * iz * iz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        x.Tm[k] = J00 * R[k] + J02 * R[6 + k];
        x.Tm[3 + k] = J11 * R[3 + k] + J12 * R[6 + k];
    }
    float u0[3], u1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u0[k] = x.Sig[3 * k] * x.Tm[0] + x.Sig[3 * k + 1] * x.Tm[1] + x.Sig[3 * k + 2] * x.Tm[2];
        u1[k] = x.Sig[3 * k] * x.Tm[3] + x.Sig[3 * k + 1] * x.Tm[4] + x.Sig[3 * k + 2] * x.Tm[5];
    }
    x.A = x.Tm[0] * u0[0] + x.Tm[1] * u0[1] + x.Tm[2] * u0[2] + rc.dilation;
    x.B = x.Tm[3] * u0[0] + x.Tm[4] * u0[1] + x.Tm[5] * u0[2];
    x.C = x.Tm[3] * u1[0] + x.Tm[4] * u1[1] + x.Tm[5] * u1[2] + rc.dilation;
    // det = A C - B^2 by Kahan's difference of products (the rounding error of
    // B^2 recovered with an FMA and added back; within 1.5 ulp, Jeannerod,
    // Louvet and Muller 2013), so that near-degenerate covariances keep an
    // accurate determinant without FP64 arithmetic
    float bb = __fmul_rn(x.B, x.B);
    float err = __fmaf_rn(-x.B, x.B, bb);
    float det = __fadd_rn(__fmaf_rn(x.A, x.C, -bb), err);
    if (!(det > 0.f)) return false;
    float idet = __frcp_rn(det);
    x.a = x.C * idet;
    x.b = -x.B * idet;
    x.c = x.A * idet;
    return true;
}

// one thread per Gaussian of the batch (global index g of view v)
__global__ void __launch_bounds__(256) k_project(const __grid_constant__ BatchDev b, RasterDev rc,
                                                 float4* __restrict__ rec, uint32_t* __restrict__ key,
                                                 uint32_t* __restrict__ idx, uint2* __restrict__ rect,
                                                 uint32_t* __restrict__ cnt) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= b.total_g) return;
    const ViewDev& vw = b.v[view_of_gaussian(b, g)];
    const CamDev& cam = vw.cam;
    const float4* params = vw.params + 4 * (size_t)(g - vw.g_off);
    float4 p0 = params[0], p1 = params[1], p2 = params[2], p3 = params[3];
    idx[g] = g;
    key[g] = 0xffffffffu;
    cnt[g] = 0;
    Proj x;
    if (!project_core(p0, p1, p2, cam, rc, x)) return;
    float op = 1.f / (1.f + expf(-p0.w));
    if (!(op >= rc.alpha_min)) return;  // no pixel can reach alpha_min
    float lthr2 = log2f(rc.alpha_min / op);
    float mx = cam.fx * x.t[0] / x.t[2] + cam.cx;
    float my = cam.fy * x.t[1] / x.t[2] + cam.cy;
    // alpha >= alpha_min  =>  d^T conic d <= k = 2 ln(op / alpha_min): an
    // ellipse whose bounding box has half-widths sqrt(k Sigma_xx) and
    // sqrt(k Sigma_yy) (Sigma = A, B, C, the inverse of the conic).  The
    // margins cover the rounding of the FP32 conic the pixels are tested with.
    const float k = -2.f * lthr2 * kLn2;
    const float rx = sqrtf(k * x.A) * 1.005f + 0.05f, ry = sqrtf(k * x.C) * 1.005f + 0.05f;
    if (!isfinite(mx) || !isfinite(my) || !isfinite(rx) || !isfinite(ry)) return;
    float xl = ceilf(fmaxf(mx - rx - 0.5f, -1.f)), xh = floorf(fminf(mx + rx - 0.5f, (float)cam.W));
    float yl = ceilf(fmaxf(my - ry - 0.5f, -1.f)), yh = floorf(fminf(my + ry - 0.5f, (float)cam.H));
    int ilo = max(0, (int)xl), ihi = min(cam.W - 1, (int)xh);
    int jlo = max(0, (int)yl), jhi = min(cam.H - 1, (int)yh);
    if (ilo > ihi || jlo > jhi) return;
    uint32_t tx0 = ilo / rc.tile_w, tx1 = ihi / rc.tile_w + 1;
    uint32_t ty0 = jlo / rc.tile_h, ty1 = jhi / rc.tile_h + 1;
    rect[g] = make_uint2(tx0 | (tx1 << 16), ty0 | (ty1 << 16));
    uint32_t bx0 = ilo / vw.bin, bx1 = ihi / vw.bin + 1;
    uint32_t by0 = jlo / vw.bin, by1 = jhi / vw.bin + 1;
    cnt[g] = (bx1 - bx0) * (by1 - by0);
    key[g] = __float_as_uint(x.t[2]);
    float h = -0.5f * kLog2e;
    rec[3 * (size_t)g] = make_float4(mx, my, h * x.a, -kLog2e * x.b);
    rec[3 * (size_t)g + 1] = make_float4(h * x.c, op, lthr2, 0.f);
    rec[3 * (size_t)g + 2] = make_float4(fmaxf(p3.x, 0.f), fmaxf(p3.y, 0.f), fmaxf(p3.z, 0.f), 0.f);
}

// Largest log2-falloff p = qa dx^2 + qb dx dy + qc dy^2 (negative definite)
// of a Gaussian over the rectangle [x0, x1] x [y0, y1] of pixel centres:
// 0 if its mean lies inside, else the best of the four edges, each a 1-D
// concave quadratic maximised at its clamped stationary point.
// The stationary point comes from an approximate reciprocal of 2 qc: an
// error d in it lowers the value found by |qc| d^2 (the quadratic is flat
// at its maximum), some 1e-6 here, far inside the cull margin below.
__device__ __forceinline__ float edge_max(float qa, float qb, float qc, float inv2qc, float fixed, float lo,
                                          float hi) {
    // p(fixed, t) = qa fixed^2 + qb fixed t + qc t^2, maximum over t in [lo, hi]
    float t = -qb * fixed * inv2qc;
    t = fminf(fmaxf(t, lo), hi);
    return qa * fixed * fixed + qb * fixed * t + qc * t * t;
}

__device__ __forceinline__ float rect_max_falloff(float4 r0, float qc, float x0, float x1, float y0, float y1) {
    float ax = x0 - r0.x, bx = x1 - r0.x, ay = y0 - r0.y, by = y1 - r0.y;
    if (ax <= 0.f && bx >= 0.f && ay <= 0.f && by >= 0.f) return 0.f;
    const float ic = rcp_approx(2.f * qc), ia = rcp_approx(2.f * r0.z);
    float m = edge_max(r0.z, r0.w, qc, ic, ax, ay, by);
    m = fmaxf(m, edge_max(r0.z, r0.w, qc, ic, bx, ay, by));
    m = fmaxf(m, edge_max(qc, r0.w, r0.z, ia, ay, ax, bx));
    m = fmaxf(m, edge_max(qc, r0.w, r0.z, ia, by, ax, bx));
    return m;
}

// A bin entry is kept for a tile if its tile rectangle covers the tile and
// its falloff can reach its alpha_min threshold at some pixel centre of the
// tile.  The margin (in log2 units) keeps the test conservative against the
// rounding of the per-pixel evaluation, so no composited pair is dropped.
constexpr float kCullMargin = 4e-3f;

// One warp emits the (bin, Gaussian) pairs of 32 consecutive depth-ordered
// Gaussians.  Their outputs form one contiguous run (the offsets are an
// exclusive scan in that order), so the warp walks the run 32 elements at a
// time: element e belongs to the last lane whose offset is <= e (a five-step
// search over the lanes' offsets), and every store instruction is contiguous.
// The bin rectangle follows from the tile rectangle.  A bin of that
// rectangle whose pixel centres the Gaussian's falloff cannot bring to its
// alpha_min threshold (the bound of the tile filter over the whole bin,
// with a wider margin) gets the key total_bins, which sorts after every bin
// and belongs to no bin's list: no tile of the bin would have kept it.
constexpr float kBinCullMargin = 4.f * kCullMargin;
__global__ void __launch_bounds__(256) k_emit(const __grid_constant__ BatchDev b, const uint32_t* __restrict__ sidx,
                                              const uint32_t* __restrict__ off, const uint32_t* __restrict__ cnt,
                                              const uint2* __restrict__ rect, const float4* __restrict__ rec,
                                              RasterDev rc, const uint32_t* __restrict__ counters,
                                              uint32_t* __restrict__ pkey, uint32_t* __restrict__ pval,
                                              unsigned long long* __restrict__ stats) {
    const uint32_t N = b.total_g;
    const uint32_t total = counters[kCntPairs];
    const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid * 32 >= N || total == 0) return;  // warp-uniform
    const uint32_t i = wid * 32 + lane;
    uint32_t g = 0, c = 0, o = 0;
    if (i < N) {
        g = sidx[i];
        c = cnt[g];
        o = off[i];
    }
    // lanes past N continue the run with no pairs, keeping the offsets monotone
    const uint32_t nv = min(32u, N - wid * 32);
    const uint32_t last_o = __shfl_sync(kFull, o, nv - 1), last_c = __shfl_sync(kFull, c, nv - 1);
    if (i >= N) o = last_o + last_c;
    const uint32_t start = __shfl_sync(kFull, o, 0);
    const uint32_t end = min(last_o + last_c, total);
    // per lane: bin rectangle origin and width, bins of its view
    uint32_t bx0 = 0, by0 = 0, wx = 1, boff = 0, bins_x = 0, bsz = 0;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (c) {
        uint2 rr = rect[g];
        const ViewDev& vw = b.v[view_of_gaussian(b, g)];
        r0 = rec[3 * (size_t)g];
        r1 = rec[3 * (size_t)g + 1];
        bsz = (uint32_t)vw.bin;
        bx0 = (rr.x & 0xffffu) / vw.spt_x;
        uint32_t bx1 = ((rr.x >> 16) - 1) / vw.spt_x + 1;
        by0 = (rr.y & 0xffffu) / vw.spt_y;
        wx = bx1 - bx0;
        boff = vw.bin_off;
        bins_x = (uint32_t)vw.bins_x;
    }
    uint32_t n_cull = 0;
    for (uint32_t e0 = start; e0 < end; e0 += 32) {
        const uint32_t e = e0 + lane;
        int j = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            uint32_t oj = __shfl_sync(kFull, o, j + step);
            if (j + step < 32 && oj <= e) j += step;
        }
        const uint32_t k = e - __shfl_sync(kFull, o, j);
        const uint32_t gj = __shfl_sync(kFull, g, j);
        const uint32_t wj = __shfl_sync(kFull, wx, j);
        const uint32_t x0 = __shfl_sync(kFull, bx0, j), y0 = __shfl_sync(kFull, by0, j);
        const uint32_t bo = __shfl_sync(kFull, boff, j), bxn = __shfl_sync(kFull, bins_x, j);
        const uint32_t bs = __shfl_sync(kFull, bsz, j);
        const float4 q0 = make_float4(__shfl_sync(kFull, r0.x, j), __shfl_sync(kFull, r0.y, j),
                                      __shfl_sync(kFull, r0.z, j), __shfl_sync(kFull, r0.w, j));
        const float qc = __shfl_sync(kFull, r1.x, j), thr = __shfl_sync(kFull, r1.z, j);
        if (e < end) {
            // row of pair k in a rectangle wj bins wide, floor((k + 1/2) / wj)
            // in FP32: the quotient stays 1 / (2 wj) away from an integer and
            // its two roundings move it by at most (k + 1/2) 2^-23 / wj, which
            // is less while k < 2^22 - 1/2 (a view has at most 2048 x 2048
            // bins of 32 px, so k < 2^22)
            const uint32_t ky = (uint32_t)(((float)k + 0.5f) * __frcp_rn((float)wj));
            const uint32_t kx = k - ky * wj;
            const float px0 = (float)((x0 + kx) * bs) + 0.5f, py0 = (float)((y0 + ky) * bs) + 0.5f;
            const float m = rect_max_falloff(q0, qc, px0, px0 + (float)(bs - 1), py0, py0 + (float)(bs - 1));
            const bool reach = m >= thr - kBinCullMargin * (1.f + fabsf(thr));
            pkey[e] = reach ? bo + (y0 + ky) * bxn + x0 + kx : b.total_bins;
            pval[e] = gj;
            n_cull += reach ? 0u : 1u;
        }
    }
    n_cull = __reduce_add_sync(kFull, n_cull);
    if (lane == 0 && n_cull) atomicAdd(&stats[kStCulled], (unsigned long long)n_cull);
}

// bin ranges from the sorted keys; keys >= nbins (culled pairs) have none
__global__ void k_ranges(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ counters,
                         uint2* __restrict__ ranges, uint32_t nbins) {
    uint32_t n = counters[kCntPairs];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t k = keys[i];
        if (k >= nbins) continue;
        if (i == 0 || keys[i - 1] != k) ranges[k].x = i;
        if (i == n - 1 || keys[i + 1] != k) ranges[k].y = i + 1;
    }
}



__device__ __forceinline__ bool tile_in(uint2 r, int tx, int ty) {
    return tx >= (int)(r.x & 0xffffu) && tx < (int)(r.x >> 16) && ty >= (int)(r.y & 0xffffu) &&
           ty < (int)(r.y >> 16);
}

__device__ __forceinline__ bool tile_hit(uint2 rect, float4 r0, float4 r1, int tx, int ty, int TW, int TH) {
    if (!tile_in(rect, tx, ty)) return false;
    float x0 = (float)(tx * TW) + 0.5f, y0 = (float)(ty * TH) + 0.5f;
    float m = rect_max_falloff(r0, r1.x, x0, x0 + (float)(TW - 1), y0, y0 + (float)(TH - 1));
    return m >= r1.z - kCullMargin * (1.f + fabsf(r1.z));
}

// Block-wide exclusive scan of small per-thread counts (in thread order) and
// their total.  Two barriers.
template <int NT>
__device__ __forceinline__ uint32_t block_scan_count(uint32_t v, int* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = (int)x;
    __syncthreads();
    uint32_t off = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) {
        const uint32_t c = (uint32_t)s_warp[k];
        off += k < w ? c : 0u;
        tot += c;
    }
    __syncthreads();
    total = tot;
    return off + x - v;
}

// Candidates a thread tests per filter round: one while a tile keeps most of
// its bin list, up to kMaxRound while it keeps few (a tile of a long list of
// large bins may keep 2% of it), so that long sparse lists cost few rounds
// of barriers.
constexpr int kMaxRound = 4;

// One filter round of a tile over its bin list [pos, end): thread t tests
// the kc candidates pos + t kc + k (k < kc), so that thread order is list
// order.  Returns the thread's hit bits (bit k: candidate pos + t kc + k);
// rank0 is the rank of its first hit among the round's hits, total their
// number.
template <int NT>
__device__ __forceinline__ uint32_t filter_round(uint32_t pos, uint32_t end, int kc,
                                                 const uint32_t* __restrict__ vals, const uint2* __restrict__ rect,
                                                 const float4* __restrict__ rec, int tx, int ty, int TW, int TH,
                                                 int* s_warp, uint32_t& rank0, uint32_t& total) {
    uint32_t mask = 0;
    if (kc == 1) {  // dense lists: one candidate per thread
        const uint32_t c = pos + threadIdx.x;
        if (c < end) {
            const uint32_t g = vals[c];
            const uint2 rr = rect[g];
            if (tile_in(rr, tx, ty) && tile_hit(rr, rec[3 * (size_t)g], rec[3 * (size_t)g + 1], tx, ty, TW, TH))
                mask = 1u;
        }
    } else {
        const uint32_t base = pos + threadIdx.x * (uint32_t)kc;
        uint32_t g[kMaxRound];
#pragma unroll
        for (int k = 0; k < kMaxRound; ++k) {
            const uint32_t c = base + (uint32_t)k;
            g[k] = (k < kc && c < end) ? vals[c] : 0xffffffffu;
        }
        // all gathers of the round before any test, so that their latencies overlap
        uint2 rr[kMaxRound];
#pragma unroll
        for (int k = 0; k < kMaxRound; ++k) rr[k] = g[k] != 0xffffffffu ? rect[g[k]] : make_uint2(0u, 0u);
        uint32_t in = 0;
#pragma unroll
        for (int k = 0; k < kMaxRound; ++k) in |= (g[k] != 0xffffffffu && tile_in(rr[k], tx, ty)) ? 1u << k : 0u;
        for (uint32_t m = in; m; m &= m - 1) {  // few candidates reach the exact test
            const int k = __ffs(m) - 1;
            const uint32_t gk = vals[base + (uint32_t)k];  // both loads hit L1 now
            if (tile_hit(rect[gk], rec[3 * (size_t)gk], rec[3 * (size_t)gk + 1], tx, ty, TW, TH)) mask |= 1u << k;
        }
    }
    rank0 = block_scan_count<NT>((uint32_t)__popc(mask), s_warp, total);
    return mask;
}

// one warp of the block counts its pixels' evaluated pairs with one atomic
__device__ __forceinline__ void warp_count(unsigned long long* dst, uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, (unsigned long long)v);
}

// ------------------------------------------------------------------ forward
//
// One CTA per tile; each thread owns PPT pixels of a column, (x, y) and
// (x, y + TH/PPT).  The tile walks the depth-ordered list of its bin in
// rounds: the CTA tests NT candidates at a time against the tile (tile
// rectangle, then the exact ellipse bound), compacts the hits in list order
// into shared memory (their 48-B records) until `cap` are staged, then every
// pixel composites the staged entries.  The CTA stops when all its pixels
// have reached T_min.
template <int TW, int TH, int PPT>
__global__ void __launch_bounds__(TW* TH / PPT) k_render(const __grid_constant__ BatchDev b,
                                                         const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ vals,
                                                         const uint2* __restrict__ rect,
                                                         const float4* __restrict__ rec, RasterDev rc,
                                                         uint32_t* __restrict__ queue,
                                                         unsigned long long* __restrict__ stats,
                                                         const uint32_t* __restrict__ order) {
    constexpr int NT = TW * TH / PPT;
    constexpr int ROWS = TH / PPT;
    extern __shared__ float4 smem[];
    __shared__ int s_warp[NT / 32];
    const int cap = rc.cap;
    float4* s0 = smem;
    float4* s1 = smem + cap;
    float4* s2 = smem + 2 * cap;
    uint32_t n_eval = 0, n_comp = 0;
    __shared__ uint32_t s_tile, s_resume;
    // persistent CTAs: tiles of all views are handed out by an atomic counter,
    // in the order of their expected cost (longest bin list first)
    for (;;) {
    if (threadIdx.x == 0) {
        uint32_t q = atomicAdd(queue, 1u);
        s_tile = q < b.total_tiles ? order[q] : b.total_tiles;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    __syncthreads();
    if (tile >= b.total_tiles) break;
    const ViewDev& vw = b.v[view_of_tile(b, tile)];
    const CamDev& cam = vw.cam;
    const uint32_t lt = tile - vw.tile_off;
    const int tx = (int)(lt % (uint32_t)vw.tiles_x), ty = (int)(lt / (uint32_t)vw.tiles_x);
    int px = tx * TW + (threadIdx.x % TW), py0 = ty * TH + (threadIdx.x / TW);
    float fx = (float)px + 0.5f;
    float fy[PPT], T[PPT], Cr[PPT], Cg[PPT], Cb[PPT];
    bool inside[PPT];
    // entries a pixel evaluated, set when it reaches T_min; all ones while it
    // has not (a pixel outside the image starts at 0: nothing to evaluate)
    uint32_t ev[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int py = py0 + q * ROWS;
        inside[q] = px < cam.W && py < cam.H;
        fy[q] = (float)py + 0.5f;
        T[q] = 1.f;
        Cr[q] = Cg[q] = Cb[q] = 0.f;
        ev[q] = inside[q] ? 0xffffffffu : 0u;
    }
    uint2 rg = ranges[vw.bin_off + (ty / vw.spt_y) * vw.bins_x + tx / vw.spt_x];
    uint32_t pos = rg.x;
    uint32_t hbase = 0;  // entries staged by earlier batches of this tile
    int kc = 1;          // candidates per thread and filter round
    for (;;) {
        bool tdone = true;
#pragma unroll
        for (int q = 0; q < PPT; ++q) tdone = tdone && ev[q] != 0xffffffffu;
        if (__syncthreads_count(tdone) == NT || pos >= rg.y) break;
        int staged = 0;
        while (pos < rg.y && staged < cap) {
            uint32_t r, tot;
            const uint32_t mask = filter_round<NT>(pos, rg.y, kc, vals, rect, rec, tx, ty, TW, TH, s_warp, r, tot);
            const uint32_t room = (uint32_t)(cap - staged), base = pos + threadIdx.x * (uint32_t)kc;
            for (uint32_t m = mask; m; m &= m - 1, ++r) {
                const uint32_t c = base + (uint32_t)(__ffs(m) - 1);
                if (r < room) {
                    const uint32_t g = vals[c];
                    s0[staged + r] = rec[3 * (size_t)g];
                    s1[staged + r] = rec[3 * (size_t)g + 1];
                    s2[staged + r] = rec[3 * (size_t)g + 2];
                } else if (r == room) {
                    s_resume = c;  // the first hit that did not fit: the next round starts there
                }
            }
            if (tot > room) {
                __syncthreads();
                pos = s_resume;
                staged = cap;
                kc = max(kc >> 1, 1);
            } else {
                pos += (uint32_t)kc * NT;
                staged += (int)tot;
                if (4 * tot < room && kc < kMaxRound) kc <<= 1;
            }
        }
        __syncthreads();
        if (!tdone) {
            for (int k = 0; k < staged; ++k) {
                float4 r0 = s0[k];
                float4 r1 = s1[k];
                float wx, xx = falloff_col(r0, __fsub_rn(fx, r0.x), wx);
                bool all = true;
                const float4 c = s2[k];
                // only the done test branches; the alpha_min and T_min decisions
                // select (adding a zero weight leaves a colour unchanged)
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    if (ev[q] != 0xffffffffu) continue;
                    const float p = falloff_row(xx, wx, r1.x, __fsub_rn(fy[q], r0.y));
                    const bool hit = !(p < r1.z);
                    const float alpha = fminf(rc.alpha_max, __fmul_rn(r1.y, ex2_approx(p)));
                    const float Tn = transmit(T[q], alpha);
                    const bool stop = hit && Tn < rc.T_min;
                    const bool comp = hit && !stop;
                    ev[q] = stop ? hbase + (uint32_t)k + 1u : ev[q];
                    all = all && stop;
                    n_comp += comp ? 1u : 0u;
                    const float wgt = comp ? alpha * T[q] : 0.f;
                    Cr[q] = fmaf(c.x, wgt, Cr[q]);
                    Cg[q] = fmaf(c.y, wgt, Cg[q]);
                    Cb[q] = fmaf(c.z, wgt, Cb[q]);
                    T[q] = comp ? Tn : T[q];
                }
                if (all) break;  // every pixel of the thread has stopped
            }
        }
        hbase += (uint32_t)staged;
    }
    size_t HW = (size_t)cam.W * cam.H;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        n_eval += ev[q] == 0xffffffffu ? hbase : ev[q];  // a pixel that never stopped saw every entry
        if (inside[q]) {
            size_t p = (size_t)(py0 + q * ROWS) * cam.W + px;
            vw.image[p] = Cr[q];
            vw.image[HW + p] = Cg[q];
            vw.image[2 * HW + p] = Cb[q];
        }
    }
    }  // tiles
    warp_count(&stats[kStEvalFwd], n_eval);
    warp_count(&stats[kStCompFwd], n_comp);
}

// ------------------------------------------------------------------ backward

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Warp reduce-scatter of eight values: at each butterfly step a lane keeps
// half of its values and adds the partner's copy of that half, so 4 + 2 + 1
// shuffles leave lane l with the sum over its 8-lane group of value
// (l >> 2) & 7, and two more finish the sum over all 32 lanes (9 shuffles
// instead of 8 x 5).
__device__ __forceinline__ float warp_reduce_scatter8(const float (&a)[8], int lane) {
    float b[4], c[2];
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float send = h4 ? a[k] : a[k + 4];
        float keep = h4 ? a[k + 4] : a[k];
        b[k] = keep + __shfl_xor_sync(kFull, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float send = h3 ? b[k] : b[k + 2];
        float keep = h3 ? b[k + 2] : b[k];
        c[k] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    float send = h2 ? c[0] : c[1];
    float d = (h2 ? c[1] : c[0]) + __shfl_xor_sync(kFull, send, 4);
    d += __shfl_xor_sync(kFull, d, 2);
    d += __shfl_xor_sync(kFull, d, 1);
    return d;
}

// Phase 1 re-walks the bin list front to back with the forward's decisions.
// The entries that pass the tile filter ("hits") are numbered in list order;
// their Gaussian ids go to a shared-memory ring of `ring` slots (a power of
// two), and the list position of every ring-th hit is recorded, so that phase 2 can
// rebuild any chunk of hits without scanning from the start.  Each pixel
// keeps its final T and the hit number of the entry that stopped it (none if
// it never stopped: it then saw every hit).
// Phase 2 walks the hits back to front, chunk by chunk (the last chunk is
// still in the ring; earlier ones are re-filtered from their recorded
// position), stages their records, and per entry sums the nine 2D gradient
// terms over the warp (reduce-scatter) before the global atomics.
//
// LOSS != kLossNone is the training step with the HDR loss folded in: phase 1
// also composites the colours (the forward's arithmetic, so the image is the
// forward's bit for bit), then every pixel evaluates the loss against its
// target and its own dL/dC, writes the image and adds its loss term to the
// tile's partial sum, and phase 2 runs on that gradient.  Nothing per pixel
// leaves the tile.
constexpr int kMaxChunks = 256;

// Loss partials per tile of the training step, one per pixel slot class
// q mod SLOTS: as many as the parts the order may split a tile into (4 with
// one-warp CTAs, 2 with larger ones), so that every part owns whole classes
// and the loss does not depend on the split.
__host__ __device__ constexpr int loss_slots(int threads) { return threads <= 32 ? 4 : 2; }

// CTAs per SM the register allocation is sized for.  At 4 pixels per thread
// 12 CTAs of 64 threads (80 registers; the 17 KB of shared memory per CTA
// allow 12 too) were measured 9% faster than 9 (96 registers, 22 KB with a
// 2048-entry hit ring) and 5% faster than 14 (72 registers, 512 entries); at
// 2 pixels per thread 7 CTAs of 128 threads (72 registers) beat 6 and 8.
constexpr int bwd_min_blocks(int ppt) { return ppt == 1 ? 4 : (ppt == 2 ? 7 : (ppt == 4 ? 12 : 15)); }

template <int TW, int TH, int PPT, int LOSS>
__global__ void __launch_bounds__(TW* TH / PPT, bwd_min_blocks(PPT)) k_render_bwd(const __grid_constant__ BatchDev b,
                                                             const uint2* __restrict__ ranges,
                                                             const uint32_t* __restrict__ vals,
                                                             const uint2* __restrict__ rect,
                                                             const float4* __restrict__ rec, RasterDev rc,
                                                             float4* __restrict__ g2d, uint32_t* __restrict__ queue,
                                                             unsigned long long* __restrict__ stats,
                                                             float* __restrict__ tile_loss,
                                                             const uint32_t* __restrict__ order,
                                                             const uint32_t* __restrict__ fb_state,
                                                             uint32_t* __restrict__ fb, uint32_t fb_stride) {
    constexpr int NT = TW * TH / PPT;
    constexpr int ROWS = TH / PPT;
    constexpr int SLOTS = loss_slots(NT);
    extern __shared__ float4 smem[];
    __shared__ int s_warp[NT / 32];
    __shared__ uint32_t s_end;
    __shared__ uint32_t s_chunk_pos[kMaxChunks];
    __shared__ float s_loss[SLOTS][NT / 32];
    const int cap = rc.cap;
    float4* s0 = smem;
    float4* s1 = smem + cap;
    float4* s2 = smem + 2 * cap;
    uint32_t* hits = reinterpret_cast<uint32_t*>(smem + 3 * cap);
    const uint32_t rmask = (1u << rc.ring_log2) - 1u;
    uint32_t n_eval1 = 0, n_eval2 = 0, n_hit2 = 0;
    __shared__ uint32_t s_item, s_resume;
    // work items and the feedback buffer of this launch (set by the order kernel)
    const uint32_t n_items = fb_state[kFbItems];
    uint32_t* const fb_hit = fb + 2 * (size_t)fb_stride * (fb_state[kFbParity] & 1u);
    // persistent CTAs: work items (tiles, or parts of the heaviest tiles) of
    // all views are handed out by an atomic counter, longest first
    for (;;) {
    if (threadIdx.x == 0) {
        uint32_t q = atomicAdd(queue, 1u);
        s_item = q < n_items ? order[q] : kItemNone;
    }
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item == kItemNone) break;
    const uint32_t tile = item & 0xffffffu;
    // a part owns the pixel slots q with q mod nparts == part
    const int part = (int)((item >> 24) & 15u), pmask = (1 << (item >> 28)) - 1;
    const ViewDev& vw = b.v[view_of_tile(b, tile)];
    const CamDev& cam = vw.cam;
    const uint32_t lt = tile - vw.tile_off;
    const int tx = (int)(lt % (uint32_t)vw.tiles_x), ty = (int)(lt / (uint32_t)vw.tiles_x);
    const float* dL_dimg = vw.dL;
    int px = tx * TW + (threadIdx.x % TW), py0 = ty * TH + (threadIdx.x / TW);
    float fx = (float)px + 0.5f;
    size_t HW = (size_t)cam.W * cam.H;
    float fy[PPT], gr[PPT], gg[PPT], gb[PPT], T[PPT];
    bool active[PPT];
    uint32_t last[PPT], ev[PPT];
    float Cr[PPT], Cg[PPT], Cb[PPT];  // composited colour (training step only)
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int py = py0 + q * ROWS;
        bool inside = px < cam.W && py < cam.H && (q & pmask) == part;
        fy[q] = (float)py + 0.5f;
        gr[q] = gg[q] = gb[q] = 0.f;
        Cr[q] = Cg[q] = Cb[q] = 0.f;
        if (LOSS == kLossNone) {
            if (inside) {
                size_t pix = (size_t)py * cam.W + px;
                gr[q] = dL_dimg[pix];
                gg[q] = dL_dimg[HW + pix];
                gb[q] = dL_dimg[2 * HW + pix];
            }
            active[q] = inside && (gr[q] != 0.f || gg[q] != 0.f || gb[q] != 0.f);
        } else {
            active[q] = inside;  // the gradient is known after phase 1
        }
        T[q] = 1.f;
        ev[q] = active[q] ? 0xffffffffu : 0u;
    }
    uint2 rg = ranges[vw.bin_off + (ty / vw.spt_y) * vw.bins_x + tx / vw.spt_x];

    // ---- phase 1
    uint32_t nhit = 0;  // hits found so far (uniform)
    uint32_t pos = rg.x;
    int kc = 1;         // candidates per thread and filter round
    for (;;) {
        bool tdone = true;
#pragma unroll
        for (int q = 0; q < PPT; ++q) tdone = tdone && ev[q] != 0xffffffffu;
        if (__syncthreads_count(tdone) == NT || pos >= rg.y) break;
        int staged = 0;
        uint32_t h0 = nhit;
        while (pos < rg.y && staged < cap) {
            uint32_t r, tot;
            const uint32_t mask = filter_round<NT>(pos, rg.y, kc, vals, rect, rec, tx, ty, TW, TH, s_warp, r, tot);
            const uint32_t room = (uint32_t)(cap - staged), base = pos + threadIdx.x * (uint32_t)kc;
            for (uint32_t m = mask; m; m &= m - 1, ++r) {
                const uint32_t c = base + (uint32_t)(__ffs(m) - 1);
                if (r < room) {
                    const uint32_t g = vals[c];
                    s0[staged + r] = rec[3 * (size_t)g];
                    s1[staged + r] = rec[3 * (size_t)g + 1];
                    if (LOSS != kLossNone) s2[staged + r] = rec[3 * (size_t)g + 2];
                    const uint32_t hid = nhit + r;
                    hits[hid & rmask] = g;
                    if ((hid & rmask) == 0 && (hid >> rc.ring_log2) < kMaxChunks) s_chunk_pos[hid >> rc.ring_log2] = c;
                } else if (r == room) {
                    s_resume = c;  // the first hit that did not fit: the next round starts there
                }
            }
            if (tot > room) {
                __syncthreads();
                pos = s_resume;
                staged = cap;
                nhit += room;
                kc = max(kc >> 1, 1);
            } else {
                pos += (uint32_t)kc * NT;
                staged += (int)tot;
                nhit += tot;
                if (4 * tot < room && kc < kMaxRound) kc <<= 1;
            }
        }
        __syncthreads();
        if (!tdone) {
            for (int k = 0; k < staged; ++k) {
                float4 r0 = s0[k];
                float4 r1 = s1[k];
                float wx, xx = falloff_col(r0, __fsub_rn(fx, r0.x), wx);
                float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
                if (LOSS != kLossNone) c = s2[k];
                // only the done test branches; the alpha_min and T_min decisions
                // select (measured 2.5-3% faster than branching on all three)
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    if (ev[q] != 0xffffffffu) continue;  // stopped (or inactive)
                    const float p = falloff_row(xx, wx, r1.x, __fsub_rn(fy[q], r0.y));
                    const bool hit = !(p < r1.z);
                    const float alpha = fminf(rc.alpha_max, __fmul_rn(r1.y, ex2_approx(p)));
                    const float Tn = transmit(T[q], alpha);
                    const bool stop = hit && Tn < rc.T_min;
                    const bool comp = hit && !stop;
                    ev[q] = stop ? h0 + (uint32_t)k + 1u : ev[q];
                    if (LOSS != kLossNone) {  // the forward's colour arithmetic
                        const float wgt = comp ? alpha * T[q] : 0.f;
                        Cr[q] = fmaf(c.x, wgt, Cr[q]);
                        Cg[q] = fmaf(c.y, wgt, Cg[q]);
                        Cb[q] = fmaf(c.z, wgt, Cb[q]);
                    }
                    T[q] = comp ? Tn : T[q];
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q)
        if (active[q]) n_eval1 += ev[q] == 0xffffffffu ? nhit : ev[q];
    if (LOSS != kLossNone) {
        // image out, loss term and dL/dC of every pixel; the tile's loss goes
        // to SLOTS partials, one per pixel slot class q mod SLOTS (fixed
        // order: pixels of a thread, warp butterfly, warps in order), so that
        // the sums do not depend on how the tile was split into parts
        float lsum[SLOTS];
#pragma unroll
        for (int r = 0; r < SLOTS; ++r) lsum[r] = 0.f;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            if (!active[q]) continue;
            size_t pix = (size_t)(py0 + q * ROWS) * cam.W + px;
            if (vw.image) {
                vw.image[pix] = Cr[q];
                vw.image[HW + pix] = Cg[q];
                vw.image[2 * HW + pix] = Cb[q];
            }
            const float* tg = vw.target;
            lsum[q & (SLOTS - 1)] += hdr_term(Cr[q], tg[pix]) + hdr_term(Cg[q], tg[HW + pix]) + hdr_term(Cb[q], tg[2 * HW + pix]);
            gr[q] = hdr_grad(Cr[q], tg[pix], LOSS == kLossHdrFull, vw.invk);
            gg[q] = hdr_grad(Cg[q], tg[HW + pix], LOSS == kLossHdrFull, vw.invk);
            gb[q] = hdr_grad(Cb[q], tg[2 * HW + pix], LOSS == kLossHdrFull, vw.invk);
            active[q] = gr[q] != 0.f || gg[q] != 0.f || gb[q] != 0.f;
        }
#pragma unroll
        for (int r = 0; r < SLOTS; ++r) {
            const float ls = warp_sum(lsum[r]);
            if ((threadIdx.x & 31) == 0) s_loss[r][threadIdx.x >> 5] = ls;
        }
        __syncthreads();
        if (threadIdx.x < SLOTS && (threadIdx.x & pmask) == part) {  // the partials this item owns
            float t = 0.f;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) t += s_loss[threadIdx.x][w];
            tile_loss[SLOTS * (size_t)tile + threadIdx.x] = t;
        }
    }
    if (threadIdx.x == 0) s_end = 0;
    __syncthreads();
    // Phase 2 evaluates a pixel at the entries [0, last): up to the one that
    // stopped it, else to the end of the list (the entries after its last
    // composited one are then non-hits, skipped by the alpha_min test).
    uint32_t mylast = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        last[q] = !active[q] ? 0u : (ev[q] == 0xffffffffu ? nhit : ev[q] - 1u);
        mylast = max(mylast, last[q]);
        n_eval2 += last[q];
    }
    if (mylast) atomicMax(&s_end, mylast);
    __syncthreads();
    const uint32_t hend = s_end;
    // feedback for the next launch's order: the tile's (parts': largest) hits
    // front to back and length back to front
    if (threadIdx.x == 0) {
        atomicMax(&fb_hit[tile], nhit);
        atomicMax(&fb_hit[fb_stride + tile], hend);
    }
    uint32_t wlast = mylast;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wlast = max(wlast, __shfl_xor_sync(kFull, wlast, o));

    // ---- phase 2
    // DS = dL/dC . S, with S the colour composited behind the current entry:
    // dL/dalpha = T dL/dC . c - DS / (1 - alpha), and DS grows by
    // alpha T dL/dC . c, so the three channels of S need not be kept.
    float DS[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) DS[q] = 0.f;
    int lane = threadIdx.x & 31;
    int ring_chunk = nhit ? (int)((nhit - 1) >> rc.ring_log2) : -1;  // chunk whose hits the ring holds
    for (int ch = hend ? (int)((hend - 1) >> rc.ring_log2) : -1; ch >= 0; --ch) {
        const uint32_t hc0 = (uint32_t)ch << rc.ring_log2;
        const uint32_t hc1 = min(hc0 + rmask + 1u, hend);
        if (ch != ring_chunk) {
            // rebuild hits [hc0, hc1) from the nearest recorded chunk start
            int base_chunk = ch < kMaxChunks ? ch : kMaxChunks - 1;
            uint32_t p = s_chunk_pos[base_chunk];
            uint32_t h = (uint32_t)base_chunk << rc.ring_log2;
            __syncthreads();
            int kr = 1;
            while (h < hc1 && p < rg.y) {
                uint32_t r, tot;
                const uint32_t mask = filter_round<NT>(p, rg.y, kr, vals, rect, rec, tx, ty, TW, TH, s_warp, r, tot);
                const uint32_t base = p + threadIdx.x * (uint32_t)kr;
                for (uint32_t m = mask; m; m &= m - 1, ++r) {
                    const uint32_t hid = h + r;
                    if (hid >= hc0 && hid < hc1) hits[hid & rmask] = vals[base + (uint32_t)(__ffs(m) - 1)];
                }
                h += tot;
                p += (uint32_t)kr * NT;
                if (4 * tot < (uint32_t)(kr * NT) && kr < kMaxRound) kr <<= 1;
            }
            ring_chunk = ch;
        }
        // back to front over the chunk, staged in batches of cap records
        for (uint32_t b1 = hc1; b1 > hc0;) {
            uint32_t b0 = b1 - hc0 > (uint32_t)cap ? b1 - cap : hc0;
            int n = (int)(b1 - b0);
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += NT) {
                uint32_t g = hits[(b0 + i) & rmask];
                s0[i] = rec[3 * (size_t)g];
                s1[i] = rec[3 * (size_t)g + 1];
                s2[i] = rec[3 * (size_t)g + 2];
            }
            __syncthreads();
            for (int k = n - 1; k >= 0; --k) {
                uint32_t j = b0 + k;
                if (j >= wlast) continue;  // warp-uniform
                float4 r0 = s0[k];
                float4 r1 = s1[k];
                float4 c = s2[k];
                const float dx = __fsub_rn(fx, r0.x);
                float wx, xx = falloff_col(r0, dx, wx);
                // per entry: sum w dx, sum w dy, sum w dx^2, sum w dx dy, sum w dy^2
                // (w = dL/dalpha alpha), sum w, red, green; blue apart.  The
                // pixels of a thread share dx, so the thread sums w, w dy and
                // w dy^2 and scales by dx (and dx^2) once per entry.
                float v8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float sw = 0.f, dcb = 0.f;
                bool any = false;
                // stage A for all pixels (independent chains, so their ex2
                // latencies overlap), stage B only for the pixels that take
                // the entry (measured 1.5-2.5% faster than one stage)
                float dyv[PPT], ev2[PPT];
                bool hq[PPT];
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    dyv[q] = __fsub_rn(fy[q], r0.y);
                    const float p = falloff_row(xx, wx, r1.x, dyv[q]);
                    hq[q] = j < last[q] && !(p < r1.z);
                    ev2[q] = ex2_approx(p);
                }
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    if (!hq[q]) continue;
                    any = true;
                    ++n_hit2;
                    const float dy = dyv[q], e = ev2[q];
                    const float araw = __fmul_rn(r1.y, e);
                    float alpha = fminf(rc.alpha_max, araw);
                    float inv = rcp_approx(1.f - alpha);
                    T[q] = T[q] * inv;  // transmittance in front of this entry
                    float wgt = alpha * T[q];
                    v8[6] = fmaf(wgt, gr[q], v8[6]);
                    v8[7] = fmaf(wgt, gg[q], v8[7]);
                    dcb = fmaf(wgt, gb[q], dcb);
                    float dc = fmaf(gb[q], c.z, fmaf(gg[q], c.y, gr[q] * c.x));
                    float dal = fmaf(T[q], dc, -inv * DS[q]);
                    DS[q] = fmaf(wgt, dc, DS[q]);
                    if (araw < rc.alpha_max) {
                        float w = dal * alpha;
                        float wy = w * dy;
                        sw += w;
                        v8[1] += wy;
                        v8[4] = fmaf(wy, dy, v8[4]);
                    }
                }
                v8[0] = sw * dx;
                v8[2] = v8[0] * dx;
                v8[3] = v8[1] * dx;
                v8[5] = sw;
                if (__any_sync(kFull, any)) {
                    // values 0..7 -> floats 0..5, 8, 9 of the 12-float 2D gradient record
                    float tot = warp_reduce_scatter8(v8, lane);
                    float blue = warp_sum(dcb);
                    float* gg2 = reinterpret_cast<float*>(g2d + 3 * (size_t)hits[j & rmask]);
                    if ((lane & 3) == 0) {
                        int v = lane >> 2;
                        atomicAdd(gg2 + (v < 6 ? v : v + 2), tot);
                    }
                    if (lane == 1) atomicAdd(gg2 + 10, blue);
                }
            }
            b1 = b0;
        }
    }
    }  // tiles
    warp_count(&stats[kStEvalRewalk], n_eval1);
    warp_count(&stats[kStEvalBack], n_eval2);
    // the entries a pixel meets in phase 2 (before the one that stopped it)
    // whose falloff passes alpha_min are exactly the pairs phase 1 composited
    warp_count(&stats[kStCompRewalk], n_hit2);
    warp_count(&stats[kStHitBack], n_hit2);
}

// The parameter gradient of one Gaussian from its 2D gradient record a0..a2
// (zero record or not projected: false, o untouched).
__device__ __forceinline__ bool project_grad(const float4& a0, const float4& a1, const float4& a2, const float4& p0,
                                             const float4& p1, const float4& p2, const float4& p3, const CamDev& cam,
                                             const RasterDev& rc, float4& o0, float4& o1, float4& o2, float4& o3) {
    if (a0.x == 0.f && a0.y == 0.f && a0.z == 0.f && a0.w == 0.f && a1.x == 0.f && a1.y == 0.f && a2.x == 0.f &&
        a2.y == 0.f && a2.z == 0.f)
        return false;
    Proj x;
    if (!project_core(p0, p1, p2, cam, rc, x)) return false;
    const float* R = cam.R;
    // The record holds, summed over pixels, w dx, w dy, w dx^2, w dx dy,
    // w dy^2 with w = dL/dalpha alpha = dL/dpower (power = -d^T Q d / 2,
    // d = pixel - mean), then sum w and the colour terms.  Where alpha =
    // o G is not clamped, dL/do = sum dL/dalpha G = sum w / o.
    float qa = x.a, qb = x.b, qc = x.c;
    float gmx = qa * a0.x + qb * a0.y, gmy = qb * a0.x + qc * a0.y;
    float ga = -0.5f * a0.z, gb = -a0.w, gc = -0.5f * a1.x;
    // dL/dSigma2D = -Q G Q with G = [[ga, gb/2], [gb/2, gc]]
    float dA = -(ga * qa * qa + gb * qa * qb + gc * qb * qb);
    float dC = -(ga * qb * qb + gb * qb * qc + gc * qc * qc);
    float dB = -(2.f * ga * qa * qb + gb * (qa * qc + qb * qb) + 2.f * gc * qb * qc);
    const float* T0 = x.Tm;
    const float* T1 = x.Tm + 3;
    float st0[3], st1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        st0[k] = x.Sig[3 * k] * T0[0] + x.Sig[3 * k + 1] * T0[1] + x.Sig[3 * k + 2] * T0[2];
        st1[k] = x.Sig[3 * k] * T1[0] + x.Sig[3 * k + 1] * T1[1] + x.Sig[3 * k + 2] * T1[2];
    }
    float dT0[3], dT1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dT0[k] = 2.f * dA * st0[k] + dB * st1[k];
        dT1[k] = dB * st0[k] + 2.f * dC * st1[k];
    }
    // Tm = J R: only J00, J02, J11, J12 are non-zero
    float dJ00 = dT0[0] * R[0] + dT0[1] * R[1] + dT0[2] * R[2];
    float dJ02 = dT0[0] * R[6] + dT0[1] * R[7] + dT0[2] * R[8];
    float dJ11 = dT1[0] * R[3] + dT1[1] * R[4] + dT1[2] * R[5];
    float dJ12 = dT1[0] * R[6] + dT1[1] * R[7] + dT1[2] * R[8];
    float tx = x.t[0], ty = x.t[1], tz = x.t[2];
    float iz = 1.f / tz, iz2 = iz * iz, iz3 = iz2 * iz;
    float dtx = dJ02 * (-cam.fx * iz2) + gmx * cam.fx * iz;
    float dty = dJ12 * (-cam.fy * iz2) + gmy * cam.fy * iz;
    float dtz = dJ00 * (-cam.fx * iz2) + dJ02 * (2.f * cam.fx * tx * iz3) + dJ11 * (-cam.fy * iz2) +
                dJ12 * (2.f * cam.fy * ty * iz3) - gmx * cam.fx * tx * iz2 - gmy * cam.fy * ty * iz2;
    o0.x += R[0] * dtx + R[3] * dty + R[6] * dtz;
    o0.y += R[1] * dtx + R[4] * dty + R[7] * dtz;
    o0.z += R[2] * dtx + R[5] * dty + R[8] * dtz;
    float op = 1.f / (1.f + expf(-p0.w));
    o0.w += a1.y * (1.f - op);  // (sum w / o) do/dlogit, do/dlogit = o (1 - o)
    // Sigma = M M^T: dL/dM = (G + G^T) M with G = dA T0 T0^T + dB T0 T1^T + dC T1 T1^T
    float Gs[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Gs[3 * i + j] = 2.f * dA * T0[i] * T0[j] + dB * (T0[i] * T1[j] + T1[i] * T0[j]) + 2.f * dC * T1[i] * T1[j];
    float dR[9];
    float dls[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        float ds = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float dM = Gs[3 * k] * x.M[l] + Gs[3 * k + 1] * x.M[3 + l] + Gs[3 * k + 2] * x.M[6 + l];
            ds += dM * x.Rq[3 * k + l];
            dR[3 * k + l] = dM * x.s[l];
        }
        dls[l] = ds * x.s[l];
    }
    o1.x += dls[0];
    o1.y += dls[1];
    o1.z += dls[2];
    float w = x.qn[0], qx = x.qn[1], qy = x.qn[2], qz = x.qn[3];
    float dw = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
    float dx = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - w * dR[5] + qz * dR[6] + w * dR[7]) -
               4.f * qx * (dR[4] + dR[8]);
    float dy = 2.f * (qx * dR[1] + w * dR[2] + qx * dR[3] + qz * dR[5] - w * dR[6] + qz * dR[7]) -
               4.f * qy * (dR[0] + dR[8]);
    float dz = 2.f * (-w * dR[1] + qx * dR[2] + w * dR[3] + qy * dR[5] + qx * dR[6] + qy * dR[7]) -
               4.f * qz * (dR[0] + dR[4]);
    float dot = w * dw + qx * dx + qy * dy + qz * dz;
    o2.x += (dw - w * dot) * x.qinv;
    o2.y += (dx - qx * dot) * x.qinv;
    o2.z += (dy - qy * dot) * x.qinv;
    o2.w += (dz - qz * dot) * x.qinv;
    if (p3.x > 0.f) o3.x += a2.x;
    if (p3.y > 0.f) o3.y += a2.y;
    if (p3.z > 0.f) o3.z += a2.z;
    return true;
}

// 2D gradients -> packed parameter gradients (+=), with vector atomics when
// two views of the batch share a parameter set.
// The training step's loss of view v from its tiles' partials (`slots` per
// tile), summed by one 128-thread block in a fixed order in FP64: four
// strided accumulators per thread, then the warps in order.  The gradient
// kernels below give their first nviews blocks this work, so that it runs
// beside theirs instead of as a launch of its own.
__device__ void view_loss_sum(const BatchDev& b, const float* __restrict__ tile_loss, int slots, int v) {
    __shared__ double sm[4];
    const ViewDev& vw = b.v[v];
    const uint32_t n = (uint32_t)slots * (uint32_t)vw.tiles_x * (uint32_t)vw.tiles_y;
    const float* x = tile_loss + (size_t)slots * vw.tile_off;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    uint32_t i = threadIdx.x;
    for (; i + 384 < n; i += 512) {
        a0 += (double)x[i];
        a1 += (double)x[i + 128];
        a2 += (double)x[i + 256];
        a3 += (double)x[i + 384];
    }
    for (; i < n; i += 128) a0 += (double)x[i];
    double acc = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && vw.loss) *vw.loss = (float)(((sm[0] + sm[1]) + (sm[2] + sm[3])) * (double)vw.invk);
}

__global__ void __launch_bounds__(128) k_project_bwd(const __grid_constant__ BatchDev b, RasterDev rc,
                                                     const uint32_t* __restrict__ cnt,
                                                     const float4* __restrict__ g2d, int shared_params,
                                                     const float* __restrict__ tile_loss, int slots) {
    const uint32_t nl = tile_loss ? (uint32_t)b.nviews : 0u;
    if (blockIdx.x < nl) {
        view_loss_sum(b, tile_loss, slots, (int)blockIdx.x);
        return;
    }
    uint32_t g = (blockIdx.x - nl) * blockDim.x + threadIdx.x;
    if (g >= b.total_g || cnt[g] == 0) return;
    const ViewDev& vw = b.v[view_of_gaussian(b, g)];
    const size_t l = g - vw.g_off;
    const float4* prm = vw.params + 4 * l;
    float4* grd = vw.grads + 4 * l;
    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0, o2 = o0, o3 = o0;
    if (!project_grad(g2d[3 * (size_t)g], g2d[3 * (size_t)g + 1], g2d[3 * (size_t)g + 2], prm[0], prm[1], prm[2],
                      prm[3], vw.cam, rc, o0, o1, o2, o3))
        return;
    if (shared_params) {
        atomicAdd(&grd[0], o0);
        atomicAdd(&grd[1], o1);
        atomicAdd(&grd[2], o2);
        atomicAdd(&grd[3], o3);
    } else {
        float4 c0 = grd[0], c1 = grd[1], c2 = grd[2], c3 = grd[3];
        grd[0] = make_float4(c0.x + o0.x, c0.y + o0.y, c0.z + o0.z, c0.w + o0.w);
        grd[1] = make_float4(c1.x + o1.x, c1.y + o1.y, c1.z + o1.z, c1.w + o1.w);
        grd[2] = make_float4(c2.x + o2.x, c2.y + o2.y, c2.z + o2.z, c2.w + o2.w);
        grd[3] = make_float4(c3.x + o3.x, c3.y + o3.y, c3.z + o3.z, c3.w + o3.w);
    }
}

// The fused training step's per-Gaussian kernel: the parameter gradient of
// every Gaussian of the batch (zero where no tile saw it), plus the
// accumulated one when the view has a gradient array (which is then zeroed),
// and the AdamW step of its record, exactly as gsc_cache_step would take it.
// One thread per Gaussian: the projection gradient is computed once (four
// threads per Gaussian, each owning one float4 of the record, were measured
// 1.6x slower: the projection arithmetic then runs four times).  64
// registers, 8 CTAs per SM: 5% faster than 80 registers and 6 CTAs (the
// kernel waits on memory), 30% faster than 12 CTAs with their spills.
__global__ void __launch_bounds__(128, 8) k_project_bwd_step(const __grid_constant__ BatchDev b, RasterDev rc,
                                                          const uint32_t* __restrict__ cnt,
                                                          const float4* __restrict__ g2d,
                                                          const __grid_constant__ AdamDev adam,
                                                          const float* __restrict__ tile_loss, int slots) {
    const uint32_t nl = tile_loss ? (uint32_t)b.nviews : 0u;
    if (blockIdx.x < nl) {
        view_loss_sum(b, tile_loss, slots, (int)blockIdx.x);
        return;
    }
    const uint32_t g = (blockIdx.x - nl) * blockDim.x + threadIdx.x;
    if (g >= b.total_g) return;
    const ViewDev& vw = b.v[view_of_gaussian(b, g)];
    const size_t l = g - vw.g_off;
    float4* prm = const_cast<float4*>(vw.params) + 4 * l;
    float4 P[4] = {prm[0], prm[1], prm[2], prm[3]};
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 G[4] = {z, z, z, z};
    if (cnt[g] != 0)
        project_grad(g2d[3 * (size_t)g], g2d[3 * (size_t)g + 1], g2d[3 * (size_t)g + 2], P[0], P[1], P[2], P[3],
                     vw.cam, rc, G[0], G[1], G[2], G[3]);
    float4* grd = vw.grads ? vw.grads + 4 * l : nullptr;
    float4* mp = vw.m + 4 * l;
    float4* vp = vw.v + 4 * l;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (grd) {
            const float4 c = grd[q];
            G[q] = make_float4(c.x + G[q].x, c.y + G[q].y, c.z + G[q].z, c.w + G[q].w);
            grd[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float4 m = mp[q], v = vp[q];
        adam_four(P[q], m, v, G[q], q, adam);
        prm[q] = P[q];
        mp[q] = m;
        vp[q] = v;
    }
}

// ------------------------------------------------------------------ host

static int bits_for(uint32_t n) {
    int b = 1;
    while (b < 32 && (1u << b) < n) ++b;
    return b;
}

// Order in which the persistent CTAs take the tiles: by the length of the
// tile's bin list, longest first (a longest-processing-time-first schedule,
// so that the cheap tiles fill the end of the launch).  Class of a bin (and
// of its tiles) = 255 - 8 log2(length + 1).  The tiles of a bin are placed
// together in row-major order; the order of the bins within a class is
// whatever the atomics give, since it only decides which CTA renders a tile,
// never a result.
constexpr int kOrderThreads = 1024;

// Cost class of a tile or bin (0: the most costly), with the hardware log2:
// a class only decides which CTA renders a tile, never a result.
__device__ __forceinline__ uint32_t order_class(float c) {
    const float l = __log2f(c + 1.0f) * 8.0f;
    return (uint32_t)(kOrderClasses - 1) - (uint32_t)fminf(l, (float)(kOrderClasses - 1));
}
// Parts a tile of feedback cost c is split into.  A one-warp CTA splits a
// tile above half the mean load of a CTA into up to 4 parts.  A larger CTA
// walks a tile faster alone, and every part redoes the list filter and the
// gradient reductions, so it splits only the tiles that would outlast the
// mean load (above 0.75 of it), in 2 parts: once the cache has trained, a
// few such tiles set the length of the launch (measured at 2 and 4 pixels
// per thread).  `total`: the summed cost of all tiles, `grid`: the CTAs.
struct SplitRule {
    float split_at;
    uint32_t max_parts;
    __device__ SplitRule(const RasterDev& rc, unsigned long long total, int grid) {
        const bool one_warp = rc.tile_w * rc.tile_h / rc.ppt <= 32;
        max_parts = (uint32_t)min(one_warp ? 4 : 2, rc.ppt);
        split_at = (one_warp ? 0.5f : 0.75f) * (float)total / (float)max(grid, 1);
    }
    __device__ uint32_t parts(uint32_t c) const { return (max_parts > 1 && (float)c > split_at) ? max_parts : 1u; }
};
// cost of one part of a tile of cost c split in p: a part redoes the
// per-entry work, (p + 1) / 2p of it
__device__ __forceinline__ float part_cost(uint32_t c, uint32_t p) {
    return (float)c * (p == 1u ? 1.0f : (p == 2u ? 0.75f : 0.625f));
}

__device__ __forceinline__ int view_of_bin(const BatchDev& b, uint32_t bin) {
    int v = 0;
    while (v + 1 < b.nviews && bin >= b.v[v + 1].bin_off) ++v;
    return v;
}

// Geometry of a batch as far as the per-tile feedback is concerned: the tile
// grid of every view (FNV-1a over the words; never 0, which means none).
__device__ uint32_t batch_signature(const BatchDev& b, const RasterDev& rc) {
    uint32_t h = 2166136261u;
    auto mix = [&](uint32_t w) { h = (h ^ w) * 16777619u; };
    mix((uint32_t)b.nviews);
    mix(b.total_tiles);
    mix((uint32_t)rc.tile_w);
    mix((uint32_t)rc.tile_h);
    for (int v = 0; v < b.nviews; ++v) {
        mix((uint32_t)b.v[v].tiles_x);
        mix((uint32_t)b.v[v].tiles_y);
    }
    return h | 1u;
}

// Per-tile cost for the feedback order, ahead of k_tile_order: the largest
// front-to-back hit count plus back-to-front length of the last gradient
// launch among a tile and its eight neighbours (the view moves a little
// between frames), and the sum of the tiles' own costs.  It also clears the
// buffer the coming gradient kernel writes.
constexpr int kCostThreads = 256;
__global__ void __launch_bounds__(kCostThreads) k_tile_cost(const __grid_constant__ BatchDev b,
                                                            uint32_t* __restrict__ fb, uint32_t fb_stride,
                                                            uint32_t* __restrict__ fb_state) {
    __shared__ unsigned long long s_sum[kCostThreads / 32];
    const uint32_t parity = fb_state[kFbParity];
    const uint32_t* fb_hit = fb + 2 * (size_t)fb_stride * (parity & 1u);  // written by the last gradient launch
    const uint32_t* fb_len = fb_hit + fb_stride;
    uint32_t* w_hit = fb + 2 * (size_t)fb_stride * ((parity + 1u) & 1u);
    uint32_t* cost = fb + 4 * (size_t)fb_stride;
    unsigned long long own = 0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < b.total_tiles; t += gridDim.x * blockDim.x) {
        const ViewDev& vw = b.v[view_of_tile(b, t)];
        const uint32_t lt = t - vw.tile_off;
        const int tx = (int)(lt % (uint32_t)vw.tiles_x), ty = (int)(lt / (uint32_t)vw.tiles_x);
        uint32_t c = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = tx + dx, y = ty + dy;
                if (x < 0 || y < 0 || x >= vw.tiles_x || y >= vw.tiles_y) continue;
                const uint32_t u = vw.tile_off + (uint32_t)(y * vw.tiles_x + x);
                c = max(c, fb_hit[u] + fb_len[u]);
            }
        cost[t] = c;
        own += fb_hit[t] + fb_len[t];
        w_hit[t] = 0u;
        w_hit[fb_stride + t] = 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) own += __shfl_xor_sync(kFull, own, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = own;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kCostThreads / 32; ++w) t += s_sum[w];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(fb_state + kFbTotal), t);
    }
}

// Per tile its parts and cost class from the feedback cost (k_tile_cost),
// stored in place of the cost as class | parts << 8, and the work items per
// class summed into order_cls[0 .. kOrderClasses) (a histogram per CTA
// first).  Many CTAs, so that no single SM walks every tile.
__global__ void __launch_bounds__(kCostThreads) k_tile_class(const __grid_constant__ BatchDev b, RasterDev rc,
                                                             uint32_t* __restrict__ fb, uint32_t fb_stride,
                                                             const uint32_t* __restrict__ fb_state, int grid,
                                                             uint32_t* __restrict__ order_cls) {
    __shared__ uint32_t h[kOrderClasses];
    for (int k = threadIdx.x; k < kOrderClasses; k += kCostThreads) h[k] = 0;
    __syncthreads();
    const SplitRule rule(rc, *reinterpret_cast<const unsigned long long*>(fb_state + kFbTotal), grid);
    uint32_t* cost = fb + 4 * (size_t)fb_stride;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < b.total_tiles; t += gridDim.x * blockDim.x) {
        const uint32_t c = cost[t], p = rule.parts(c), k = order_class(part_cost(c, p));
        cost[t] = k | (p << 8);
        atomicAdd(&h[k], p);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kOrderClasses; k += kCostThreads)
        if (h[k]) atomicAdd(&order_cls[k], h[k]);
}

// Work items of the feedback order: every tile takes its parts' slots in
// its class from the class cursors (k_tile_order) and writes its items.  The
// order within a class is whatever the atomics give.
__global__ void __launch_bounds__(kCostThreads) k_tile_scatter(const __grid_constant__ BatchDev b,
                                                               const uint32_t* __restrict__ fb, uint32_t fb_stride,
                                                               const uint32_t* __restrict__ fb_state,
                                                               uint32_t* __restrict__ order_cls,
                                                               uint32_t* __restrict__ order) {
    if (fb_state[kFbUse] == 0u) return;  // the order kernel took the plain order
    const uint32_t* kp = fb + 4 * (size_t)fb_stride;
    uint32_t* cursor = order_cls + kOrderClasses;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < b.total_tiles; t += gridDim.x * blockDim.x) {
        const uint32_t v = kp[t], k = v & 0xffu, p = v >> 8;
        const uint32_t st = atomicAdd(&cursor[k], p);
        const uint32_t lp = p == 4 ? 2u : (p == 2 ? 1u : 0u);
        for (uint32_t q = 0; q < p; ++q) order[st + q] = make_item(t, q, lp);
    }
}

// One CTA.  With `totals` (the digit counts of a one-pass pair sort, where
// the digit is the whole bin id) it first writes every bin's range as the
// exclusive scan of the counts.  Then the work items, longest first:
//
// kOrderPlain, or kOrderFeedback without usable feedback: per bin its class
// and tile count; the tile counts are summed per class and scanned, and every
// bin takes its start in its class and writes its tiles there in row-major
// order.
//
// kOrderFeedback with feedback from the last gradient launch of the same
// geometry: the items are ordered by the tile costs k_tile_cost wrote and
// split by SplitRule; k_tile_class has counted the items per class, this
// kernel scans the counts into class cursors, and k_tile_scatter writes the
// items.  The order and the split decide which CTA renders which pixels,
// never a result.  In feedback mode it also advances the launch parity and
// resets the cost sum.
__global__ void __launch_bounds__(kOrderThreads) k_tile_order(const __grid_constant__ BatchDev b,
                                                              const uint32_t* __restrict__ totals,
                                                              uint2* __restrict__ ranges, RasterDev rc,
                                                              uint32_t* __restrict__ order, int mode, int grid,
                                                              uint32_t* __restrict__ fb, uint32_t fb_stride,
                                                              uint32_t* __restrict__ fb_state,
                                                              uint32_t* __restrict__ order_cls) {
    __shared__ uint32_t cls[kOrderClasses];
    __shared__ uint32_t wsum[kOrderThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // exclusive scan of one value per thread
    auto block_scan = [&](uint32_t v) -> uint32_t {
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        __syncthreads();
        return before + x - v;
    };
    const uint32_t nb = b.total_bins, nt = b.total_tiles;
    if (totals) {  // the caller guarantees nb <= kOrderThreads here
        uint32_t c = threadIdx.x < nb ? totals[threadIdx.x] : 0u;
        uint32_t s = block_scan(c);
        if (threadIdx.x < nb) ranges[threadIdx.x] = make_uint2(s, s + c);
    }
    if (threadIdx.x < kOrderClasses) cls[threadIdx.x] = 0;
    bool use_fb = false;
    uint32_t sig = 0, parity = 0;
    if (mode == kOrderFeedback) {
        sig = batch_signature(b, rc);
        parity = fb_state[kFbParity];
        use_fb = fb_state[kFbSignature] == sig && grid > 0;
    }
    __syncthreads();  // also makes the ranges written above visible to the CTA
    auto klass_of = [](float c) -> uint32_t { return order_class(c); };
    if (use_fb) {
        // the classes and their item counts come from k_tile_class; the
        // cursors go to k_tile_scatter, which writes the items
        uint32_t v = threadIdx.x < kOrderClasses ? order_cls[threadIdx.x] : 0u;
        uint32_t sc = block_scan(v);
        if (threadIdx.x < kOrderClasses) {
            order_cls[kOrderClasses + threadIdx.x] = sc;
            order_cls[threadIdx.x] = 0u;  // for the next binning
        }
        if (threadIdx.x == kOrderClasses - 1) fb_state[kFbItems] = sc + v;
        if (threadIdx.x == 0) fb_state[kFbUse] = 1u;
    } else {
        auto bin_info = [&](uint32_t bin, uint32_t& klass, uint32_t& ntiles) {
            const ViewDev& vw = b.v[view_of_bin(b, bin)];
            const uint32_t lb = bin - vw.bin_off;
            const int bx = (int)(lb % (uint32_t)vw.bins_x), by = (int)(lb / (uint32_t)vw.bins_x);
            const int w = min(vw.spt_x, vw.tiles_x - bx * vw.spt_x), h = min(vw.spt_y, vw.tiles_y - by * vw.spt_y);
            ntiles = (uint32_t)(w * h);
            const uint2 rg = ranges[bin];
            klass = klass_of((float)(rg.y - rg.x));
        };
        for (uint32_t bin = threadIdx.x; bin < nb; bin += kOrderThreads) {
            uint32_t k, n;
            bin_info(bin, k, n);
            atomicAdd(&cls[k], n);
        }
        __syncthreads();
        uint32_t c = threadIdx.x < kOrderClasses ? cls[threadIdx.x] : 0u;
        uint32_t s = block_scan(c);
        if (threadIdx.x < kOrderClasses) cls[threadIdx.x] = s;
        __syncthreads();
        // one warp per bin: it takes the bin's start in its class and writes
        // the bin's tiles, row-major, 32 at a time
        for (uint32_t bin = warp; bin < nb; bin += kOrderThreads / 32) {
            uint32_t k, n;
            bin_info(bin, k, n);
            uint32_t st = 0;
            if (lane == 0) st = atomicAdd(&cls[k], n);
            st = __shfl_sync(kFull, st, 0);
            const ViewDev& vw = b.v[view_of_bin(b, bin)];
            const uint32_t lb = bin - vw.bin_off;
            const int bx = (int)(lb % (uint32_t)vw.bins_x), by = (int)(lb / (uint32_t)vw.bins_x);
            const int w = min(vw.spt_x, vw.tiles_x - bx * vw.spt_x);
            for (uint32_t li = (uint32_t)lane; li < n; li += 32) {
                const int ry = (int)li / w, rx = (int)li - ry * w;
                order[st + li] = vw.tile_off + (uint32_t)((by * vw.spt_y + ry) * vw.tiles_x + bx * vw.spt_x + rx);
            }
        }
        if (threadIdx.x == 0) fb_state[kFbItems] = nt;
        if (mode == kOrderFeedback) {
            if (threadIdx.x < kOrderClasses) order_cls[threadIdx.x] = 0u;  // counted by k_tile_class, unused
            if (threadIdx.x == 0) fb_state[kFbUse] = 0u;
        }
    }
    if (mode == kOrderFeedback) {
        __syncthreads();  // every read of the state above is done
        if (threadIdx.x == 0) {
            fb_state[kFbParity] = parity + 1u;
            fb_state[kFbSignature] = sig;
            *reinterpret_cast<unsigned long long*>(fb_state + kFbTotal) = 0ull;
        }
    }
}

// persistent CTAs of the gradient kernel of this launch configuration
static int bwd_grid_hint(const RasterDev& rc, uint32_t tiles);

cudaError_t bin_gaussians(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t** sorted_vals,
                          cudaStream_t s, int order_mode) {
    uint32_t n = b.total_g;
    uint32_t nblk = (n + 255) / 256;
    if (nblk == 0) nblk = 1;
    {
        PhaseScope ph(kPhProject, s, 1);
        k_project<<<nblk, 256, 0, s>>>(b, rc, ws->rec, ws->key0, ws->idx0, ws->rect, ws->cnt);
    }
    int w;
    {
        // the one-sweep sort's published counts hold 30 bits
        const bool sweep = n < (1u << 30);
        PhaseScope ph(kPhDepthSort, s, sweep ? 1 + 4 : 3 * 4);
        w = sweep ? radix_sort_onesweep(ws->key0, ws->idx0, ws->key1, ws->idx1, n, ws->sweep, ws->status, s)
                  : radix_sort_pairs(ws->key0, ws->idx0, ws->key1, ws->idx1, nullptr, n, 32, sort_blocks_for(n),
                                     ws->hist, s);
    }
    const uint32_t* sidx = w ? ws->idx1 : ws->idx0;
    {
        PhaseScope ph(kPhScan, s, 3);
        scan_gathered(ws->cnt, sidx, n, ws->off, ws->scan_sums, ws->counters, ws->status, (uint32_t)ws->max_pairs,
                      ws->stats, s);
    }
    {
        PhaseScope ph(kPhEmit, s, 1);
        k_emit<<<nblk, 256, 0, s>>>(b, sidx, ws->off, ws->cnt, ws->rect, ws->rec, rc, ws->counters, ws->pkey0,
                                    ws->pval0, ws->stats);
    }
    uint32_t bins = b.total_bins;
    int bits = bits_for(bins + 1);  // key total_bins: culled pairs
    int p;
    {
        PhaseScope ph(kPhTileSort, s, 3 * radix_passes(bits));
        p = radix_sort_pairs(ws->pkey0, ws->pval0, ws->pkey1, ws->pval1, ws->counters + kCntPairs,
                             (uint32_t)ws->max_pairs, bits, ws->sort_blocks, ws->hist, s);
    }
    const uint32_t* keys = p ? ws->pkey1 : ws->pkey0;
    *sorted_vals = p ? ws->pval1 : ws->pval0;
    {
        // one radix pass: its digit counts are the bin sizes, and the ranges
        // are their exclusive scan (done by k_tile_order); more passes: the
        // ranges come from the boundaries of the sorted keys
        const bool one_pass = radix_passes(bits) == 1 && bins <= (uint32_t)kOrderThreads;
        PhaseScope ph(kPhRanges, s, (one_pass ? 1 : 2) + (order_mode == kOrderFeedback ? 3 : 0));
        if (!one_pass) {
            cudaMemsetAsync(ws->ranges, 0, sizeof(uint2) * bins, s);
            k_ranges<<<152 * 8, 256, 0, s>>>(keys, ws->counters, ws->ranges, bins);
        }
        const int grid = order_mode == kOrderFeedback ? bwd_grid_hint(rc, b.total_tiles) : 0;
        uint32_t nblk = min((b.total_tiles + kCostThreads - 1) / kCostThreads, 152u * 4u);
        nblk = nblk ? nblk : 1u;
        const uint32_t fbs = (uint32_t)ws->max_tiles;
        if (order_mode == kOrderFeedback) {
            k_tile_cost<<<nblk, kCostThreads, 0, s>>>(b, ws->fb, fbs, ws->fb_state);
            k_tile_class<<<nblk, kCostThreads, 0, s>>>(b, rc, ws->fb, fbs, ws->fb_state, grid, ws->order_cls);
        }
        k_tile_order<<<1, kOrderThreads, 0, s>>>(b, one_pass ? radix_totals(ws->hist) : nullptr, ws->ranges, rc,
                                                 ws->tile_order, order_mode, grid, ws->fb, fbs, ws->fb_state,
                                                 ws->order_cls);
        if (order_mode == kOrderFeedback)
            k_tile_scatter<<<nblk, kCostThreads, 0, s>>>(b, ws->fb, fbs, ws->fb_state, ws->order_cls, ws->tile_order);
        ws->order = ws->tile_order;
    }
    return cudaGetLastError();
}

// Raise a kernel's dynamic shared-memory limit when a launch needs more than
// the default (which also has to hold the kernel's static shared memory).
template <typename K>
static cudaError_t ensure_smem(K kern, size_t bytes, int* cached) {
    if ((int)bytes <= *cached) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) *cached = (int)bytes;
    return e;
}

// Grid of a persistent kernel: every CTA that fits on the device at once
// (queried for this kernel, block size and shared memory), at most one per tile.
template <typename K>
static int persistent_grid(K kern, int threads, size_t smem, uint32_t tiles, size_t* cached_smem, int* cached_grid) {
    if (*cached_smem != smem || *cached_grid <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
        *cached_grid = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
        *cached_smem = smem;
    }
    return (int)((uint32_t)*cached_grid < tiles ? (uint32_t)*cached_grid : (tiles ? tiles : 1));
}

template <int TW, int TH, int PPT>
static cudaError_t render_t(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                            cudaStream_t s) {
    size_t smem = sizeof(float4) * 3 * rc.cap;
    auto kern = k_render<TW, TH, PPT>;
    static int cached = 32 * 1024;
    cudaError_t e = ensure_smem(kern, smem, &cached);
    if (e != cudaSuccess) return e;
    static size_t gs = 0;
    static int gg = 0;
    int grid = persistent_grid(kern, TW * TH / PPT, smem, b.total_tiles, &gs, &gg);
    cudaMemsetAsync(ws->counters + kCntTilesFwd, 0, sizeof(uint32_t), s);
    kern<<<grid, TW * TH / PPT, smem, s>>>(b, ws->ranges, vals, ws->rect, ws->rec, rc, ws->counters + kCntTilesFwd,
                                           ws->stats, ws->order);
    return cudaGetLastError();
}

template <int TW, int TH, int PPT, int LOSS>
static size_t bwd_smem(const RasterDev& rc) {
    return sizeof(float4) * 3 * rc.cap + (sizeof(uint32_t) << rc.ring_log2);
}

// grid of the gradient kernel: every CTA that fits at once, at most one per
// work item (a tile is at most 4 items)
template <int TW, int TH, int PPT, int LOSS>
static cudaError_t bwd_grid(const RasterDev& rc, uint32_t tiles, int* grid) {
    const size_t smem = bwd_smem<TW, TH, PPT, LOSS>(rc);
    auto kern = k_render_bwd<TW, TH, PPT, LOSS>;
    static int cached = 32 * 1024;
    cudaError_t e = ensure_smem(kern, smem, &cached);
    if (e != cudaSuccess) return e;
    static size_t gs = 0;
    static int gg = 0;
    *grid = persistent_grid(kern, TW * TH / PPT, smem, 4 * tiles, &gs, &gg);
    return cudaSuccess;
}

template <int TW, int TH, int PPT, int LOSS>
static cudaError_t render_bwd_t(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                                cudaStream_t s) {
    int grid = 0;
    cudaError_t e = bwd_grid<TW, TH, PPT, LOSS>(rc, b.total_tiles, &grid);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(ws->counters + kCntTilesBwd, 0, sizeof(uint32_t), s);
    k_render_bwd<TW, TH, PPT, LOSS><<<grid, TW * TH / PPT, bwd_smem<TW, TH, PPT, LOSS>(rc), s>>>(
        b, ws->ranges, vals, ws->rect, ws->rec, rc, ws->g2d, ws->counters + kCntTilesBwd, ws->stats, ws->red,
        ws->order, ws->fb_state, ws->fb, (uint32_t)ws->max_tiles);
    return cudaGetLastError();
}

template <int TW, int TH, int PPT>
static cudaError_t bwd_plain(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                             cudaStream_t s) {
    return render_bwd_t<TW, TH, PPT, kLossNone>(b, rc, ws, vals, s);
}
template <int TW, int TH, int PPT>
static cudaError_t bwd_train_hdr(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                                 cudaStream_t s) {
    return render_bwd_t<TW, TH, PPT, kLossHdr>(b, rc, ws, vals, s);
}
template <int TW, int TH, int PPT>
static cudaError_t bwd_train_hdr_full(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws,
                                      const uint32_t* vals, cudaStream_t s) {
    return render_bwd_t<TW, TH, PPT, kLossHdrFull>(b, rc, ws, vals, s);
}

// the (tile, pixels per thread) pairs compiled; the API accepts exactly these
#define GSC_TILE_DISPATCH(FN, ...)                                                            \
    switch (rc.ppt) {                                                                         \
    case 8:                                                                                   \
        if (rc.tile_w == 16 && rc.tile_h == 16) return FN<16, 16, 8>(__VA_ARGS__);            \
        if (rc.tile_w == 32 && rc.tile_h == 8) return FN<32, 8, 8>(__VA_ARGS__);              \
        if (rc.tile_w == 8 && rc.tile_h == 32) return FN<8, 32, 8>(__VA_ARGS__);              \
        return cudaErrorInvalidValue;                                                         \
    case 4:                                                                                   \
        if (rc.tile_w == 16 && rc.tile_h == 16) return FN<16, 16, 4>(__VA_ARGS__);            \
        if (rc.tile_w == 32 && rc.tile_h == 8) return FN<32, 8, 4>(__VA_ARGS__);              \
        if (rc.tile_w == 8 && rc.tile_h == 32) return FN<8, 32, 4>(__VA_ARGS__);              \
        return cudaErrorInvalidValue;                                                         \
    case 2:                                                                                   \
        if (rc.tile_w == 16 && rc.tile_h == 16) return FN<16, 16, 2>(__VA_ARGS__);            \
        if (rc.tile_w == 32 && rc.tile_h == 8) return FN<32, 8, 2>(__VA_ARGS__);              \
        if (rc.tile_w == 16 && rc.tile_h == 8) return FN<16, 8, 2>(__VA_ARGS__);              \
        if (rc.tile_w == 8 && rc.tile_h == 16) return FN<8, 16, 2>(__VA_ARGS__);              \
        if (rc.tile_w == 8 && rc.tile_h == 32) return FN<8, 32, 2>(__VA_ARGS__);              \
        return cudaErrorInvalidValue;                                                         \
    default:                                                                                  \
        if (rc.tile_w == 16 && rc.tile_h == 16) return FN<16, 16, 1>(__VA_ARGS__);            \
        if (rc.tile_w == 8 && rc.tile_h == 8) return FN<8, 8, 1>(__VA_ARGS__);                \
        if (rc.tile_w == 32 && rc.tile_h == 8) return FN<32, 8, 1>(__VA_ARGS__);              \
        if (rc.tile_w == 16 && rc.tile_h == 8) return FN<16, 8, 1>(__VA_ARGS__);              \
        if (rc.tile_w == 8 && rc.tile_h == 16) return FN<8, 16, 1>(__VA_ARGS__);              \
        if (rc.tile_w == 8 && rc.tile_h == 32) return FN<8, 32, 1>(__VA_ARGS__);              \
        if (rc.tile_w == 32 && rc.tile_h == 4) return FN<32, 4, 1>(__VA_ARGS__);              \
        return cudaErrorInvalidValue;                                                         \
    }

template <int TW, int TH, int PPT>
static cudaError_t bwd_grid_t(const RasterDev& rc, uint32_t tiles, int* grid) {
    return bwd_grid<TW, TH, PPT, kLossHdr>(rc, tiles, grid);
}

static int bwd_grid_hint(const RasterDev& rc, uint32_t tiles) {
    int g = 0;
    auto f = [&]() -> cudaError_t { GSC_TILE_DISPATCH(bwd_grid_t, rc, tiles, &g) };
    return f() == cudaSuccess ? g : 0;
}

cudaError_t launch_render(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                          cudaStream_t s) {
    PhaseScope ph(kPhRender, s, 1);
    GSC_TILE_DISPATCH(render_t, b, rc, ws, vals, s)
}

// tile_loss (nullable): the training step's loss partials, `slots` per tile,
// summed into each view's loss by the first blocks of the launch
static cudaError_t project_backward(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, bool shared_params,
                                    const AdamDev* adam, const float* tile_loss, int slots, cudaStream_t s) {
    uint32_t nblk = (b.total_g + 127) / 128 + (tile_loss ? (uint32_t)b.nviews : 0u);
    if (nblk == 0) nblk = 1;
    if (adam) {
        PhaseScope ph(kPhAdam, s, 1);
        k_project_bwd_step<<<nblk, 128, 0, s>>>(b, rc, ws->cnt, ws->g2d, *adam, tile_loss, slots);
    } else {
        PhaseScope ph(kPhProjectBwd, s, 1);
        k_project_bwd<<<nblk, 128, 0, s>>>(b, rc, ws->cnt, ws->g2d, shared_params ? 1 : 0, tile_loss, slots);
    }
    return cudaGetLastError();
}

cudaError_t launch_render_backward(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                                   bool shared_params, cudaStream_t s) {
    cudaError_t e;
    {
        PhaseScope ph(kPhRenderBwd, s, 1);
        cudaMemsetAsync(ws->g2d, 0, sizeof(float4) * 3 * (size_t)b.total_g, s);
        auto launch = [&]() -> cudaError_t { GSC_TILE_DISPATCH(bwd_plain, b, rc, ws, vals, s) };
        e = launch();
    }
    if (e != cudaSuccess) return e;
    return project_backward(b, rc, ws, shared_params, nullptr, nullptr, 0, s);
}

cudaError_t launch_train(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                         int full_grad, bool shared_params, const AdamDev* adam, cudaStream_t s) {
    cudaError_t e;
    {
        PhaseScope ph(kPhTrain, s, 1);
        cudaMemsetAsync(ws->g2d, 0, sizeof(float4) * 3 * (size_t)b.total_g, s);
        auto launch = [&]() -> cudaError_t {
            if (full_grad) { GSC_TILE_DISPATCH(bwd_train_hdr_full, b, rc, ws, vals, s) }
            GSC_TILE_DISPATCH(bwd_train_hdr, b, rc, ws, vals, s)
        };
        e = launch();
    }
    if (e != cudaSuccess) return e;
    return project_backward(b, rc, ws, shared_params, adam, ws->red, loss_slots(rc.tile_w * rc.tile_h / rc.ppt), s);
}

}  // namespace gsc
