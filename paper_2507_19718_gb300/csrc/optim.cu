// Losses of the cache optimisation and the per-frame AdamW step
// (GSCache Sec. 3.6: HDR loss, per-attribute learning rates, the Eq. 4
// schedule folded into lr_scale, AdamW's decoupled weight decay).
//
// All kernels stream their operands once with coalesced float4 / float
// accesses; they are HBM-bound.  Loss sums are reduced deterministically
// (fixed per-CTA partials, then one CTA in FP64).
#include "gsc_internal.cuh"

namespace gsc {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 152 * 4;

__device__ __forceinline__ float block_sum(float v, float* sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sm[k];
    return t;  // valid in thread 0
}

// (x - y)^2 / (y + 0.01)^2 per element of the crop; y = prediction
__global__ void __launch_bounds__(kRedThreads) k_loss_hdr(const float* __restrict__ pred,
                                                          const float* __restrict__ tgt, int C, int H, int W, int x0,
                                                          int y0, int w, int h, int full, float invk,
                                                          float* __restrict__ dL, float* __restrict__ partial) {
    __shared__ float sm[32];
    size_t n = (size_t)C * w * h, plane = (size_t)w * h;
    float acc = 0.f;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        int ch = (int)(e / plane);
        size_t r = e - (size_t)ch * plane;
        int jj = (int)(r / w), ii = (int)(r - (size_t)jj * w);
        size_t p = ((size_t)ch * H + (y0 + jj)) * W + (x0 + ii);
        float y = pred[p], x = tgt[p];
        acc += hdr_term(y, x);
        if (dL) dL[p] = hdr_grad(y, x, full != 0, invk);
    }
    float t = block_sum(acc, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_reduce_final(const float* __restrict__ partial, int n, double scale, float* __restrict__ out) {
    __shared__ double sm[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += (double)partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sm[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sm[k];
        *out = (float)(t * scale);
    }
}

// ------------------------------------------------------------------ L1 + D-SSIM
//
// 0.8 L1 + 0.2 (1 - SSIM) over the crop, treated as its own zero-padded
// image; SSIM of Wang et al. (2004) per channel with an 11x11 Gaussian window
// (sigma 1.5, normalised), C1 = 0.01^2, C2 = 0.03^2.  Pass 1 computes the
// windowed moments of every crop pixel directly (121 taps), the SSIM value
// and its partial derivatives with respect to mu_x, E[x^2] and E[xy]; pass 2
// correlates those three maps with the window:
//   d mean(SSIM) / d x_q = (w * g_mu)(q) + 2 x_q (w * g_xx)(q) + y_q (w * g_xy)(q).
struct SsimDev {
    float w[11];
};

constexpr int kSsimScratchOffset = 65536;  // floats of the reduction area before the maps

__global__ void __launch_bounds__(kRedThreads) k_ssim_fwd(const float* __restrict__ pred,
                                                          const float* __restrict__ tgt, int C, int H, int W,
                                                          int x0, int y0, int w, int h, SsimDev win,
                                                          float* __restrict__ gmaps, float* __restrict__ partial) {
    __shared__ float sm[32];
    const float C1 = 1e-4f, C2 = 9e-4f;
    size_t plane = (size_t)w * h, n = (size_t)C * plane;
    float l1 = 0.f, ssum = 0.f;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        int ch = (int)(e / plane);
        size_t r = e - (size_t)ch * plane;
        int j = (int)(r / w), i = (int)(r - (size_t)j * w);
        float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
        for (int dy = -5; dy <= 5; ++dy) {
            int jj = j + dy;
            if (jj < 0 || jj >= h) continue;
            const float* px = pred + ((size_t)ch * H + (y0 + jj)) * W + x0;
            const float* py = tgt + ((size_t)ch * H + (y0 + jj)) * W + x0;
            float wy = win.w[dy + 5];
#pragma unroll
            for (int dx = -5; dx <= 5; ++dx) {
                int ii = i + dx;
                if (ii < 0 || ii >= w) continue;
                float ww = wy * win.w[dx + 5];
                float xv = px[ii], yv = py[ii];
                mx = fmaf(ww, xv, mx);
                my = fmaf(ww, yv, my);
                exx = fmaf(ww, xv * xv, exx);
                eyy = fmaf(ww, yv * yv, eyy);
                exy = fmaf(ww, xv * yv, exy);
            }
        }
        float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
        float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy + C2;
        float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
        float inv = 1.f / (B1 * B2);
        float sv = A1 * A2 * inv;
        ssum += sv;
        // partials with mu_y and E[y^2] held fixed
        float gmu = (2.f * my * A2 - 2.f * my * A1) * inv - sv * (2.f * mx * B2 - 2.f * mx * B1) * inv;
        gmaps[e] = gmu;
        gmaps[n + e] = -sv / B2;
        gmaps[2 * n + e] = 2.f * A1 * inv;
        size_t p = ((size_t)ch * H + (y0 + j)) * W + (x0 + i);
        l1 += fabsf(pred[p] - tgt[p]);
    }
    float t1 = block_sum(l1, sm);
    float t2 = block_sum(ssum, sm);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = t1;
        partial[gridDim.x + blockIdx.x] = t2;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_ssim_bwd(const float* __restrict__ pred,
                                                          const float* __restrict__ tgt, int C, int H, int W,
                                                          int x0, int y0, int w, int h, SsimDev win, float invk,
                                                          const float* __restrict__ gmaps, float* __restrict__ dL) {
    size_t plane = (size_t)w * h, n = (size_t)C * plane;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        int ch = (int)(e / plane);
        size_t r = e - (size_t)ch * plane;
        int j = (int)(r / w), i = (int)(r - (size_t)j * w);
        float fmu = 0.f, fxx = 0.f, fxy = 0.f;
        for (int dy = -5; dy <= 5; ++dy) {
            int jj = j + dy;
            if (jj < 0 || jj >= h) continue;
            size_t rowb = (size_t)ch * plane + (size_t)jj * w;
            float wy = win.w[dy + 5];
#pragma unroll
            for (int dx = -5; dx <= 5; ++dx) {
                int ii = i + dx;
                if (ii < 0 || ii >= w) continue;
                float ww = wy * win.w[dx + 5];
                size_t q = rowb + ii;
                fmu = fmaf(ww, gmaps[q], fmu);
                fxx = fmaf(ww, gmaps[n + q], fxx);
                fxy = fmaf(ww, gmaps[2 * n + q], fxy);
            }
        }
        size_t p = ((size_t)ch * H + (y0 + j)) * W + (x0 + i);
        float xv = pred[p], yv = tgt[p];
        float ds = fmu + 2.f * xv * fxx + yv * fxy;
        float d = xv - yv;
        float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        dL[p] = (0.8f * sg - 0.2f * ds) * invk;
    }
}

__global__ void k_ssim_final(const float* __restrict__ partial, int nb, double invk, float* __restrict__ out) {
    __shared__ double sm1[32], sm2[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += (double)partial[i];
        b += (double)partial[nb + i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(kFull, a, o);
        b += __shfl_xor_sync(kFull, b, o);
    }
    int wq = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sm1[wq] = a;
        sm2[wq] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double l1 = 0.0, ss = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            l1 += sm1[k];
            ss += sm2[k];
        }
        *out = (float)(0.8 * l1 * invk + 0.2 * (1.0 - ss * invk));
    }
}

cudaError_t launch_loss(int kind, const float* pred, const float* target, int C, int H, int W, int x0, int y0,
                        int w, int h, float* dL_dpred, float* loss_out, float* red, size_t red_floats,
                        cudaStream_t s) {
    size_t n = (size_t)C * w * h;
    if (dL_dpred && (x0 != 0 || y0 != 0 || w != W || h != H)) {
        cudaError_t e = cudaMemsetAsync(dL_dpred, 0, sizeof(float) * (size_t)C * H * W, s);
        if (e != cudaSuccess) return e;
    }
    if (kind == GSC_LOSS_HDR || kind == GSC_LOSS_HDR_FULLGRAD) {
        int blocks = (int)((n + kRedThreads - 1) / kRedThreads);
        if (blocks > kRedBlocks) blocks = kRedBlocks;
        if (blocks < 1) blocks = 1;
        if ((size_t)blocks > red_floats) return cudaErrorInvalidValue;
        float invk = n ? (float)(1.0 / (double)n) : 0.f;
        PhaseScope ph(kPhLoss, s, 2);
        k_loss_hdr<<<blocks, kRedThreads, 0, s>>>(pred, target, C, H, W, x0, y0, w, h,
                                                  kind == GSC_LOSS_HDR_FULLGRAD, invk, dL_dpred, red);
        k_reduce_final<<<1, 1024, 0, s>>>(red, blocks, n ? 1.0 / (double)n : 0.0, loss_out);
        return cudaGetLastError();
    }
    if (kind == GSC_LOSS_L1_SSIM) {
        if (red_floats < (size_t)kSsimScratchOffset + 3 * n) return cudaErrorMemoryAllocation;
        SsimDev win;
        double ws[11], tot = 0.0;
        for (int k = 0; k < 11; ++k) {
            ws[k] = exp(-(double)((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5));
            tot += ws[k];
        }
        for (int k = 0; k < 11; ++k) win.w[k] = (float)(ws[k] / tot);
        int blocks = (int)((n + kRedThreads - 1) / kRedThreads);
        if (blocks > kRedBlocks) blocks = kRedBlocks;
        if (blocks < 1) blocks = 1;
        float* gmaps = red + kSsimScratchOffset;
        PhaseScope ph(kPhLoss, s, dL_dpred ? 3 : 2);
        k_ssim_fwd<<<blocks, kRedThreads, 0, s>>>(pred, target, C, H, W, x0, y0, w, h, win, gmaps, red);
        if (dL_dpred)
            k_ssim_bwd<<<blocks, kRedThreads, 0, s>>>(pred, target, C, H, W, x0, y0, w, h, win,
                                                      (float)(1.0 / (double)n), gmaps, dL_dpred);
        k_ssim_final<<<1, 1024, 0, s>>>(red, blocks, 1.0 / (double)n, loss_out);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ loss without a workspace
//
// gsc_loss_noalloc: the same two kernels as gsc_loss, launched with one CTA
// per 256 elements, whose partial sums go to the file-scope array below
// instead of a workspace.  The array is the library's own: every device that
// loads the library holds it (128 KiB) until the process exits.  Host code
// may not pass the symbol itself to a kernel (on the host it is only a
// stand-in); its device address is looked up once per device.

constexpr int kNoAllocSlots = 32768;  // partial sums = CTAs of 256 elements
static __device__ __align__(256) float g_noalloc_partials[kNoAllocSlots];

}  // namespace gsc

#include <mutex>

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

extern "C" gsc_status gsc_loss_noalloc(int32_t kind, const float* pred, const float* target, int32_t C, int32_t H,
                                       int32_t W, const int32_t* crop, float* dL_dpred, float* loss_out,
                                       gsc_stream_t stream) {
    using namespace gsc;
    if (!pred || !target || !loss_out) return set_error(GSC_ERR_INVALID_ARG, "gsc_loss_noalloc: NULL argument");
    if (kind != GSC_LOSS_HDR && kind != GSC_LOSS_HDR_FULLGRAD)
        return set_error(GSC_ERR_INVALID_ARG, "gsc_loss_noalloc: loss kind %d not available", kind);
    if (C < 1 || H < 1 || W < 1) return set_error(GSC_ERR_INVALID_ARG, "gsc_loss_noalloc: empty image");
    int x0 = 0, y0 = 0, w = W, h = H;
    if (crop) {
        x0 = crop[0]; y0 = crop[1]; w = crop[2]; h = crop[3];
        if (x0 < 0 || y0 < 0 || w < 1 || h < 1 || (int64_t)x0 + w > W || (int64_t)y0 + h > H)
            return set_error(GSC_ERR_INVALID_ARG, "gsc_loss_noalloc: crop outside the image");
    }
    size_t n = (size_t)C * w * h;
    size_t blocks = (n + kRedThreads - 1) / kRedThreads;
    if (blocks > (size_t)kNoAllocSlots)
        return set_error(GSC_ERR_CAPACITY,
                         "gsc_loss_noalloc: %zu elements exceed the fixed scratch (at most %d elements)", n,
                         kNoAllocSlots * kRedThreads);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(GSC_ERR_CUDA, "gsc_loss_noalloc: no current device");
    float* partials = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p)
                return set_error(GSC_ERR_CUDA, "gsc_loss_noalloc: scratch address lookup failed: %s",
                                 cudaGetErrorString(e));
            g_noalloc_ptr[dev] = (float*)p;
        }
        partials = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (dL_dpred && (x0 != 0 || y0 != 0 || w != W || h != H))
        if (cudaMemsetAsync(dL_dpred, 0, sizeof(float) * (size_t)C * H * W, s) != cudaSuccess)
            return set_error(GSC_ERR_CUDA, "gsc_loss_noalloc: clearing dL_dpred failed");
    float invk = (float)(1.0 / (double)n);
    PhaseScope ph(kPhLoss, s, 2);
    k_loss_hdr<<<(unsigned)blocks, kRedThreads, 0, s>>>(pred, target, C, H, W, x0, y0, w, h,
                                                        kind == GSC_LOSS_HDR_FULLGRAD, invk, dL_dpred, partials);
    k_reduce_final<<<1, 1024, 0, s>>>(partials, (int)blocks, 1.0 / (double)n, loss_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(GSC_ERR_CUDA, "gsc_loss_noalloc launch: %s", cudaGetErrorString(e));
    return GSC_OK;
}

namespace gsc {

// ------------------------------------------------------------------ AdamW

// one float4 per thread: record quarter q = i % 4 holds slots 4q .. 4q + 3
__global__ void __launch_bounds__(256) k_adamw(float4* __restrict__ P, float4* __restrict__ G, float4* __restrict__ M,
                                               float4* __restrict__ V, size_t n4, AdamDev a) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        float4 p = P[i], g = G[i], m = M[i], v = V[i];
        adam_four(p, m, v, g, (int)(i & 3), a);
        P[i] = p;
        M[i] = m;
        V[i] = v;
        G[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

AdamDev adam_dev(const gsc_adam_params& ap) {
    AdamDev a;
    for (int k = 0; k < 16; ++k) a.lr[k] = ap.lr[k] * ap.lr_scale;
    a.b1 = ap.beta1;
    a.b2 = ap.beta2;
    a.eps = ap.eps;
    a.wd = ap.weight_decay;
    a.ibc1 = (float)(1.0 / (1.0 - pow((double)ap.beta1, (double)ap.step)));
    a.ibc2 = (float)(1.0 / (1.0 - pow((double)ap.beta2, (double)ap.step)));
    return a;
}

cudaError_t launch_adamw(float* params, float* grads, float* m, float* v, int64_t N, const gsc_adam_params& ap,
                         cudaStream_t s) {
    const AdamDev a = adam_dev(ap);
    size_t n4 = (size_t)N * 4;
    size_t blocks = (n4 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    PhaseScope ph(kPhAdam, s, 1);
    k_adamw<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<float4*>(params), reinterpret_cast<float4*>(grads),
                                             reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), n4, a);
    return cudaGetLastError();
}

}  // namespace gsc
