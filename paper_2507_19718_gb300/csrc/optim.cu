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
        float den = y + 0.01f, d = x - y;
        float inv2 = 1.f / (den * den);
        acc += d * d * inv2;
        if (dL) {
            float g = 2.f * (y - x) * inv2;
            if (full) g -= 2.f * d * d * inv2 / den;
            dL[p] = g * invk;
        }
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

cudaError_t launch_loss(int kind, const float* pred, const float* target, int C, int H, int W, int x0, int y0,
                        int w, int h, float* dL_dpred, float* loss_out, float* red, size_t red_floats,
                        cudaStream_t s) {
    size_t n = (size_t)C * w * h;
    if (dL_dpred && (x0 != 0 || y0 != 0 || w != W || h != H))
        cudaMemsetAsync(dL_dpred, 0, sizeof(float) * (size_t)C * H * W, s);
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
        if (x0 < 0 || y0 < 0 || w < 1 || h < 1 || x0 + w > W || y0 + h > H)
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

struct AdamDev {
    float lr[16];
    float b1, b2, eps, wd, bc1, bc2;
};

__device__ __forceinline__ void adam_one(float& p, float& m, float& v, float g, float lr, const AdamDev& a) {
    if (lr == 0.f) return;
    m = a.b1 * m + (1.f - a.b1) * g;
    v = a.b2 * v + (1.f - a.b2) * g * g;
    float mh = m / a.bc1, vh = v / a.bc2;
    p = p - lr * (mh / (sqrtf(vh) + a.eps) + a.wd * p);
}

// one float4 per thread: record quarter q = i % 4 holds slots 4q .. 4q + 3
__global__ void __launch_bounds__(256) k_adamw(float4* __restrict__ P, float4* __restrict__ G, float4* __restrict__ M,
                                               float4* __restrict__ V, size_t n4, AdamDev a) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        int q = (int)(i & 3);
        float4 p = P[i], g = G[i], m = M[i], v = V[i];
        adam_one(p.x, m.x, v.x, g.x, a.lr[4 * q + 0], a);
        adam_one(p.y, m.y, v.y, g.y, a.lr[4 * q + 1], a);
        adam_one(p.z, m.z, v.z, g.z, a.lr[4 * q + 2], a);
        adam_one(p.w, m.w, v.w, g.w, a.lr[4 * q + 3], a);
        P[i] = p;
        M[i] = m;
        V[i] = v;
        G[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

cudaError_t launch_adamw(float* params, float* grads, float* m, float* v, int64_t N, const gsc_adam_params& ap,
                         cudaStream_t s) {
    AdamDev a;
    for (int k = 0; k < 16; ++k) a.lr[k] = ap.lr[k] * ap.lr_scale;
    a.b1 = ap.beta1;
    a.b2 = ap.beta2;
    a.eps = ap.eps;
    a.wd = ap.weight_decay;
    a.bc1 = (float)(1.0 - pow((double)ap.beta1, (double)ap.step));
    a.bc2 = (float)(1.0 - pow((double)ap.beta2, (double)ap.step));
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
