// Cache initialisation (GSCache Sec. 3.2 "Cache Initialization", Eq. 3).
//
// One delta-tracked point cloud of N points (k_init_sample, trace.cu); level
// k takes its first N >> k points.  Per level, the mean distance of every
// point to its three nearest neighbours comes from a uniform grid (cell
// keys, radix sort by cell, cell ranges, a search in growing rings of cells
// that stops once the third distance is within the searched cube), then the
// mean and standard deviation of those distances (FP64, deterministic
// order), and finally one Gaussian per point: mean = the point, colour = its
// albedo, identity rotation, the given opacity, and the isotropic scale
// s = min(mu + 2 sigma, mean 3-NN distance) / 2.
#include <math.h>

#include "gsc_internal.cuh"

namespace gsc {

constexpr int kInitMaxGrid = 160;      // cells per axis (160^3 ranges = 33 MB)
constexpr int kInitRedBlocks = 1024;

__device__ __forceinline__ int cell_of(float x, int G) {
    int c = (int)(x * (float)G);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
}

__global__ void __launch_bounds__(256) k_cell_keys(const float4* __restrict__ pos, uint32_t n, int G,
                                                   uint32_t* __restrict__ key, uint32_t* __restrict__ idx) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = pos[i];
    key[i] = ((uint32_t)cell_of(p.z, G) * (uint32_t)G + (uint32_t)cell_of(p.y, G)) * (uint32_t)G +
             (uint32_t)cell_of(p.x, G);
    idx[i] = i;
}

__global__ void k_cell_ranges(const uint32_t* __restrict__ keys, uint32_t n, uint2* __restrict__ ranges) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) ranges[k].x = i;
        if (i == n - 1 || keys[i + 1] != k) ranges[k].y = i + 1;
    }
}

__device__ __forceinline__ void keep3(float d2, float& b0, float& b1, float& b2) {
    if (d2 < b2) {
        if (d2 < b1) {
            b2 = b1;
            if (d2 < b0) {
                b1 = b0;
                b0 = d2;
            } else {
                b1 = d2;
            }
        } else {
            b2 = d2;
        }
    }
}

// mean distance of point i to its three nearest other points of [0, n)
__global__ void __launch_bounds__(128) k_knn3(const float4* __restrict__ pos, const uint32_t* __restrict__ sidx,
                                              const uint2* __restrict__ ranges, uint32_t n, int G,
                                              float* __restrict__ mbar) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = pos[i];
    const int cx = cell_of(p.x, G), cy = cell_of(p.y, G), cz = cell_of(p.z, G);
    const float h = 1.0f / (float)G;
    float b0 = INFINITY, b1 = INFINITY, b2 = INFINITY;
    for (int r = 0; r <= G; ++r) {
        for (int dz = -r; dz <= r; ++dz) {
            int z = cz + dz;
            if (z < 0 || z >= G) continue;
            for (int dy = -r; dy <= r; ++dy) {
                int y = cy + dy;
                if (y < 0 || y >= G) continue;
                bool face = dz == -r || dz == r || dy == -r || dy == r;
                // cells of ring r only: on a z or y face every x, else the two x ends
                for (int dx = -r; dx <= r; dx += (face || r == 0) ? 1 : 2 * r) {
                    int x = cx + dx;
                    if (x < 0 || x >= G) continue;
                    uint2 rg = ranges[((uint32_t)z * (uint32_t)G + (uint32_t)y) * (uint32_t)G + (uint32_t)x];
                    for (uint32_t e = rg.x; e < rg.y; ++e) {
                        uint32_t j = sidx[e];
                        if (j == i) continue;
                        float4 q = pos[j];
                        float ex = q.x - p.x, ey = q.y - p.y, ez = q.z - p.z;
                        keep3(ex * ex + ey * ey + ez * ez, b0, b1, b2);
                    }
                }
            }
        }
        // every point outside the searched cube is farther than r h
        float reach = (float)r * h;
        if (b2 <= reach * reach) break;
    }
    int m = 0;
    float acc = 0.0f;
    if (b0 < INFINITY) { acc += sqrtf(b0); ++m; }
    if (b1 < INFINITY) { acc += sqrtf(b1); ++m; }
    if (b2 < INFINITY) { acc += sqrtf(b2); ++m; }
    mbar[i] = m ? acc / (float)m : 0.0f;
}

// per-CTA partial sums of mbar (mode 0) or of (mbar - mu)^2 (mode 1), FP64
__global__ void __launch_bounds__(256) k_init_moment(const float* __restrict__ mbar, uint32_t n,
                                                     const double* __restrict__ stats, int mode,
                                                     double* __restrict__ partial) {
    __shared__ double sm[8];
    double mu = mode ? stats[0] : 0.0;
    double acc = 0.0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = (double)mbar[i];
        acc += mode ? (v - mu) * (v - mu) : v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sm[w];
        partial[blockIdx.x] = t;
    }
}

// one thread: stats[0] = mu (mode 0) or stats[1] = sigma (mode 1)
__global__ void k_init_moment_final(const double* __restrict__ partial, int nb, uint32_t n, int mode,
                                    double* __restrict__ stats) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += partial[b];
    if (mode == 0) stats[0] = t / (double)n;
    else stats[1] = sqrt(t / (double)n);
}

__global__ void __launch_bounds__(256) k_init_params(const float4* __restrict__ pos, const float4* __restrict__ alb,
                                                     const float* __restrict__ mbar, uint32_t n,
                                                     const double* __restrict__ stats, float logit,
                                                     float4* __restrict__ out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float cap = (float)(stats[0] + 2.0 * stats[1]);
    float m = mbar[i];
    float ls = logf(0.5f * (m < cap ? m : cap));
    float4 p = pos[i], a = alb[i];
    out[4 * (size_t)i] = make_float4(p.x, p.y, p.z, logit);
    out[4 * (size_t)i + 1] = make_float4(ls, ls, ls, 0.0f);
    out[4 * (size_t)i + 2] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    out[4 * (size_t)i + 3] = make_float4(a.x, a.y, a.z, 0.0f);
}

int init_grid_for(uint32_t n) {
    int g = (int)ceil(cbrt((double)n / 2.0));
    return g < 1 ? 1 : (g > kInitMaxGrid ? kInitMaxGrid : g);
}

// scratch layout (256-B aligned pieces)
struct InitScratch {
    float4 *pos, *alb;
    uint32_t *key0, *key1, *idx0, *idx1, *hist;
    uint2* ranges;
    float* mbar;
    double *partial, *stats;
    unsigned int* fails;
};

size_t init_layout(int64_t N, char* base, InitScratch* s) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    InitScratch t;
    t.pos = (float4*)take(sizeof(float4) * N);
    t.alb = (float4*)take(sizeof(float4) * N);
    t.key0 = (uint32_t*)take(4 * N);
    t.key1 = (uint32_t*)take(4 * N);
    t.idx0 = (uint32_t*)take(4 * N);
    t.idx1 = (uint32_t*)take(4 * N);
    t.hist = (uint32_t*)take(4 * kHistWords);
    t.ranges = (uint2*)take(sizeof(uint2) * (size_t)kInitMaxGrid * kInitMaxGrid * kInitMaxGrid);
    t.mbar = (float*)take(4 * N);
    t.partial = (double*)take(sizeof(double) * kInitRedBlocks);
    t.stats = (double*)take(sizeof(double) * 2);
    t.fails = (unsigned int*)take(sizeof(unsigned int));
    if (s) *s = t;
    return off;
}

cudaError_t run_init(const gsc_scene* sc, int64_t N, int K, uint64_t seed, int max_attempts, float opacity,
                     char* scratch, float* params, unsigned int* fails_host, cudaStream_t s) {
    InitScratch w;
    init_layout(N, scratch, &w);
    cudaError_t e = cudaMemsetAsync(w.fails, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    e = launch_init_sample(sc, (uint32_t)N, seed, max_attempts, w.pos, w.alb, w.fails, s);
    if (e != cudaSuccess) return e;
    const float logit = logf(opacity / (1.0f - opacity));
    size_t row = 0;
    for (int k = 0; k < K; ++k) {
        uint32_t n = (uint32_t)(N >> k);
        int G = init_grid_for(n);
        uint32_t nb = (n + 255) / 256;
        {
            PhaseScope ph(kPhInit, s, 8);
            k_cell_keys<<<nb, 256, 0, s>>>(w.pos, n, G, w.key0, w.idx0);
            int bits = 1;
            while (bits < 32 && (1ull << bits) < (uint64_t)G * G * G) ++bits;
            int cur = radix_sort_pairs(w.key0, w.idx0, w.key1, w.idx1, nullptr, n, bits, sort_blocks_for(n), w.hist,
                                       s);
            const uint32_t* keys = cur ? w.key1 : w.key0;
            const uint32_t* sidx = cur ? w.idx1 : w.idx0;
            cudaMemsetAsync(w.ranges, 0, sizeof(uint2) * (size_t)G * G * G, s);
            k_cell_ranges<<<152 * 4, 256, 0, s>>>(keys, n, w.ranges);
            k_knn3<<<(n + 127) / 128, 128, 0, s>>>(w.pos, sidx, w.ranges, n, G, w.mbar);
            int rb = (int)(nb < (uint32_t)kInitRedBlocks ? nb : (uint32_t)kInitRedBlocks);
            k_init_moment<<<rb, 256, 0, s>>>(w.mbar, n, w.stats, 0, w.partial);
            k_init_moment_final<<<1, 1, 0, s>>>(w.partial, rb, n, 0, w.stats);
            k_init_moment<<<rb, 256, 0, s>>>(w.mbar, n, w.stats, 1, w.partial);
            k_init_moment_final<<<1, 1, 0, s>>>(w.partial, rb, n, 1, w.stats);
            k_init_params<<<nb, 256, 0, s>>>(w.pos, w.alb, w.mbar, n, w.stats, logit,
                                             reinterpret_cast<float4*>(params) + 4 * row);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        row += n;
    }
    e = cudaMemcpyAsync(fails_host, w.fails, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace gsc
