// Internal declarations of the GB300 GSCache library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsc.h"

namespace gsc {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// --------------------------------------------------------------- sorting
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 8;                              // items per thread
constexpr int kSortTile = kSortThreads * kSortIPT;      // 2048 items per tile
constexpr int kMaxSortBlocks = 152 * 8;                 // GB300: 152 SMs x 8 resident blocks
constexpr int kMaxDigitBits = 9;                        // radix digits of 8 or 9 bits
constexpr int kMaxDigits = 1 << kMaxDigitBits;
constexpr size_t kHistWords = (size_t)kMaxSortBlocks * kMaxDigits + kMaxDigits;  // histogram + digit totals
constexpr int kScanTile = 2048;

// --------------------------------------------------------------- raster
// Projected record of one Gaussian, three float4 (48 B):
//   r0 = (mean2D.x, mean2D.y, qa, qb)   r1 = (qc, opacity, lthr2, 0)   r2 = (r, g, b, 0)
// with p2 = qa dx^2 + qb dx dy + qc dy^2 = log2(exp(-d^T conic d / 2)), i.e.
// qa = -a log2(e) / 2, qb = -b log2(e), qc = -c log2(e) / 2, and
// lthr2 = log2(alpha_min / opacity): a pair is composited iff p2 >= lthr2.
struct CamDev {
    float R[9], t[3], pos[3], fx, fy, cx, cy;
    int W, H;
};

// launch configuration and compositing constants shared by all views of a call
struct RasterDev {
    float alpha_max, alpha_min, T_min, near_plane, dilation;
    int tile_w, tile_h, cap;
    int bin;  // bin size (px) of every view; 0: each view picks its own (auto_bin)
    int ppt;  // pixels per thread (1, 2, 4 or 8)
    int ring_log2;  // hit ring of the gradient kernels: 1 << ring_log2 entries
};

// One view of a (possibly batched) render: its camera, its Gaussians (global
// indices [g_off, g_off + N) of the call), its tiles and bins (global
// numbering from tile_off / bin_off) and its images.
constexpr int kMaxViews = 32;
struct ViewDev {
    CamDev cam;
    const float4* params;
    float* image;
    const float* dL;
    float4* grads;
    const float* target;  // training step: the loss target (3 x H x W)
    float* loss;          // training step: the view's loss (device scalar)
    float invk;           // training step: 1 / (3 H W)
    float4* m;            // fused AdamW step: first and second moments (N x 16 each)
    float4* v;
    uint32_t g_off, N, tile_off, bin_off;
    int tiles_x, tiles_y, bins_x, bins_y;
    int bin, spt_x, spt_y;  // the view's bin size (px) and tiles per bin side
};
struct BatchDev {
    int nviews;
    uint32_t total_g, total_tiles, total_bins;
    ViewDev v[kMaxViews];
};

// view owning global Gaussian g / global tile t (linear scans: <= 32 views)
__device__ __forceinline__ int view_of_gaussian(const BatchDev& b, uint32_t g) {
    int v = 0;
    while (v + 1 < b.nviews && g >= b.v[v + 1].g_off) ++v;
    return v;
}
__device__ __forceinline__ int view_of_tile(const BatchDev& b, uint32_t t) {
    int v = 0;
    while (v + 1 < b.nviews && t >= b.v[v + 1].tile_off) ++v;
    return v;
}

// HDR loss of Sec. 3.6 per element, y = prediction, x = target:
// (x - y)^2 / (y + 0.01)^2, and its derivative in y scaled by 1/k, with the
// denominator held constant (full = 0) or differentiated too (full = 1).
// One definition for the loss kernel and the fused training step, so both
// produce the same gradient bits.
constexpr int kLossNone = 0, kLossHdr = 1, kLossHdrFull = 2;
__device__ __forceinline__ float hdr_term(float y, float x) {
    float den = __fadd_rn(y, 0.01f), d = __fsub_rn(x, y);
    float inv2 = __fdiv_rn(1.f, __fmul_rn(den, den));
    return __fmul_rn(__fmul_rn(d, d), inv2);
}
__device__ __forceinline__ float hdr_grad(float y, float x, bool full, float invk) {
    float den = __fadd_rn(y, 0.01f), d = __fsub_rn(x, y);
    float inv2 = __fdiv_rn(1.f, __fmul_rn(den, den));
    float g = __fmul_rn(__fmul_rn(2.f, __fsub_rn(y, x)), inv2);
    if (full) g = __fsub_rn(g, __fdiv_rn(__fmul_rn(__fmul_rn(__fmul_rn(2.f, d), d), inv2), den));
    return __fmul_rn(g, invk);
}

// sets the calling thread's last error message (api.cu) and returns st
gsc_status set_error(gsc_status st, const char* fmt, ...);

// instrumentation (api.cu): event-timed phases and the launch counter
enum Phase : int {
    kPhProject, kPhDepthSort, kPhScan, kPhEmit, kPhTileSort, kPhRanges, kPhRender, kPhRenderBwd, kPhProjectBwd,
    kPhLoss, kPhAdam, kPhTrace, kPhTrain, kPhInit, kNumPhases
};
void count_launch(int n);
struct PhaseScope {
    PhaseScope(int phase, cudaStream_t s, int launches);
    ~PhaseScope();
    int phase;
    cudaStream_t stream;
    int slot;
};

// status words in the workspace
enum : int { kStatusCode = 0, kStatusWords = 4 };
// counters in the workspace
enum : int { kCntPairs = 0, kCntPairsMax = 1, kCntTilesFwd = 2, kCntTilesBwd = 3, kCounterWords = 8 };
// feedback state: launches so far (its parity picks the buffer the next
// gradient kernel writes), signature of the batch geometry the last
// feedback belongs to (0: none), number of work items of the current order
// and (words 4-5, 64-bit) the summed per-tile cost of the coming order;
// kFbUse: whether the current order came from the feedback (1) or not (0)
enum : int { kFbParity = 0, kFbSignature = 1, kFbItems = 2, kFbUse = 3, kFbTotal = 4, kFbWords = 8 };
// cost classes of the tile order: per class a count and a cursor
constexpr int kOrderClasses = 256;
// A work item of the persistent render kernels: a tile, or part `part` of
// `1 << lp` parts of a tile (the part owns the tile's pixel rows whose slot
// q of the thread has q mod (1 << lp) == part).  A whole tile is its id.
constexpr uint32_t kItemNone = 0xffffffffu;
__host__ __device__ __forceinline__ uint32_t make_item(uint32_t tile, uint32_t part, uint32_t lp) {
    return tile | (part << 24) | (lp << 28);
}
// order of a binning: kOrderPlain (by bin-list length, whole tiles) or
// kOrderFeedback (by the last gradient launch's per-tile work when the
// geometry is the same, splitting the heaviest tiles)
enum : int { kOrderPlain = 0, kOrderFeedback = 1 };
// 64-bit work statistics in the workspace
enum : int { kStEvalFwd = 0, kStCompFwd = 1, kStEvalRewalk = 2, kStEvalBack = 3, kStPairsSum = 4, kStBinnings = 5,
             kStCompRewalk = 6, kStHitBack = 7, kStCulled = 8, kStatWords = 9 };

}  // namespace gsc

// The workspace handle.  Every device pointer points into the caller's buffer.
struct gsc_workspace {
    char* base;
    size_t bytes;
    int64_t max_gaussians, max_pairs, max_tiles;
    int32_t max_w, max_h;
    int sort_blocks;  // grid of the pair sort
    int32_t* status;
    uint32_t* counters;
    unsigned long long* stats;
    float4* rec;       // 3 x NG
    uint32_t *key0, *key1, *idx0, *idx1;
    uint2* rect;       // packed tile rectangle per Gaussian
    uint32_t* cnt;     // tiles touched per Gaussian
    uint32_t* off;     // exclusive prefix of cnt in depth order
    uint32_t* scan_sums;
    uint32_t *pkey0, *pkey1, *pval0, *pval1;
    uint32_t* hist;    // kHistWords
    uint32_t* sweep;   // onesweep_words(max_gaussians): scratch of the depth sort
    uint2* ranges;     // [start, end) per bin
    uint32_t* tile_order;   // work items (tiles or parts of tiles) by expected cost, longest first
    const uint32_t* order;  // the order of the last binning
    // per-tile feedback of the gradient kernels (hits of the front-to-back
    // walk and length of the back-to-front walk) in two buffers that swap
    // every gradient launch, and a scratch of per-tile costs: 5 x max_tiles
    uint32_t* fb;
    uint32_t* fb_state;     // kFbWords: launch parity, geometry of the feedback, item count
    uint32_t* order_cls;    // 2 x kOrderClasses: work items per cost class, then each class's cursor
    float4* g2d;       // 3 x NG: 2D gradients
    float* red;        // reduction scratch for losses
    size_t red_floats;
};

struct gsc_scene {
    gsc_scene_desc desc;
    float sbar;  // majorant
};

namespace gsc {

// sort.cu
void scan_gathered(const uint32_t* cnt, const uint32_t* idx, uint32_t n, uint32_t* out, uint32_t* sums,
                   uint32_t* counters, int32_t* status, uint32_t capacity, unsigned long long* stats, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
// The count is n_host, or *n_dev if n_dev != NULL (clamped to n_host).
// Returns 0 if the sorted data ends in (k0, v0), 1 if in (k1, v1).
int radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* n_dev,
                     uint32_t n_host, int bits, int blocks, uint32_t* hist, cudaStream_t s);
int sort_blocks_for(uint64_t n);
// Stable LSD radix sort of n (key, value) pairs on all 32 key bits, the
// count known on the host: one launch counts the digits of the four 8-bit
// passes, then one launch per pass (decoupled look-back instead of a scan
// pass).  `scratch`: onesweep_words(n) words; a bounded wait that runs out
// sets GSC_ERR_TIMEOUT in status[kStatusCode].  Returns as radix_sort_pairs.
size_t onesweep_words(uint64_t n);
int radix_sort_onesweep(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t n, uint32_t* scratch,
                        int32_t* status, cudaStream_t s);
// digit counts of the last pass of radix_sort_pairs (in its histogram buffer)
inline uint32_t* radix_totals(uint32_t* hist) { return hist + (size_t)kMaxSortBlocks * kMaxDigits; }
int radix_passes(int bits);

struct AdamDev;  // below, with the AdamW arithmetic

// raster.cu (every view of the batch shares rc)
cudaError_t bin_gaussians(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t** sorted_vals,
                          cudaStream_t s, int order_mode = kOrderPlain);
cudaError_t launch_render(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                          cudaStream_t s);
// shared_params: two views write the same parameter gradients (atomics needed)
cudaError_t launch_render_backward(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                                   bool shared_params, cudaStream_t s);
// training step: render, HDR loss (full_grad: the denominator differentiated
// too) and backward in one persistent launch; per-view loss to ViewDev::loss.
// With adam, the per-Gaussian gradient kernel also takes the AdamW step of
// every view's parameters (ViewDev::m, v; parameters not shared).
cudaError_t launch_train(const BatchDev& b, const RasterDev& rc, gsc_workspace* ws, const uint32_t* vals,
                         int full_grad, bool shared_params, const AdamDev* adam, cudaStream_t s);

// trace.cu
cudaError_t launch_trace(const gsc_scene* sc, const CamDev& cam, const gsc_trace_params& p, const float* cache,
                         float* targets, float* image, cudaStream_t s);
// cache initialisation: delta-tracked point samples (pos, albedo; *fails
// counts points without a collision in max_attempts rays)
cudaError_t launch_init_sample(const gsc_scene* sc, uint32_t n, uint64_t seed, int max_attempts, float4* pos,
                               float4* alb, unsigned int* fails, cudaStream_t s);

// init.cu: scratch bytes for N points (layout measured with base = NULL),
// and the whole initialisation (synchronises s; *fails_host as above)
struct InitScratch;
size_t init_layout(int64_t N, char* base, InitScratch* s);
cudaError_t run_init(const gsc_scene* sc, int64_t N, int K, uint64_t seed, int max_attempts, float opacity,
                     char* scratch, float* params, unsigned int* fails_host, cudaStream_t s);

// AdamW (Sec. 3.6; Eq. 4 scales the rates) of one slot with learning rate lr;
// a slot with lr = 0 keeps its value and moments.  One definition for the
// optimiser kernel and the fused training step, so both give the same bits.
struct AdamDev {
    float lr[16];
    float b1, b2, eps, wd;
    float ibc1, ibc2;  // 1 / (1 - beta^t), the bias corrections
};
__device__ __forceinline__ void adam_one(float& p, float& m, float& v, float g, float lr, const AdamDev& a) {
    if (lr == 0.f) return;
    m = a.b1 * m + (1.f - a.b1) * g;
    v = a.b2 * v + (1.f - a.b2) * g * g;
    float mh = m * a.ibc1, vh = v * a.ibc2;
    // correctly rounded square root and quotient with subnormal inputs read
    // as zero: tiny moments then take the fast hardware path (measured 4-9%
    // faster over the step); the effect on p is far below its last bit
    float r, d;
    asm("sqrt.rn.ftz.f32 %0, %1;" : "=f"(r) : "f"(vh));
    asm("div.rn.ftz.f32 %0, %1, %2;" : "=f"(d) : "f"(mh), "f"(r + a.eps));
    p = p - lr * (d + a.wd * p);
}
__device__ __forceinline__ void adam_four(float4& p, float4& m, float4& v, const float4& g, int q, const AdamDev& a) {
    adam_one(p.x, m.x, v.x, g.x, a.lr[4 * q + 0], a);
    adam_one(p.y, m.y, v.y, g.y, a.lr[4 * q + 1], a);
    adam_one(p.z, m.z, v.z, g.z, a.lr[4 * q + 2], a);
    adam_one(p.w, m.w, v.w, g.w, a.lr[4 * q + 3], a);
}
AdamDev adam_dev(const gsc_adam_params& ap);

// optim.cu
cudaError_t launch_loss(int kind, const float* pred, const float* target, int C, int H, int W, int x0, int y0,
                        int w, int h, float* dL_dpred, float* loss_out, float* red, size_t red_floats,
                        cudaStream_t s);
cudaError_t launch_adamw(float* params, float* grads, float* m, float* v, int64_t N, const gsc_adam_params& a,
                         cudaStream_t s);

}  // namespace gsc
