// C ABI of the GB300 GSCache library (declared in include/gsc.h).  Host-side
// validation, workspace layout over the caller's device buffer, and the
// mapping of each call onto the kernels.  Nothing here allocates device
// memory or synchronises, except gsc_workspace_status.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "gsc_internal.cuh"

using namespace gsc;

// ------------------------------------------------------------------ instrumentation
namespace gsc {

static std::atomic<int64_t> g_launches{0};

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
const char* kPhaseNames[kNumPhases] = {"project", "depth_sort", "scan", "emit", "tile_sort", "ranges",
                                       "render", "render_bwd", "project_bwd", "loss", "adamw", "trace", "train",
                                       "init"};
struct Pending {
    int phase, launches;
    cudaEvent_t a, b;
};
struct ProfState {
    std::mutex mu;
    std::atomic<bool> on{false};
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[kNumPhases] = {};
    int64_t launches[kNumPhases] = {}, calls[kNumPhases] = {};
};
ProfState& prof() {
    static ProfState p;
    return p;
}
cudaEvent_t take_event(ProfState& p) {
    if (!p.pool.empty()) {
        cudaEvent_t e = p.pool.back();
        p.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

PhaseScope::PhaseScope(int ph, cudaStream_t s, int launches) : phase(ph), stream(s), slot(-1) {
    count_launch(launches);
    ProfState& p = prof();
    if (!p.on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> g(p.mu);
    cudaEvent_t a = take_event(p), b = take_event(p);
    if (!a || !b) return;
    cudaEventRecord(a, s);
    p.pending.push_back({ph, launches, a, b});
    slot = (int)p.pending.size() - 1;
}

PhaseScope::~PhaseScope() {
    if (slot < 0) return;
    ProfState& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    if (slot < (int)p.pending.size()) cudaEventRecord(p.pending[slot].b, stream);
}

}  // namespace gsc

namespace {

thread_local char g_err[512] = "";

gsc_status fail(gsc_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

}  // namespace

gsc_status gsc::set_error(gsc_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

namespace {

gsc_status cuda_fail(cudaError_t e, const char* where) {
    return fail(GSC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define GSC_CUDA(call)                                         \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// (tile_w, tile_h, pixels per thread) combinations the rasterizer is compiled for
bool valid_tile(int w, int h, int ppt) {
    static const int ok[][3] = {{16, 16, 1}, {8, 8, 1},  {32, 8, 1}, {16, 8, 1}, {8, 16, 1}, {8, 32, 1},
                                {32, 4, 1},  {16, 16, 2}, {32, 8, 2}, {16, 8, 2}, {8, 16, 2}, {8, 32, 2},
                                {16, 16, 4}, {32, 8, 4},  {8, 32, 4}, {16, 16, 8}, {32, 8, 8}, {8, 32, 8}};
    for (auto& t : ok)
        if (t[0] == w && t[1] == h && t[2] == ppt) return true;
    return false;
}

gsc_status check_cfg(const gsc_raster_cfg* c) {
    if (!c) return fail(GSC_ERR_INVALID_ARG, "raster cfg is NULL");
    int ppt = c->pixels_per_thread ? c->pixels_per_thread : 1;
    if (!valid_tile(c->tile_w, c->tile_h, ppt))
        return fail(GSC_ERR_INVALID_ARG, "unsupported tile %dx%d with %d pixels per thread", c->tile_w, c->tile_h,
                    c->pixels_per_thread);
    if (c->list_capacity < 32 || c->list_capacity > 2048 || c->list_capacity % 32)
        return fail(GSC_ERR_INVALID_ARG, "list_capacity %d not a multiple of 32 in [32, 2048]", c->list_capacity);
    if (c->bin_size != 0 && (c->bin_size < 32 || c->bin_size > 512 || c->bin_size % c->tile_w ||
                             c->bin_size % c->tile_h))
        return fail(GSC_ERR_INVALID_ARG, "bin_size %d must be 0 or a multiple of the tile in [32, 512]",
                    c->bin_size);
    if (!(c->alpha_max > 0.f && c->alpha_max < 1.f) || !(c->alpha_min > 0.f && c->alpha_min < c->alpha_max) ||
        !(c->T_min > 0.f && c->T_min < 1.f) || !(c->near_plane > 0.f) || !(c->dilation >= 0.f))
        return fail(GSC_ERR_INVALID_ARG, "compositing constants out of range");
    return GSC_OK;
}

gsc_status check_cam(const gsc_camera* c) {
    if (!c) return fail(GSC_ERR_INVALID_ARG, "camera is NULL");
    if (c->width < 1 || c->height < 1 || c->width > 65535 || c->height > 65535)
        return fail(GSC_ERR_INVALID_ARG, "camera size %dx%d", c->width, c->height);
    if (!(c->fx > 0.f) || !(c->fy > 0.f)) return fail(GSC_ERR_INVALID_ARG, "camera focal lengths must be > 0");
    return GSC_OK;
}

CamDev cam_dev(const gsc_camera* c) {
    CamDev d;
    memcpy(d.R, c->R, sizeof d.R);
    memcpy(d.t, c->t, sizeof d.t);
    memcpy(d.pos, c->pos, sizeof d.pos);
    d.fx = c->fx; d.fy = c->fy; d.cx = c->cx; d.cy = c->cy;
    d.W = c->width; d.H = c->height;
    return d;
}

RasterDev raster_dev(const gsc_raster_cfg* c) {
    RasterDev r;
    r.alpha_max = c->alpha_max; r.alpha_min = c->alpha_min; r.T_min = c->T_min;
    r.near_plane = c->near_plane; r.dilation = c->dilation;
    r.tile_w = c->tile_w; r.tile_h = c->tile_h;
    r.ppt = c->pixels_per_thread ? c->pixels_per_thread : 1;
    int nt = c->tile_w * c->tile_h / r.ppt;
    r.cap = c->list_capacity < nt ? nt : c->list_capacity;
    r.bin = c->bin_size;
    // the gradient kernels' hit ring: 2048 entries beside a small staging
    // (the shared memory of 12 CTAs per SM still fits), so that the long
    // lists of sparse tiles are walked back to front without rebuilding
    // chunks; 1024 beside a large one
    r.ring_log2 = r.cap <= 128 ? 11 : 10;
    return r;
}

// Bin size of a view when the configuration leaves it open: the largest of
// 256, 128, 64 and 32 px at most a twelfth of the longer image side (32 at
// least), so that a tile's bin list stays a small part of the image
// whatever its resolution (1080p: 128, the size tuned for it; 720p: 64;
// 640x480 and below: 32).  Every candidate is a multiple of every tile side.
static int auto_bin(int w, int h) {
    const int side = w > h ? w : h;
    int bin = 256;
    while (bin > 32 && bin * 12 > side) bin /= 2;
    return bin;
}

// Append one view to a batch table (tiles and bins numbered after the
// previous views').
void add_view(BatchDev& b, const RasterDev& rc, const gsc_camera* cam, const float* params, int64_t N,
              float* image, const float* dL, float* grads) {
    ViewDev& v = b.v[b.nviews];
    v.cam = cam_dev(cam);
    v.params = reinterpret_cast<const float4*>(params);
    v.image = image;
    v.dL = dL;
    v.grads = reinterpret_cast<float4*>(grads);
    v.target = nullptr;
    v.loss = nullptr;
    v.invk = 1.f / (3.f * (float)cam->width * (float)cam->height);
    v.g_off = b.total_g;
    v.N = (uint32_t)N;
    v.tiles_x = (cam->width + rc.tile_w - 1) / rc.tile_w;
    v.tiles_y = (cam->height + rc.tile_h - 1) / rc.tile_h;
    v.bin = rc.bin ? rc.bin : auto_bin(cam->width, cam->height);
    v.spt_x = v.bin / rc.tile_w;
    v.spt_y = v.bin / rc.tile_h;
    v.bins_x = (cam->width + v.bin - 1) / v.bin;
    v.bins_y = (cam->height + v.bin - 1) / v.bin;
    v.tile_off = b.total_tiles;
    v.bin_off = b.total_bins;
    b.total_g += (uint32_t)N;
    b.total_tiles += (uint32_t)(v.tiles_x * v.tiles_y);
    b.total_bins += (uint32_t)(v.bins_x * v.bins_y);
    b.nviews += 1;
}

void batch_init(BatchDev& b) {
    b.nviews = 0;
    b.total_g = b.total_tiles = b.total_bins = 0;
}

int64_t max_tiles_for(int32_t w, int32_t h) {
    static const int ok[][2] = {{16, 16}, {8, 8}, {32, 8}, {16, 8}, {8, 16}, {8, 32}, {32, 4}};
    int64_t m = 1;
    for (auto& t : ok) {
        int64_t n = (int64_t)((w + t[0] - 1) / t[0]) * ((h + t[1] - 1) / t[1]);
        if (n > m) m = n;
    }
    return m;
}

// Carve the workspace out of `base` (NULL: only measure).  Returns bytes used.
size_t layout(int64_t NG, int64_t NP, int32_t W, int32_t H, int32_t NV, gsc_workspace* ws, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~(size_t)255;
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    int64_t tiles = max_tiles_for(W, H) * (NV > 0 ? NV : 1);  // bins of all views
    size_t ng = (size_t)(NG > 0 ? NG : 1), np = (size_t)(NP > 0 ? NP : 1);
    // reduction partials, then three SSIM derivative maps of a full 3-channel image
    size_t red = 65536 + 9 * (size_t)W * (size_t)H;
    gsc_workspace tmp;
    gsc_workspace* w = ws ? ws : &tmp;
    w->status = (int32_t*)take(sizeof(int32_t) * kStatusWords);
    w->counters = (uint32_t*)take(sizeof(uint32_t) * kCounterWords);
    w->stats = (unsigned long long*)take(sizeof(unsigned long long) * kStatWords);
    w->rec = (float4*)take(sizeof(float4) * 3 * ng);
    w->key0 = (uint32_t*)take(4 * ng);
    w->key1 = (uint32_t*)take(4 * ng);
    w->idx0 = (uint32_t*)take(4 * ng);
    w->idx1 = (uint32_t*)take(4 * ng);
    w->rect = (uint2*)take(sizeof(uint2) * ng);
    w->cnt = (uint32_t*)take(4 * ng);
    w->off = (uint32_t*)take(4 * ng);
    w->scan_sums = (uint32_t*)take(4 * (ng / kScanTile + 2));
    w->pkey0 = (uint32_t*)take(4 * np);
    w->pkey1 = (uint32_t*)take(4 * np);
    w->pval0 = (uint32_t*)take(4 * np);
    w->pval1 = (uint32_t*)take(4 * np);
    w->hist = (uint32_t*)take(4 * kHistWords);
    w->sweep = (uint32_t*)take(4 * onesweep_words(ng));
    w->ranges = (uint2*)take(sizeof(uint2) * (size_t)tiles);
    w->tile_order = (uint32_t*)take(4 * 4 * (size_t)tiles);  // up to 4 parts per tile
    w->fb = (uint32_t*)take(4 * 5 * (size_t)tiles);
    w->fb_state = (uint32_t*)take(4 * kFbWords);
    w->order_cls = (uint32_t*)take(4 * 2 * kOrderClasses);
    w->g2d = (float4*)take(sizeof(float4) * 3 * ng);
    w->red = (float*)take(sizeof(float) * red);
    w->red_floats = red;
    w->max_gaussians = NG;
    w->max_pairs = NP;
    w->max_tiles = tiles;
    w->max_w = W;
    w->max_h = H;
    w->sort_blocks = sort_blocks_for((uint64_t)np);
    return (off + 255) & ~(size_t)255;
}

gsc_status check_ws(const gsc_workspace* ws, int64_t N, const gsc_camera* cam) {
    if (!ws) return fail(GSC_ERR_INVALID_ARG, "workspace is NULL");
    if (N < 0 || N > ws->max_gaussians)
        return fail(GSC_ERR_INVALID_ARG, "N = %lld outside [0, %lld]", (long long)N, (long long)ws->max_gaussians);
    if (cam && (cam->width > ws->max_w || cam->height > ws->max_h))
        return fail(GSC_ERR_INVALID_ARG, "image %dx%d larger than the workspace's %dx%d", cam->width, cam->height,
                    ws->max_w, ws->max_h);
    return GSC_OK;
}

}  // namespace

extern "C" {

int32_t gsc_abi_version(void) { return GSC_ABI_VERSION; }

gsc_status gsc_last_error(char* buf, size_t n) {
    if (buf && n) {
        strncpy(buf, g_err, n - 1);
        buf[n - 1] = 0;
    }
    return GSC_OK;
}

// ------------------------------------------------------------------ scenes

static gsc_status check_tf(int32_t n, const float* pos, const float* rgba) {
    if (n < 1 || n > 16) return fail(GSC_ERR_INVALID_ARG, "tf_count %d outside [1, 16]", n);
    for (int k = 0; k < n; ++k) {
        if (!(pos[k] >= 0.f && pos[k] <= 1.f)) return fail(GSC_ERR_INVALID_ARG, "tf_pos[%d] outside [0, 1]", k);
        if (k && !(pos[k] > pos[k - 1])) return fail(GSC_ERR_INVALID_ARG, "tf_pos not strictly ascending");
        for (int c = 0; c < 4; ++c)
            if (!(rgba[4 * k + c] >= 0.f) || !isfinite(rgba[4 * k + c]))
                return fail(GSC_ERR_INVALID_ARG, "tf_rgba[%d] negative or not finite", k);
    }
    return GSC_OK;
}

static float majorant(const gsc_scene_desc& d) {
    float amax = 0.f;
    for (int k = 0; k < d.tf_count; ++k)
        if (d.tf_rgba[k][3] > amax) amax = d.tf_rgba[k][3];
    float sbar = d.sigma_max * amax;  // FP32 product
    return sbar;
}

gsc_status gsc_scene_create(const gsc_scene_desc* desc, gsc_scene** out) {
    if (!desc || !out) return fail(GSC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (desc->nx < 2 || desc->ny < 2 || desc->nz < 2) return fail(GSC_ERR_INVALID_ARG, "grid dims must be >= 2");
    if (!desc->density || !aligned(desc->density, 4)) return fail(GSC_ERR_INVALID_ARG, "density pointer");
    if (!(desc->density_max > 0.f) || !(desc->sigma_max >= 0.f) || !(desc->albedo >= 0.f) ||
        !isfinite(desc->sigma_max))
        return fail(GSC_ERR_INVALID_ARG, "density_max must be > 0, sigma_max and albedo >= 0");
    gsc_status st = check_tf(desc->tf_count, desc->tf_pos, &desc->tf_rgba[0][0]);
    if (st) return st;
    if (desc->n_spheres < 0 || desc->n_spheres > GSC_MAX_SPHERE_LIGHTS)
        return fail(GSC_ERR_INVALID_ARG, "n_spheres must be in [0, %d]", GSC_MAX_SPHERE_LIGHTS);
    for (int l = 0; l < desc->n_spheres; ++l) {
        const float* c = desc->sphere_center[l];
        float r = desc->sphere_radius[l];
        double d2 = 0.0;  // squared distance from the centre to the unit box
        for (int a = 0; a < 3; ++a) {
            double e = c[a] < 0.f ? -(double)c[a] : (c[a] > 1.f ? (double)c[a] - 1.0 : 0.0);
            d2 += e * e;
        }
        if (!(r > 0.f) || !(d2 > (double)r * r) || !isfinite(c[0] + c[1] + c[2]))
            return fail(GSC_ERR_INVALID_ARG, "sphere light %d must have radius > 0 and lie outside the unit box", l);
        for (int ch = 0; ch < 3; ++ch)
            if (!(desc->sphere_radiance[l][ch] >= 0.f))
                return fail(GSC_ERR_INVALID_ARG, "sphere light %d radiance must be >= 0", l);
    }
    gsc_scene* sc = new (std::nothrow) gsc_scene;
    if (!sc) return fail(GSC_ERR_OOM, "host allocation");
    sc->desc = *desc;
    sc->sbar = majorant(sc->desc);
    *out = sc;
    return GSC_OK;
}

gsc_status gsc_scene_set_tf(gsc_scene* scene, int32_t n, const float* pos, const float* rgba) {
    if (!scene || !pos || !rgba) return fail(GSC_ERR_INVALID_ARG, "NULL argument");
    gsc_status st = check_tf(n, pos, rgba);
    if (st) return st;
    scene->desc.tf_count = n;
    for (int k = 0; k < n; ++k) {
        scene->desc.tf_pos[k] = pos[k];
        for (int c = 0; c < 4; ++c) scene->desc.tf_rgba[k][c] = rgba[4 * k + c];
    }
    scene->sbar = majorant(scene->desc);
    return GSC_OK;
}

gsc_status gsc_scene_destroy(gsc_scene* scene) {
    delete scene;
    return GSC_OK;
}

gsc_status gsc_trace(const gsc_scene* scene, const gsc_camera* cam, const gsc_trace_params* p,
                     const float* cache_imgs, float* targets, float* image, gsc_stream_t stream) {
    if (!scene || !p || !image) return fail(GSC_ERR_INVALID_ARG, "NULL argument");
    gsc_status st = check_cam(cam);
    if (st) return st;
    if (p->spp < 1 || p->max_bounces < 1 || p->levels < 0 || p->levels > 16)
        return fail(GSC_ERR_INVALID_ARG, "spp >= 1, max_bounces >= 1, levels in [0, 16] required");
    if (p->levels > 0 && !targets) return fail(GSC_ERR_INVALID_ARG, "targets NULL with levels > 0");
    if (p->C > 0.f && !cache_imgs) return fail(GSC_ERR_INVALID_ARG, "C > 0 needs cache images");
    if (!(p->eps >= 0.f)) return fail(GSC_ERR_INVALID_ARG, "eps must be >= 0");
    if ((p->tr_out != GSC_TR_OUT_CUMULATIVE && p->tr_out != GSC_TR_OUT_PER_CALL) || p->pad != 0)
        return fail(GSC_ERR_INVALID_ARG, "tr_out must be GSC_TR_OUT_CUMULATIVE or GSC_TR_OUT_PER_CALL, pad 0");
    if (cache_imgs && p->levels == 0) return fail(GSC_ERR_INVALID_ARG, "cache images with levels = 0");
    cudaError_t e = launch_trace(scene, cam_dev(cam), *p, cache_imgs, targets, image, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "gsc_trace launch");
    return GSC_OK;
}

// ------------------------------------------------------------------ workspaces

gsc_status gsc_workspace_size(int64_t max_gaussians, int64_t max_pairs, int32_t max_w, int32_t max_h,
                              int32_t max_views, const gsc_raster_cfg* cfg, size_t* bytes) {
    (void)cfg;
    if (!bytes) return fail(GSC_ERR_INVALID_ARG, "bytes is NULL");
    if (max_gaussians < 0 || max_gaussians > (1ll << 31) - 1 || max_pairs < 0 || max_pairs > (1ll << 31) - 1 ||
        max_w < 1 || max_h < 1 || max_w > 65535 || max_h > 65535 || max_views < 1 || max_views > kMaxViews)
        return fail(GSC_ERR_INVALID_ARG, "workspace limits out of range");
    *bytes = layout(max_gaussians, max_pairs, max_w, max_h, max_views, nullptr, nullptr);
    return GSC_OK;
}

gsc_status gsc_workspace_create(void* device_buffer, size_t bytes, int64_t max_gaussians, int64_t max_pairs,
                                int32_t max_w, int32_t max_h, int32_t max_views, const gsc_raster_cfg* cfg,
                                gsc_workspace** out) {
    if (!out) return fail(GSC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    size_t need;
    gsc_status st = gsc_workspace_size(max_gaussians, max_pairs, max_w, max_h, max_views, cfg, &need);
    if (st) return st;
    if (!device_buffer || !aligned(device_buffer, 256)) return fail(GSC_ERR_INVALID_ARG, "buffer not 256-B aligned");
    if (bytes < need) return fail(GSC_ERR_OOM, "workspace buffer has %zu bytes, needs %zu", bytes, need);
    gsc_workspace* ws = new (std::nothrow) gsc_workspace;
    if (!ws) return fail(GSC_ERR_OOM, "host allocation");
    ws->base = (char*)device_buffer;
    ws->bytes = bytes;
    layout(max_gaussians, max_pairs, max_w, max_h, max_views, ws, (char*)device_buffer);
    cudaError_t e = cudaMemset(ws->status, 0, sizeof(int32_t) * kStatusWords);
    if (e == cudaSuccess) e = cudaMemset(ws->counters, 0, sizeof(uint32_t) * kCounterWords);
    if (e == cudaSuccess) e = cudaMemset(ws->stats, 0, sizeof(unsigned long long) * kStatWords);
    if (e == cudaSuccess) e = cudaMemset(ws->fb_state, 0, sizeof(uint32_t) * kFbWords);
    if (e == cudaSuccess) e = cudaMemset(ws->order_cls, 0, sizeof(uint32_t) * 2 * kOrderClasses);
    if (e != cudaSuccess) {
        delete ws;
        return cuda_fail(e, "workspace init");
    }
    *out = ws;
    return GSC_OK;
}

gsc_status gsc_workspace_destroy(gsc_workspace* ws) {
    delete ws;
    return GSC_OK;
}

gsc_status gsc_workspace_status(gsc_workspace* ws, gsc_stream_t stream, int64_t* pairs_needed) {
    if (!ws) return fail(GSC_ERR_INVALID_ARG, "workspace is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    GSC_CUDA(cudaStreamSynchronize(s));
    int32_t status[kStatusWords];
    uint32_t counters[kCounterWords];
    GSC_CUDA(cudaMemcpy(status, ws->status, sizeof status, cudaMemcpyDeviceToHost));
    GSC_CUDA(cudaMemcpy(counters, ws->counters, sizeof counters, cudaMemcpyDeviceToHost));
    GSC_CUDA(cudaMemset(ws->status, 0, sizeof status));
    GSC_CUDA(cudaMemset(ws->counters + kCntPairsMax, 0, sizeof(uint32_t)));
    if (pairs_needed) *pairs_needed = counters[kCntPairsMax];
    if (status[kStatusCode] == GSC_ERR_CAPACITY)
        return fail(GSC_ERR_CAPACITY, "a render needed %u (Gaussian, tile) pairs; the workspace holds %lld",
                    counters[kCntPairsMax], (long long)ws->max_pairs);
    if (status[kStatusCode] != 0) return fail((gsc_status)status[kStatusCode], "device status %d", status[kStatusCode]);
    return GSC_OK;
}

gsc_status gsc_workspace_counters(gsc_workspace* ws, gsc_stream_t stream, int64_t* out, int32_t n) {
    if (!ws || !out || n < 0 || n > GSC_COUNTER_WORDS) return fail(GSC_ERR_INVALID_ARG, "bad arguments");
    GSC_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t counters[kCounterWords];
    unsigned long long st[kStatWords];
    GSC_CUDA(cudaMemcpy(counters, ws->counters, sizeof counters, cudaMemcpyDeviceToHost));
    GSC_CUDA(cudaMemcpy(st, ws->stats, sizeof st, cudaMemcpyDeviceToHost));
    GSC_CUDA(cudaMemset(ws->stats, 0, sizeof st));
    uint32_t fb[kFbWords];
    GSC_CUDA(cudaMemcpy(fb, ws->fb_state, sizeof fb, cudaMemcpyDeviceToHost));
    int64_t all[GSC_COUNTER_WORDS] = {counters[kCntPairs], counters[kCntPairsMax], (int64_t)st[kStEvalFwd],
                                      (int64_t)st[kStCompFwd], (int64_t)st[kStEvalRewalk], (int64_t)st[kStEvalBack],
                                      (int64_t)st[kStPairsSum], (int64_t)st[kStBinnings],
                                      (int64_t)st[kStCompRewalk], (int64_t)st[kStHitBack], (int64_t)fb[kFbItems],
                                      (int64_t)st[kStCulled]};
    for (int k = 0; k < n; ++k) out[k] = all[k];
    return GSC_OK;
}

// ------------------------------------------------------------------ raster

static gsc_status raster_common(const float* params, int64_t N, const gsc_camera* cam, const gsc_raster_cfg* cfg,
                                const gsc_workspace* ws) {
    gsc_status st = check_cam(cam);
    if (st) return st;
    if ((st = check_cfg(cfg))) return st;
    if ((st = check_ws(ws, N, cam))) return st;
    if (N > 0 && (!params || !aligned(params, 16))) return fail(GSC_ERR_INVALID_ARG, "params NULL or not 16-B aligned");
    return GSC_OK;
}

gsc_status gsc_cache_render(const float* params, int64_t N, const gsc_camera* cam, const gsc_raster_cfg* cfg,
                            gsc_workspace* ws, float* image, gsc_stream_t stream) {
    gsc_status st = raster_common(params, N, cam, cfg, ws);
    if (st) return st;
    if (!image) return fail(GSC_ERR_INVALID_ARG, "image is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) {
        GSC_CUDA(cudaMemsetAsync(image, 0, sizeof(float) * 3 * (size_t)cam->width * cam->height, s));
        return GSC_OK;
    }
    RasterDev rc = raster_dev(cfg);
    BatchDev b;
    batch_init(b);
    add_view(b, rc, cam, params, N, image, nullptr, nullptr);
    const uint32_t* vals = nullptr;
    cudaError_t e = bin_gaussians(b, rc, ws, &vals, s);
    if (e == cudaSuccess) e = launch_render(b, rc, ws, vals, s);
    if (e != cudaSuccess) return cuda_fail(e, "gsc_cache_render launch");
    return GSC_OK;
}

gsc_status gsc_cache_backward(const float* params, int64_t N, const gsc_camera* cam, const gsc_raster_cfg* cfg,
                              gsc_workspace* ws, const float* dL_dimage, float* grads, gsc_stream_t stream) {
    gsc_status st = raster_common(params, N, cam, cfg, ws);
    if (st) return st;
    if (!dL_dimage || (N > 0 && (!grads || !aligned(grads, 16))))
        return fail(GSC_ERR_INVALID_ARG, "dL_dimage/grads NULL or grads not 16-B aligned");
    if (N == 0) return GSC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    RasterDev rc = raster_dev(cfg);
    BatchDev b;
    batch_init(b);
    add_view(b, rc, cam, params, N, nullptr, dL_dimage, grads);
    const uint32_t* vals = nullptr;
    cudaError_t e = bin_gaussians(b, rc, ws, &vals, s, kOrderFeedback);
    if (e == cudaSuccess) e = launch_render_backward(b, rc, ws, vals, false, s);
    if (e != cudaSuccess) return cuda_fail(e, "gsc_cache_backward launch");
    return GSC_OK;
}

gsc_status gsc_render_batch(const gsc_view* views, int32_t n_views, int32_t mode, const gsc_raster_cfg* cfg,
                            gsc_workspace* ws, gsc_stream_t stream) {
    if (!views || n_views < 1 || n_views > kMaxViews)
        return fail(GSC_ERR_INVALID_ARG, "n_views must be in [1, %d]", kMaxViews);
    if (mode < GSC_BATCH_FWD || mode > (GSC_BATCH_FWD | GSC_BATCH_BWD))
        return fail(GSC_ERR_INVALID_ARG, "mode must be GSC_BATCH_FWD, GSC_BATCH_BWD or both");
    gsc_status st = check_cfg(cfg);
    if (st) return st;
    if (!ws) return fail(GSC_ERR_INVALID_ARG, "workspace is NULL");
    int64_t total = 0;
    // larger views first: the persistent kernels hand out their tiles first
    int order[kMaxViews];
    for (int i = 0; i < n_views; ++i) order[i] = i;
    for (int i = 1; i < n_views; ++i)
        for (int j = i; j > 0; --j) {
            const gsc_camera& a = views[order[j - 1]].cam;
            const gsc_camera& c = views[order[j]].cam;
            if ((int64_t)a.width * a.height >= (int64_t)c.width * c.height) break;
            int t = order[j - 1];
            order[j - 1] = order[j];
            order[j] = t;
        }
    bool shared = false;
    for (int i = 0; i < n_views; ++i) {
        const gsc_view& v = views[i];
        if ((st = check_cam(&v.cam))) return st;
        if ((st = check_ws(ws, v.N, &v.cam))) return st;
        if (v.N > 0 && (!v.params || !aligned(v.params, 16)))
            return fail(GSC_ERR_INVALID_ARG, "view %d: params NULL or not 16-B aligned", i);
        if ((mode & GSC_BATCH_FWD) && !v.image) return fail(GSC_ERR_INVALID_ARG, "view %d: image is NULL", i);
        if ((mode & GSC_BATCH_BWD) && (!v.dL_dimage || (v.N > 0 && (!v.grads || !aligned(v.grads, 16)))))
            return fail(GSC_ERR_INVALID_ARG, "view %d: dL_dimage/grads NULL or misaligned", i);
        total += v.N;
        for (int j = 0; j < i; ++j)
            if (v.grads && v.grads == views[j].grads) shared = true;
    }
    if (total > ws->max_gaussians)
        return fail(GSC_ERR_INVALID_ARG, "the batch holds %lld Gaussians, the workspace %lld", (long long)total,
                    (long long)ws->max_gaussians);
    cudaStream_t s = (cudaStream_t)stream;
    RasterDev rc = raster_dev(cfg);
    BatchDev b;
    batch_init(b);
    for (int k = 0; k < n_views; ++k) {
        const gsc_view& v = views[order[k]];
        add_view(b, rc, &v.cam, v.params, v.N, v.image, v.dL_dimage, v.grads);
    }
    if ((int64_t)b.total_bins > ws->max_tiles || (int64_t)b.total_tiles > ws->max_tiles)
        return fail(GSC_ERR_INVALID_ARG, "the batch has %u tiles and %u bins, the workspace %lld (raise max_views)",
                    b.total_tiles, b.total_bins, (long long)ws->max_tiles);
    if (total == 0) {
        if (mode & GSC_BATCH_FWD)
            for (int i = 0; i < n_views; ++i)
                GSC_CUDA(cudaMemsetAsync(views[i].image, 0,
                                         sizeof(float) * 3 * (size_t)views[i].cam.width * views[i].cam.height, s));
        return GSC_OK;
    }
    const uint32_t* vals = nullptr;
    cudaError_t e = cudaSuccess;
    if (mode & GSC_BATCH_FWD) {
        e = bin_gaussians(b, rc, ws, &vals, s);
        if (e == cudaSuccess) e = launch_render(b, rc, ws, vals, s);
    }
    if (e == cudaSuccess && (mode & GSC_BATCH_BWD)) {
        e = bin_gaussians(b, rc, ws, &vals, s, kOrderFeedback);
        if (e == cudaSuccess) e = launch_render_backward(b, rc, ws, vals, shared, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gsc_render_batch launch");
    return GSC_OK;
}

// gsc_train_batch, and with adam (m, v: per-view moment arrays) gsc_train_step
static gsc_status train_views(const gsc_train_view* views, float* const* m, float* const* v_, int32_t n_views,
                              int32_t loss_kind, const gsc_adam_params* adam, const gsc_raster_cfg* cfg,
                              gsc_workspace* ws, gsc_stream_t stream) {
    if (!views || n_views < 1 || n_views > kMaxViews)
        return fail(GSC_ERR_INVALID_ARG, "n_views must be in [1, %d]", kMaxViews);
    if (loss_kind != GSC_LOSS_HDR && loss_kind != GSC_LOSS_HDR_FULLGRAD)
        return fail(GSC_ERR_INVALID_ARG, "the training step folds in pixel-local losses only (HDR), not %d",
                    loss_kind);
    gsc_status st = check_cfg(cfg);
    if (st) return st;
    if (!ws) return fail(GSC_ERR_INVALID_ARG, "workspace is NULL");
    int order[kMaxViews];
    for (int i = 0; i < n_views; ++i) order[i] = i;
    for (int i = 1; i < n_views; ++i)
        for (int j = i; j > 0; --j) {
            const gsc_camera& a = views[order[j - 1]].cam;
            const gsc_camera& c = views[order[j]].cam;
            if ((int64_t)a.width * a.height >= (int64_t)c.width * c.height) break;
            int t = order[j - 1];
            order[j - 1] = order[j];
            order[j] = t;
        }
    int64_t total = 0;
    bool shared = false;
    for (int i = 0; i < n_views; ++i) {
        const gsc_train_view& v = views[i];
        if ((st = check_cam(&v.cam))) return st;
        if ((st = check_ws(ws, v.N, &v.cam))) return st;
        // the fused step may go without an accumulated gradient (grads NULL)
        if (v.N > 0 && (!v.params || !aligned(v.params, 16) || (!v.grads && !adam) || !aligned(v.grads, 16)))
            return fail(GSC_ERR_INVALID_ARG, "view %d: params/grads NULL or not 16-B aligned", i);
        if (!v.target || !v.loss) return fail(GSC_ERR_INVALID_ARG, "view %d: target or loss is NULL", i);
        if (adam && v.N > 0 && (!m[i] || !v_[i] || !aligned(m[i], 16) || !aligned(v_[i], 16)))
            return fail(GSC_ERR_INVALID_ARG, "view %d: m/v NULL or not 16-B aligned", i);
        total += v.N;
        for (int j = 0; j < i; ++j) {
            if (v.grads && v.grads == views[j].grads) shared = true;
            if (adam && v.N > 0 && views[j].N > 0 &&
                (v.params == views[j].params || (v.grads && v.grads == views[j].grads)))
                return fail(GSC_ERR_INVALID_ARG, "views %d and %d share parameters: the fused step needs them apart",
                            j, i);
        }
    }
    if (total > ws->max_gaussians)
        return fail(GSC_ERR_INVALID_ARG, "the batch holds %lld Gaussians, the workspace %lld", (long long)total,
                    (long long)ws->max_gaussians);
    cudaStream_t s = (cudaStream_t)stream;
    RasterDev rc = raster_dev(cfg);
    BatchDev b;
    batch_init(b);
    for (int k = 0; k < n_views; ++k) {
        const gsc_train_view& v = views[order[k]];
        add_view(b, rc, &v.cam, v.params, v.N, v.image, nullptr, v.grads);
        b.v[k].target = v.target;
        b.v[k].loss = v.loss;
        if (adam) {
            b.v[k].m = reinterpret_cast<float4*>(m[order[k]]);
            b.v[k].v = reinterpret_cast<float4*>(v_[order[k]]);
        }
    }
    if ((int64_t)b.total_bins > ws->max_tiles || (int64_t)b.total_tiles > ws->max_tiles)
        return fail(GSC_ERR_INVALID_ARG, "the batch has %u tiles and %u bins, the workspace %lld (raise max_views)",
                    b.total_tiles, b.total_bins, (long long)ws->max_tiles);
    if ((size_t)b.total_tiles * 4 > ws->red_floats)  // four loss partials per tile
        return fail(GSC_ERR_INVALID_ARG, "the batch has %u tiles, the loss scratch %zu", b.total_tiles,
                    ws->red_floats);
    AdamDev ad;
    if (adam) ad = adam_dev(*adam);
    const uint32_t* vals = nullptr;
    cudaError_t e = bin_gaussians(b, rc, ws, &vals, s, kOrderFeedback);
    if (e == cudaSuccess)
        e = launch_train(b, rc, ws, vals, loss_kind == GSC_LOSS_HDR_FULLGRAD ? 1 : 0, shared, adam ? &ad : nullptr,
                         s);
    if (e != cudaSuccess) return cuda_fail(e, adam ? "gsc_train_step launch" : "gsc_train_batch launch");
    return GSC_OK;
}

gsc_status gsc_train_batch(const gsc_train_view* views, int32_t n_views, int32_t loss_kind,
                           const gsc_raster_cfg* cfg, gsc_workspace* ws, gsc_stream_t stream) {
    return train_views(views, nullptr, nullptr, n_views, loss_kind, nullptr, cfg, ws, stream);
}

gsc_status gsc_train_step(const gsc_train_view* views, float* const* m, float* const* v, int32_t n_views,
                          int32_t loss_kind, const gsc_adam_params* adam, const gsc_raster_cfg* cfg,
                          gsc_workspace* ws, gsc_stream_t stream) {
    if (!adam || !m || !v) return fail(GSC_ERR_INVALID_ARG, "adam, m or v is NULL");
    return train_views(views, m, v, n_views, loss_kind, adam, cfg, ws, stream);
}

// ------------------------------------------------------------------ cache initialisation

gsc_status gsc_init_scratch_size(int64_t n_points, size_t* bytes) {
    if (!bytes || n_points < 4 || n_points > (int64_t)UINT32_MAX)
        return fail(GSC_ERR_INVALID_ARG, "n_points must be in [4, 2^32)");
    *bytes = init_layout(n_points, nullptr, nullptr);
    return GSC_OK;
}

gsc_status gsc_cache_init(const gsc_scene* sc, const gsc_init_params* p, void* scratch, size_t scratch_bytes,
                          float* params, gsc_stream_t stream) {
    if (!sc || !p || !scratch || !params) return fail(GSC_ERR_INVALID_ARG, "NULL argument");
    if (p->levels < 1 || p->levels > 16 || p->n_points < 4 || p->n_points > (int64_t)UINT32_MAX ||
        (p->n_points >> (p->levels - 1)) < 4)
        return fail(GSC_ERR_INVALID_ARG, "need levels in [1, 16] and at least 4 points in the last level");
    float op = p->opacity > 0.f ? p->opacity : 0.1f;
    if (!(op < 1.f)) return fail(GSC_ERR_INVALID_ARG, "opacity must be in (0, 1)");
    int attempts = p->max_attempts > 0 ? p->max_attempts : 4096;
    size_t need = init_layout(p->n_points, nullptr, nullptr);
    if (scratch_bytes < need) return fail(GSC_ERR_INVALID_ARG, "scratch holds %zu bytes, %zu needed", scratch_bytes, need);
    if (!aligned(scratch, 256) || !aligned(params, 16))
        return fail(GSC_ERR_INVALID_ARG, "scratch must be 256-B and params 16-B aligned");
    unsigned int fails = 0;
    cudaError_t e = run_init(sc, p->n_points, p->levels, p->seed, attempts, op, (char*)scratch, params, &fails,
                             (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "gsc_cache_init");
    if (fails) return fail(GSC_ERR_TIMEOUT, "%u points found no interaction in %d rays each", fails, attempts);
    return GSC_OK;
}

// ------------------------------------------------------------------ losses, optimiser

gsc_status gsc_loss(int32_t kind, const float* pred, const float* target, int32_t C, int32_t H, int32_t W,
                    const int32_t* crop, float* dL_dpred, float* loss_out, gsc_workspace* ws, gsc_stream_t stream) {
    if (!pred || !target || !loss_out || !ws) return fail(GSC_ERR_INVALID_ARG, "NULL argument");
    if (kind != GSC_LOSS_HDR && kind != GSC_LOSS_HDR_FULLGRAD && kind != GSC_LOSS_L1_SSIM)
        return fail(GSC_ERR_INVALID_ARG, "loss kind %d not available", kind);
    if (C < 1 || H < 1 || W < 1) return fail(GSC_ERR_INVALID_ARG, "empty image");
    int x0 = 0, y0 = 0, w = W, h = H;
    if (crop) {
        x0 = crop[0]; y0 = crop[1]; w = crop[2]; h = crop[3];
        // 64-bit sums: a crop such as (INT_MAX, 0, 1, H) must not wrap around into range
        if (x0 < 0 || y0 < 0 || w < 1 || h < 1 || (int64_t)x0 + w > W || (int64_t)y0 + h > H)
            return fail(GSC_ERR_INVALID_ARG, "crop outside the image");
    }
    if (kind == GSC_LOSS_L1_SSIM && (size_t)65536 + 3 * (size_t)C * w * h > ws->red_floats)
        return fail(GSC_ERR_OOM, "L1+SSIM over %d x %d x %d needs a workspace made for a larger image", C, w, h);
    cudaError_t e = launch_loss(kind, pred, target, C, H, W, x0, y0, w, h, dL_dpred, loss_out, ws->red,
                                ws->red_floats, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "gsc_loss launch");
    return GSC_OK;
}

gsc_status gsc_cache_step(float* params, float* grads, float* m, float* v, int64_t N, const gsc_adam_params* adam,
                          gsc_stream_t stream) {
    if (!adam) return fail(GSC_ERR_INVALID_ARG, "adam params NULL");
    if (N < 0) return fail(GSC_ERR_INVALID_ARG, "N < 0");
    if (N == 0) return GSC_OK;
    if (!params || !grads || !m || !v || !aligned(params, 16) || !aligned(grads, 16) || !aligned(m, 16) ||
        !aligned(v, 16))
        return fail(GSC_ERR_INVALID_ARG, "arrays must be non-NULL and 16-B aligned");
    if (adam->step < 1 || !(adam->beta1 >= 0.f && adam->beta1 < 1.f) || !(adam->beta2 >= 0.f && adam->beta2 < 1.f) ||
        !(adam->eps >= 0.f) || !(adam->weight_decay >= 0.f) || !(adam->lr_scale >= 0.f))
        return fail(GSC_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
    cudaError_t e = launch_adamw(params, grads, m, v, N, *adam, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "gsc_cache_step launch");
    return GSC_OK;
}

float gsc_lr_scale(int32_t t) { return (float)(1.0 / (1.0 + log((double)(t < 1 ? 1 : t)))); }

gsc_status gsc_profile_enable(int32_t enable) {
    prof().on.store(enable != 0);
    return GSC_OK;
}

gsc_status gsc_profile_read(gsc_profile* out, int32_t reset) {
    ProfState& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (const Pending& q : p.pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(q.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, q.a, q.b);
        if (e != cudaSuccess) return cuda_fail(e, "gsc_profile_read");
        p.ms[q.phase] += ms;
        p.launches[q.phase] += q.launches;
        p.calls[q.phase] += 1;
        p.pool.push_back(q.a);
        p.pool.push_back(q.b);
    }
    p.pending.clear();
    if (out) {
        memset(out, 0, sizeof *out);
        out->n_phases = kNumPhases;
        for (int k = 0; k < kNumPhases; ++k) {
            strncpy(out->names[k], kPhaseNames[k], 15);
            out->ms[k] = p.ms[k];
            out->launches[k] = p.launches[k];
            out->calls[k] = p.calls[k];
        }
    }
    if (reset)
        for (int k = 0; k < kNumPhases; ++k) p.ms[k] = 0, p.launches[k] = 0, p.calls[k] = 0;
    return GSC_OK;
}

int64_t gsc_launch_count(void) { return g_launches.load(); }

}  // extern "C"
