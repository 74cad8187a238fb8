/*
 * gsc.h -- C ABI of the GB300 (sm_103a) implementation of the GSCache hot
 * path: an on-the-fly trained, multi-level 3D-Gaussian path-space radiance
 * cache for volume path tracing (Bauer, Wu, Gadirov, Ma: "GSCache: Real-Time
 * Radiance Caching for Volume Path Tracing using 3D Gaussian Splatting").
 *
 * The paper exposes its caching library "via a C-style API" (Sec. 3.7); the
 * only information the cache needs from the renderer is the attenuated
 * radiance of each path sample and the path length that produced it
 * (Sec. 1).  This header is that boundary: plain C types, plain pointers and
 * sizes, no C++ or framework types.
 *
 * Conventions shared by every call
 *   - Memory.  Tensor arguments are DEVICE pointers owned by the caller,
 *     FP32, contiguous, in the layouts stated per argument.  Host-side structs
 *     are read during the call only.  The library never allocates device
 *     memory: workspaces live in a caller-provided device buffer.
 *   - Streams.  `gsc_stream_t` is a cudaStream_t (NULL = the legacy default
 *     stream).  Every call enqueues its kernels on that stream and returns
 *     without synchronising, unless its comment says otherwise.  Calls that
 *     take no workspace can be captured in a CUDA graph; workspace calls can
 *     too once the workspace exists.
 *   - Errors.  Every call returns a gsc_status.  Argument errors are found on
 *     the host before anything is enqueued (GSC_ERR_INVALID_ARG).  Launch
 *     failures return GSC_ERR_CUDA.  Conditions only the device can detect
 *     (a per-frame pair count above the workspace's capacity) set a status
 *     word in the workspace; the affected kernels then skip their work
 *     without touching memory out of bounds, and gsc_workspace_status()
 *     reports it after synchronising.  gsc_last_error() returns the message
 *     of the calling thread's last failure.  No C++ exception crosses the
 *     ABI.
 *   - Threads.  Handles are not internally locked: one thread (or one stream
 *     order) per handle.
 *
 * Packed Gaussian record (64 B, 16 FP32; the paper's 14 attributes of
 * Table 3 plus two pads so that a record is four float4 loads):
 *   [0:3] mean xyz | [3] opacity logit | [4:7] log-scale xyz | [7] pad |
 *   [8:12] rotation quaternion (w, x, y, z), need not be normalised |
 *   [12:15] linear RGB (SH degree 0, Sec. 3.6) | [15] pad
 * Gradients and the Adam moments use the same layout.
 */
#ifndef GSC_H_
#define GSC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSC_ABI_VERSION 1

typedef void* gsc_stream_t; /* a cudaStream_t */

typedef enum gsc_status {
    GSC_OK = 0,
    GSC_ERR_INVALID_ARG = 1, /* bad pointer, size, layout or configuration */
    GSC_ERR_OOM = 2,         /* a caller buffer is too small for the request */
    GSC_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    GSC_ERR_CAPACITY = 4,    /* device-detected: pairs exceed the workspace capacity */
    GSC_ERR_TIMEOUT = 5,     /* device-detected: a bounded wait ran out */
    GSC_ERR_NOT_READY = 6    /* a required earlier step has not run */
} gsc_status;

/* Pinhole camera.  x_cam = R x_world + t; R's rows are the camera's right,
 * down and forward axes in world space; pos = camera centre.  A pixel (i, j)
 * covers [i, i+1) x [j, j+1); the projection of a camera-space point is
 * (fx x/z + cx, fy y/z + cy).  Shared by the tracer and the rasterizer. */
typedef struct gsc_camera {
    float R[9];
    float t[3];
    float pos[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} gsc_camera;

/* Rasterizer configuration.  Tiles (one CTA each, one thread per pixel):
 * 16x16, 8x8, 32x8, 16x8, 8x16, 8x32 or 32x4.  Gaussians are binned into
 * coarse square bins of bin_size pixels (a multiple of tile_w and tile_h,
 * 32..512; 0 = per view, the largest of 256, 128, 64 and 32 px at most a
 * twelfth of the view's longer side); every tile walks its bin's
 * depth-ordered list and keeps the Gaussians whose support reaches the tile.  list_capacity: entries
 * staged in shared memory per batch (32..2048, multiple of 32; raised to the
 * tile's thread count if smaller).  alpha_max (0.99), alpha_min (1/255),
 * T_min (1e-4), near_plane (0.2) and dilation (0.3 px^2) are the compositing
 * constants of 3D Gaussian splatting, which the paper uses unchanged
 * (Sec. 3.1).  Tile shape, bin size and capacity change performance only,
 * never a bit of the result. */
typedef struct gsc_raster_cfg {
    int32_t tile_w, tile_h;
    int32_t list_capacity;
    float alpha_max, alpha_min, T_min, near_plane, dilation;
    int32_t bin_size;
    int32_t pixels_per_thread; /* 1, 2, 4 or 8 (0 = 1): a thread owns the pixels (x, y + k tile_h/ppt),
                                  k < ppt, of one column.  Compiled (tile, ppt): ppt 1 with 16x16, 8x8,
                                  32x8, 16x8, 8x16, 8x32, 32x4; ppt 2 with 16x16, 32x8, 16x8, 8x16, 8x32;
                                  ppt 4 and 8 with 16x16, 32x8, 8x32.  Others: GSC_ERR_INVALID_ARG. */
} gsc_raster_cfg;

/* ------------------------------------------------------------------ */
/* library                                                              */

/* ABI version (GSC_ABI_VERSION) of the loaded library. */
int32_t gsc_abi_version(void);

/* Copy the calling thread's last error message (NUL-terminated, truncated
 * to n bytes).  Returns GSC_OK. */
gsc_status gsc_last_error(char* buf, size_t n);

/* ------------------------------------------------------------------ */
/* volume scenes and the path tracer (Sec. 3.2 - 3.5)                   */

/* Volume scene: a node-centred scalar grid over the unit box [0,1]^3
 * (voxel (i,j,k) at (i/(nx-1), j/(ny-1), k/(nz-1)), trilinear, clamped to
 * the edge), mapped by a piecewise-linear RGBA transfer function of
 * s = clamp(d / density_max, 0, 1) (the paper's "predefined 1D transfer
 * function", Sec. 4.2): sigma_t = sigma_max * A(s), albedo = albedo * RGB(s).
 * Lights: one directional light (light_dir points TOWARDS the light,
 * unit length; radiance light_radiance), a constant environment
 * (env_radiance), and up to four spherical area lights outside the unit box
 * (the paper's two-light setup, Sec. 4.3), each sampled at every vertex by
 * one direction uniform in the cone it subtends; zero radiance disables a
 * light. */
#define GSC_MAX_SPHERE_LIGHTS 4
typedef struct gsc_scene_desc {
    int32_t nx, ny, nz;     /* >= 2 each */
    const float* density;   /* device, [nz][ny][nx]; caller keeps it alive while the scene exists */
    float density_max, sigma_max, albedo;
    int32_t tf_count;       /* 1..16 control points, tf_pos ascending in [0, 1] */
    float tf_pos[16];
    float tf_rgba[16][4];
    float light_dir[3], light_radiance[3], env_radiance[3];
    int32_t n_spheres;                              /* 0..GSC_MAX_SPHERE_LIGHTS */
    float sphere_center[GSC_MAX_SPHERE_LIGHTS][3];  /* the sphere may not touch the unit box */
    float sphere_radius[GSC_MAX_SPHERE_LIGHTS];     /* > 0 */
    float sphere_radiance[GSC_MAX_SPHERE_LIGHTS][3];/* emitted radiance L_e */
} gsc_scene_desc;

typedef struct gsc_scene gsc_scene;

/* Create a scene handle (host memory only; nothing is enqueued).  The
 * majorant of delta tracking is sigma_max * max_k A_k, exact for a
 * piecewise-linear TF.  Errors: GSC_ERR_INVALID_ARG for bad sizes/TF. */
gsc_status gsc_scene_create(const gsc_scene_desc* desc, gsc_scene** out);

/* Replace the transfer function (the paper's TF-change event, Sec. 1);
 * rgba holds n x 4 floats.  Takes effect for calls made afterwards. */
gsc_status gsc_scene_set_tf(gsc_scene* scene, int32_t n, const float* pos, const float* rgba);

gsc_status gsc_scene_destroy(gsc_scene* scene);

/* Path-tracing parameters.  spp >= 1 samples per pixel (jittered inside the
 * pixel when spp > 1, the pixel centre otherwise); max_bounces >= 1 (B: the
 * path stops after next-event estimation at its B-th interaction); levels K
 * in 0..16 target buffers; seed/frame select the Philox4x32-10 streams
 * (counter = (pixel, sample, frame, block), key = seed).  C > 0 enables the
 * early termination heuristic of Algorithm 1 (needs cache images); eps is
 * Algorithm 1's epsilon.  tr_out picks the reading of Algorithm 1's output
 * throughput Tr_out (Sec. 3.3-3.4): GSC_TR_OUT_CUMULATIVE (0) keeps, on a
 * surviving path, every earlier division by Tr + eps (the Russian-roulette
 * weighting of Sec. 3.4); GSC_TR_OUT_PER_CALL (1) recomputes Tr_out as the
 * product of the albedos at every call and divides by that call's Tr + eps
 * only, as the algorithm is printed.  pad must be 0. */
#define GSC_TR_OUT_CUMULATIVE 0
#define GSC_TR_OUT_PER_CALL 1
typedef struct gsc_trace_params {
    int32_t spp, max_bounces, levels;
    uint32_t frame;
    uint64_t seed;
    float C, eps;
    int32_t tr_out, pad;
} gsc_trace_params;

/* One pass of the volume path tracer with next-event estimation (Sec. 3.3):
 * delta tracking against the majorant, a path vertex at every real
 * collision (path length = number of interactions, Fig. 2), NEE of the
 * directional light (phase 1/(4 pi)) and of the environment (one uniform
 * direction) with ratio-tracked shadow transmittance, isotropic scattering.
 * Each sample's attenuated NEE radiance is written to the intermediate path
 * buffer of its length n, 1 <= n <= K (Sec. 3.5); samples of length 0 or
 * > K write nothing; buffers are averaged over spp.
 *   cache_imgs: NULL, or K x 3 x H x W cached radiance per level; when
 *               given, a path that leaves the volume with zero radiance, or
 *               is terminated early by Algorithm 1, takes the cached value
 *               of its level divided by beta (Sec. 3.3.1, Sec. 3.4, Eq. 2).
 *   targets:    K x 3 x H x W, written (K may be 0, then it may be NULL).
 *   image:      3 x H x W, the path-traced image, written.
 * H, W come from cam.  The arithmetic is FP32 without contraction and with
 * the library's own ln and sincos, so it is reproducible bit for bit. */
gsc_status gsc_trace(const gsc_scene* scene, const gsc_camera* cam, const gsc_trace_params* params,
                     const float* cache_imgs, float* targets, float* image, gsc_stream_t stream);

/* ------------------------------------------------------------------ */
/* rasterizer workspaces                                                */

typedef struct gsc_workspace gsc_workspace;

/* Bytes of device memory a workspace needs for renders of up to
 * max_gaussians Gaussians (summed over the views of a batch), up to
 * max_pairs (bin, Gaussian) pairs per binning, images up to max_w x max_h,
 * and batches of up to max_views views (1..32).  cfg is unused (NULL). */
gsc_status gsc_workspace_size(int64_t max_gaussians, int64_t max_pairs, int32_t max_w, int32_t max_h,
                              int32_t max_views, const gsc_raster_cfg* cfg, size_t* bytes);

/* Bind a workspace to the caller's device buffer (>= gsc_workspace_size
 * bytes, 256-byte aligned, owned by the caller and kept alive until
 * gsc_workspace_destroy).  Nothing is enqueued. */
gsc_status gsc_workspace_create(void* device_buffer, size_t bytes, int64_t max_gaussians, int64_t max_pairs,
                                int32_t max_w, int32_t max_h, int32_t max_views, const gsc_raster_cfg* cfg,
                                gsc_workspace** out);

gsc_status gsc_workspace_destroy(gsc_workspace* ws);

/* Synchronise `stream`, then return the device-side status of the
 * workspace (GSC_OK; GSC_ERR_CAPACITY: a binning needed more pairs than
 * the workspace holds; GSC_ERR_TIMEOUT: a bounded wait of the depth sort
 * between its CTAs ran out, which the sort's ordering rules out unless the
 * device misbehaves) and clear it.  *pairs_needed
 * (optional) receives the largest pair count any render since the last
 * call asked for, so that a caller can size a new workspace. */
gsc_status gsc_workspace_status(gsc_workspace* ws, gsc_stream_t stream, int64_t* pairs_needed);

/* Work counters of the workspace since the last call, then reset (after
 * synchronising `stream`).  out[0..9]: pairs of the last binning, largest
 * pair count, (pixel, Gaussian) pairs evaluated / composited by the
 * forward, pairs evaluated by the backward's forward re-walk, pairs
 * evaluated back to front, the sum of the pair counts of all binnings, the
 * number of binnings, pairs composited by the re-walk, and pairs that
 * contributed gradient terms back to front.  The last two are one count:
 * the pairs composited for pixels whose dL/dimage is not zero, which are the
 * pairs that contribute back to front.  out[10]: work items of the last
 * binning's order (its tiles, plus one for every extra part a gradient
 * launch split a heavy tile into; not reset).  out[11]: pairs the binnings
 * emitted for a bin of the Gaussian's tile rectangle that its falloff bound
 * cannot reach (listed in no bin; included in out[0], out[1] and out[6]).
 * n: entries wanted (<= 12). */
#define GSC_COUNTER_WORDS 12
gsc_status gsc_workspace_counters(gsc_workspace* ws, gsc_stream_t stream, int64_t* out, int32_t n);

/* ------------------------------------------------------------------ */
/* Gaussian splatting of one cache level (Sec. 3.1) and its gradient    */

/* Render the N Gaussians of one cache level into image (3 x H x W, written):
 * project each Gaussian (EWA covariance J W Sigma W^T J^T + dilation), bin it
 * into every coarse bin its alpha >= alpha_min support can touch, sort the
 * (bin, Gaussian) pairs by (bin, view depth, index), let every tile keep the
 * entries of its bin that reach it, and composite front to back per pixel
 * with early transmittance cut-off:
 *   alpha = min(alpha_max, sigmoid(o) exp(-d^T conic d / 2)), terms with
 *   alpha < alpha_min skipped, stop before a term whose T (1 - alpha) < T_min,
 *   C = sum max(c, 0) alpha T, background 0.
 * Pixel (i, j) is sampled at (i + 0.5, j + 0.5).  The result does not depend
 * on the tile size.  params: N x 16 packed records. */
gsc_status gsc_cache_render(const float* params, int64_t N, const gsc_camera* cam, const gsc_raster_cfg* cfg,
                            gsc_workspace* ws, float* image, gsc_stream_t stream);

/* Gradient of the render ("inverse splatting step", Sec. 3.5): given
 * dL/dimage (3 x H x W), ACCUMULATE (+=) dL/dparams into grads (N x 16,
 * pads untouched).  Stateless with respect to earlier renders: it re-projects,
 * re-bins and re-sorts, and re-walks each tile front to back to recover the
 * per-pixel transmittance, so no per-pixel forward state is kept. */
gsc_status gsc_cache_backward(const float* params, int64_t N, const gsc_camera* cam, const gsc_raster_cfg* cfg,
                              gsc_workspace* ws, const float* dL_dimage, float* grads, gsc_stream_t stream);

/* One view of a batched render: a cache level seen by a camera. */
typedef struct gsc_view {
    const float* params;     /* N x 16 packed records */
    int64_t N;
    gsc_camera cam;
    float* image;            /* 3 x H x W, written by the forward */
    const float* dL_dimage;  /* 3 x H x W, read by the backward */
    float* grads;            /* N x 16, accumulated (+=) by the backward; views may share it */
} gsc_view;

#define GSC_BATCH_FWD 1
#define GSC_BATCH_BWD 2

/* Render (mode & GSC_BATCH_FWD) and/or differentiate (mode & GSC_BATCH_BWD)
 * up to 32 views -- cache levels of several scenes, seen by cameras of
 * different resolutions -- with one binning over all their Gaussians and ONE
 * launch of persistent CTAs that take the tiles of all views from a shared
 * counter (the forward; the backward is another such launch).  This is the
 * paper's "joint rasterization" of several Gaussian sets (Sec. 5) as a batch.
 * Every view's result equals gsc_cache_render / gsc_cache_backward of that
 * view alone (bit for bit for the images; the gradients up to the order of
 * floating-point atomics).  All views use one cfg; the workspace must be
 * sized for the sum of the views' Gaussians and for n_views views.
 * Graph-capturable: host arguments are read during the call only. */
gsc_status gsc_render_batch(const gsc_view* views, int32_t n_views, int32_t mode, const gsc_raster_cfg* cfg,
                            gsc_workspace* ws, gsc_stream_t stream);

/* ------------------------------------------------------------------ */
/* losses (Sec. 3.6) and the optimiser step (Sec. 3.6, Eq. 4)           */

#define GSC_LOSS_HDR 0          /* (x - y)^2 / (y + 0.01)^2, denominator held constant */
#define GSC_LOSS_HDR_FULLGRAD 1 /* same value, gradient also through the denominator */
#define GSC_LOSS_L1_SSIM 2      /* 0.8 L1 + 0.2 (1 - SSIM), 11x11 Gaussian window, sigma 1.5 */

/* Loss of the prediction y = pred against the (noisy) target x = target,
 * both C x H x W, averaged over the k = C w h elements of the crop
 * (host int32 {x0, y0, w, h}; NULL = the whole image; for L1_SSIM the crop
 * is treated as its own zero-padded image).  The HDR loss is the relative L2
 * of Lehtinen et al. that the paper adopts for its unbounded radiance.
 *   dL_dpred:  C x H x W, written (0 outside the crop); may be NULL.
 *   loss_out:  device float, written.
 * Uses the workspace's reduction scratch (ws required). */
gsc_status gsc_loss(int32_t kind, const float* pred, const float* target, int32_t C, int32_t H, int32_t W,
                    const int32_t* crop, float* dL_dpred, float* loss_out, gsc_workspace* ws, gsc_stream_t stream);

/* ------------------------------------------------------------------ */
/* cache initialisation (Sec. 3.2 "Cache Initialization", Eq. 3)         */

typedef struct gsc_init_params {
    int64_t n_points;     /* N: points of level 0; level k gets N >> k (>= 4) */
    int32_t levels;       /* K, 1..16 */
    int32_t max_attempts; /* rays per point before giving up (0 = 4096) */
    uint64_t seed;        /* Philox key; ray a of point i uses the counter (i, a, 0xffffffff) */
    float opacity;        /* initial opacity of every Gaussian (0 = 0.1) */
} gsc_init_params;

/* Device scratch bytes gsc_cache_init needs for n_points points. */
gsc_status gsc_init_scratch_size(int64_t n_points, size_t* bytes);

/* Initial cache of K levels from one pass over the volume: point i casts
 * random rays (origin on the unit sphere around the box centre, aimed at a
 * uniform point of the box) until delta tracking finds a real collision, and
 * records its position and albedo.  Level k holds points 0 .. (N >> k) - 1;
 * each becomes a Gaussian at the point, coloured by its albedo, with
 * identity rotation, the given opacity and the isotropic scale of Eq. 3,
 * s = min(mu + 2 sigma, mean distance to the 3 nearest points of its level)
 * / 2, mu and sigma being the mean and population standard deviation of
 * those distances over the level.
 *   scratch: device buffer of gsc_init_scratch_size bytes, 256-B aligned.
 *   params:  device (sum_k N >> k) x 16, levels one after another (written).
 * Synchronises `stream`; GSC_ERR_TIMEOUT if some point found no collision
 * (e.g. an empty transfer function).  The paper has no further detail on the
 * rays; this is the reading used. */
gsc_status gsc_cache_init(const gsc_scene* sc, const gsc_init_params* p, void* scratch, size_t scratch_bytes,
                          float* params, gsc_stream_t stream);

/* One view of a training step: a cache level, its camera and its target
 * buffer (the path tracer's buffer for this level, Sec. 3.5). */
typedef struct gsc_train_view {
    const float* params;  /* N x 16 packed records */
    int64_t N;
    gsc_camera cam;
    const float* target;  /* 3 x H x W, the loss target x */
    float* image;         /* 3 x H x W, the rendered level (written; NULL = not wanted) */
    float* grads;         /* N x 16, accumulated (+=); views may share it */
    float* loss;          /* device float: the view's loss (written) */
} gsc_train_view;

/* The per-frame training step of the cache (render, HDR loss of Sec. 3.6,
 * backward of Sec. 3.5) for up to 32 views with the loss folded into the
 * rasterizer: one binning and ONE persistent launch in which every tile
 * composites its pixels front to back, evaluates the loss and dL/dC of each
 * pixel against its target, writes the image, and runs the back-to-front
 * gradient pass on the spot; then the per-Gaussian parameter gradients.  No
 * per-pixel quantity outlives its tile.  Equals gsc_render_batch(FWD) +
 * gsc_loss + gsc_render_batch(BWD) of the same views: images bit for bit,
 * gradients up to the order of floating-point atomics, losses up to the
 * order of summation.  loss_kind: GSC_LOSS_HDR or GSC_LOSS_HDR_FULLGRAD
 * (pixel-local losses only; others give GSC_ERR_INVALID_ARG).  The workspace
 * must be sized for the views' Gaussians and for n_views views.
 * Graph-capturable. */
gsc_status gsc_train_batch(const gsc_train_view* views, int32_t n_views, int32_t loss_kind,
                           const gsc_raster_cfg* cfg, gsc_workspace* ws, gsc_stream_t stream);

/* gsc_loss without a workspace, for callers that cannot allocate device
 * memory or hand the library a buffer at the point of the call: a plug-in
 * running inside a host application that owns every device allocation, a
 * real-time frame loop that forbids allocation after start-up, or code that
 * only has the two images.  The paper has no counterpart; this is a library
 * convenience.  Same loss kinds, crop, outputs and results as gsc_loss
 * (GSC_LOSS_L1_SSIM is not available here).
 *
 * Scratch: the per-CTA partial sums live in a fixed array inside the library
 * (32,768 floats, 128 KiB, held by every device that loads the library until
 * the process exits), so C * w * h may be at most 8,388,608 elements (e.g.
 * 3 x 1920 x 1080 fits); larger crops return GSC_ERR_CAPACITY.  The first
 * call on each device looks up the array's device address (with that device
 * current), so make that first call before capturing a stream into a graph.
 * That address is kept for the life of the process: a cudaDeviceReset (or
 * anything else that replaces the device's primary context) after the first
 * call is not supported, since later calls would write through the old address.
 * Every call uses the same array: calls that can run at the same time on the
 * GPU (different streams without ordering) race and give wrong losses.
 * Nothing in the array needs clearing between calls.  Allocates nothing. */
gsc_status gsc_loss_noalloc(int32_t kind, const float* pred, const float* target, int32_t C, int32_t H, int32_t W,
                            const int32_t* crop, float* dL_dpred, float* loss_out, gsc_stream_t stream);

/* AdamW with decoupled weight decay (Sec. 3.6 "Regularization"); per-slot
 * learning rates (the paper's per-attribute LRs, Sec. 4.1) scaled by
 * lr_scale (Eq. 4, see gsc_lr_scale).  step is 1-based (bias correction).
 * weight_decay = 0 is plain Adam.  Slots with lr 0 are left unchanged. */
typedef struct gsc_adam_params {
    float lr[16];
    float beta1, beta2, eps, weight_decay, lr_scale;
    int32_t step;
} gsc_adam_params;

/* One optimiser step over N records: updates params, m, v in place and
 * zeroes grads.  All N x 16 FP32 device arrays. */
gsc_status gsc_cache_step(float* params, float* grads, float* m, float* v, int64_t N, const gsc_adam_params* adam,
                          gsc_stream_t stream);

/* gsc_train_batch and gsc_cache_step of every view in one call: the training
 * step of Sec. 3.6 (render, HDR loss, backward) whose per-Gaussian gradient
 * kernel also takes the AdamW step, so the parameter gradients never go
 * through memory.  Views must not share parameters or gradients (each view
 * is its own cache level); params of every view are updated IN PLACE
 * (the const in gsc_train_view does not apply here), m[i] and v[i] are view
 * i's first and second moments (N x 16 FP32 device arrays, 16-B aligned),
 * and a view's grads, if not NULL, is read as an accumulated gradient (added
 * to this step's) and zeroed; NULL means none, and saves its traffic.  Every
 * Gaussian of every view takes the step, whether its view saw it or not,
 * exactly as gsc_cache_step over the same records would.  Equals
 * gsc_train_batch followed by gsc_cache_step per view up to the order of
 * floating-point atomics.  GSC_ERR_INVALID_ARG: adam, m or v NULL, a view's
 * m or v NULL or misaligned, views sharing parameters, or any condition of
 * gsc_train_batch.  Graph-capturable. */
gsc_status gsc_train_step(const gsc_train_view* views, float* const* m, float* const* v, int32_t n_views,
                          int32_t loss_kind, const gsc_adam_params* adam, const gsc_raster_cfg* cfg,
                          gsc_workspace* ws, gsc_stream_t stream);

/* Eq. 4: the learning-rate factor 1 / (1 + ln t) after t >= 1 frames of an
 * unchanged viewport (t = 1 on the first frame after a change). */
float gsc_lr_scale(int32_t t);

/* ------------------------------------------------------------------ */
/* instrumentation (no counterpart in the paper; used by benchmarks)    */

#define GSC_PROFILE_MAX_PHASES 24

/* Device time per kernel phase, measured with CUDA events recorded on the
 * stream each phase is launched on.  Phases: project, depth_sort, scan,
 * emit, tile_sort, ranges, render, render_bwd, project_bwd, loss, adamw,
 * trace. */
typedef struct gsc_profile {
    int32_t n_phases;
    char names[GSC_PROFILE_MAX_PHASES][16];
    double ms[GSC_PROFILE_MAX_PHASES];       /* summed event time */
    int64_t launches[GSC_PROFILE_MAX_PHASES]; /* kernel launches */
    int64_t calls[GSC_PROFILE_MAX_PHASES];    /* timed intervals */
} gsc_profile;

/* Start (1) or stop (0) recording phase events.  Must not be enabled while a
 * stream is being captured into a CUDA graph. */
gsc_status gsc_profile_enable(int32_t enable);

/* Synchronise the recorded events, return the per-phase sums since the last
 * reset, and reset them if reset != 0. */
gsc_status gsc_profile_read(gsc_profile* out, int32_t reset);

/* Number of kernels this library has launched since it was loaded
 * (counted on the host at each launch site). */
int64_t gsc_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* GSC_H_ */
