/*
 * airgs.h -- C ABI of the AirGS splatting library (sm_103a).
 *
 * The library evaluates the data-parallel path of AirGS (arXiv 2512.20943):
 *   - decode and apply of a frame's streamed Gaussian update, shipped as a
 *     multi-channel 16-bit 2D map with one Gaussian per pixel and one attribute
 *     per channel (Sec. II, Eq. 3), applied to the previous frame
 *     (GS_{t+1} = GS_t + d_{t+1}, Sec. III-B, Eq. 5) or to the anchor
 *     (GS_t = GC_k + D_t, Sec. III-C);
 *   - rendering of Gaussians G = {mu, alpha, c, SH, R, S}, Sigma = R S S^T R^T
 *     (Sec. II) with a differentiable tile-based splatting rasterizer: EWA
 *     projection, SH colour, 16x16 tile binning, a stable (tile, depth) order
 *     and front-to-back alpha blending with
 *       alpha = min(alpha_max, o exp(-1/2 d^T Sigma'^-1 d)),
 *     pairs with alpha < alpha_min skipped, and a pixel stopped before the
 *     Gaussian that would take T below T_min;
 *   - the adjoint of the rasterizer (the "differentiable splatting renderer" of
 *     Sec. II) with the L1 term of Eq. 1;
 *   - the per-Gaussian blend weight sum(alpha_i T_i) and blended-pair count,
 *     the usage frequency behind the adaptive pruning of Sec. III-C.
 *
 * Conventions
 *   - Every pointer argument named as "device" is CUDA device memory owned by
 *     the caller; the library never frees it.  Host pointers are read during
 *     the call only.
 *   - All work is enqueued on the context's stream and is asynchronous, except
 *     where a call says it synchronises.  The caller must keep device inputs
 *     alive and unmodified until the stream has passed the call.
 *   - Gaussian parameters are float32, structure of arrays: means [N][3],
 *     log_scales [N][3], quats [N][4] (w, x, y, z; any norm), opacity_logit [N],
 *     sh [N][K][3] with K = (sh_degree + 1)^2, sh_degree 0..3.
 *   - Images are float32 planar: view v occupies [3][H_v][W_v] starting at
 *     3 * sum_{u<v} H_u W_u in the output buffer; single-channel outputs
 *     (T, n_contrib) start at sum_{u<v} H_u W_u.
 *   - Pixel (x, y) is sampled at (x + 0.5, y + 0.5).  Cameras look down +z with
 *     x right and y down.
 *   - Return value: AIRGS_OK or a negative AIRGS_E_* code; airgs_last_error()
 *     describes the failure.  No C++ exception crosses this boundary.
 */
#ifndef AIRGS_H
#define AIRGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AIRGS_OK 0
#define AIRGS_E_ARG (-1)      /* invalid argument (sizes, degree, null pointer) */
#define AIRGS_E_OOM (-2)      /* device allocation failed */
#define AIRGS_E_CAPACITY (-3) /* a size limit was exceeded */
#define AIRGS_E_TIMEOUT (-4)  /* a bounded device wait gave up */
#define AIRGS_E_CUDA (-5)     /* a CUDA runtime call failed */
#define AIRGS_E_STATE (-6)    /* call out of order (no anchor, state released) */

/* apply_frame_update modes */
#define AIRGS_DELTA_PREV 0   /* apply d_t to the current frame state */
#define AIRGS_DELTA_ANCHOR 1 /* apply D_t to the anchor */
#define AIRGS_QUAT_ADD 2     /* flag: q = q_base + dq instead of normalize(dq (x) q_base) */

#define AIRGS_UPDATE_CHANNELS 7 /* dx, dy, dz, qw, qx, qy, qz */
#define AIRGS_MAX_VIEWS 256

typedef struct airgs_ctx airgs_ctx;     /* opaque: device state, scratch, stream */
typedef struct airgs_state airgs_state; /* opaque: what render saved for render_backward */

/* Rasterizer settings (3DGS values by default). */
typedef struct {
  float dilation;  /* added to the 2D covariance diagonal (0.3) */
  float alpha_max; /* 0.99 */
  float alpha_min; /* 1/255 */
  float T_min;     /* 1e-4 */
  float bg[3];     /* background colour, added as T_final * bg (black) */
  int kernel_shape;           /* -1: autotuned per workload (shape 0 until tuned), else a fixed index
                                 into the compiled kernel shapes (airgs_shape_count / airgs_shape_name) */
  int sort_mode;              /* 0: global two-stage radix ordering; 1: per-tile ordering (lists
                                 sorted in shared memory) when every list fits one CTA; -1 (default):
                                 per-tile for batches of at most 65536 (view, Gaussian) pairs, where
                                 the radix path's fixed cost dominates, else radix */
  const char* autotune_cache; /* nullable path of a text cache of autotune choices */
  int cull_lists;             /* 1 (default): a render that does not return n_contrib lists a Gaussian
                                 only in the tiles of its rectangle in which it can reach alpha_min;
                                 images, T, importance and the backward's gradients are those of the
                                 full lists (the dropped entries are skipped by every pixel), but a
                                 saved state's lists, list positions and pair counts are those of the
                                 culled lists.  0: always the full rectangle lists (the definition's
                                 lists, as the radix ordering builds them) */
} airgs_config;

typedef struct {
  int width, height;
  float fx, fy, cx, cy;
  float viewmat[16]; /* world -> camera, row-major 4x4 */
  float near_plane;  /* z <= near_plane is culled (0.2) */
} airgs_camera;

typedef struct {
  int64_t n;
  int sh_degree;
  const float* means;         /* device [n][3] */
  const float* log_scales;    /* device [n][3] */
  const float* quats;         /* device [n][4] */
  const float* opacity_logit; /* device [n] */
  const float* sh;            /* device [n][K][3] */
} airgs_gaussians;

/* Per-call counters, filled by airgs_state_stats. */
typedef struct {
  int64_t n_instances;   /* (tile, Gaussian) list entries over all views */
  int64_t n_tiles;       /* 16x16 tiles over all views */
  int64_t n_pixels;      /* pixels over all views */
  int64_t pairs_forward; /* (pixel, list entry) pairs of the lists the render built, up to termination */
  int64_t pairs_backward;/* pairs replayed by the backward (list positions < n_contrib) */
  int kernel_shape;      /* kernel shape the render ran */
} airgs_stats;

/* Fill *cfg with the defaults above. */
void airgs_default_config(airgs_config* cfg);

/* Create a context bound to the current CUDA device and to `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  cfg may be NULL. */
int airgs_create(airgs_ctx** out, const airgs_config* cfg, void* stream);
int airgs_destroy(airgs_ctx* ctx);
int airgs_set_stream(airgs_ctx* ctx, void* stream);
/* Block until the context's stream is idle, then report any device-side
 * status (AIRGS_E_CAPACITY, AIRGS_E_TIMEOUT) raised since the last sync. */
int airgs_sync(airgs_ctx* ctx);
/* Message of the last failure on this context ("" if none).  Valid until the
 * next call on the context. */
const char* airgs_last_error(const airgs_ctx* ctx);

/* set_anchor: copy the canonical Gaussian set GC_k of a keyframe (Sec. II
 * Eq. 2, Sec. III-C) into the context; the current frame state is reset to the
 * anchor.  Pointers are device [n]... arrays as in airgs_gaussians; copied
 * before return (asynchronously on the stream). */
int airgs_set_anchor(airgs_ctx* ctx, int64_t n, int sh_degree, const float* means, const float* log_scales,
                     const float* quats, const float* opacity_logit, const float* sh);

/* apply_frame_update: decode one frame's update map and apply it (Sec. II
 * Eq. 3; Sec. III-B Eq. 5; Sec. III-C d_t / D_t).
 *   map     device uint16 [7][map_h][map_w], channel c of Gaussian i at pixel i
 *           (row-major); pixels >= n are ignored.  Requires n <= map_w * map_h.
 *   lo, hi  host float[7]: channel c decodes as lo[c] + u (hi[c] - lo[c]) / 65535.
 *   mode    AIRGS_DELTA_PREV (base = current frame) or AIRGS_DELTA_ANCHOR
 *           (base = anchor), optionally | AIRGS_QUAT_ADD.
 * Result: means = base_means + (dx, dy, dz); quats = normalize(dq (x) base_q)
 * (Hamilton product) or base_q + dq.  Scales, opacity and SH stay the
 * anchor's.  frame_id is recorded only. */
int airgs_apply_frame_update(airgs_ctx* ctx, const uint16_t* map, int map_w, int map_h, const float* lo,
                             const float* hi, int mode, int64_t frame_id);

/* Copy the current frame's means [n][3] and quats [n][4] into device buffers. */
int airgs_get_frame_state(airgs_ctx* ctx, float* means_out, float* quats_out);

/* render: forward over n_views cameras (host array) of the current frame
 * state.  Outputs (device, caller-owned):
 *   rgb_out         float [sum 3 H W]   C + T_final bg, planar per view (required)
 *   T_out           float [sum H W]     final transmittance (nullable)
 *   n_contrib_out   int32 [sum H W]     1 + list position of the last blended Gaussian (nullable)
 *   importance_w    float [n]           += sum over blended pairs of alpha_i T_i (nullable)
 *   importance_cnt  uint32 [n]          += number of blended pairs (nullable)
 *   saved           if not NULL, receives a state for render_backward; the
 *                   state reads rgb_out again, so rgb_out must stay unmodified
 *                   until the state is released.
 * Synchronises once on the stream to size the tile lists. */
int airgs_render(airgs_ctx* ctx, const airgs_camera* cams, int n_views, float* rgb_out, float* T_out,
                 int32_t* n_contrib_out, float* importance_w, uint32_t* importance_cnt, airgs_state** saved);

/* render_gaussians: as airgs_render, for a caller-owned Gaussian set (the
 * training path); the parameters must stay unmodified while a saved state
 * refers to them. */
int airgs_render_gaussians(airgs_ctx* ctx, const airgs_gaussians* g, const airgs_camera* cams, int n_views,
                           float* rgb_out, float* T_out, int32_t* n_contrib_out, float* importance_w,
                           uint32_t* importance_cnt, airgs_state** saved);

/* render_backward: adjoint of the render that produced `saved`, given
 * dL/d(rgb) laid out like rgb_out (device).  Gradients with respect to the raw
 * parameters (means, log_scales, quats, opacity_logit, sh) are written to the
 * device buffers g_* (overwritten; shapes as the parameters).  importance_w /
 * importance_cnt (nullable) accumulate as in render, computed during the
 * backward replay. */
int airgs_render_backward(airgs_ctx* ctx, airgs_state* saved, const float* dL_drgb, float* g_means,
                          float* g_log_scales, float* g_quats, float* g_opacity_logit, float* g_sh,
                          float* importance_w, uint32_t* importance_cnt);

/* render_backward_l1: as render_backward with dL/d(rgb) taken from the L1 term
 * of Eq. 1, L = mean |rgb - target| over views, pixels and channels
 * (gradient sign(rgb - target) / (3 sum H W), sign(0) = 0), fused into the
 * backward.  target is laid out like rgb_out; loss_out (device float, nullable)
 * receives L (overwritten). */
int airgs_render_backward_l1(airgs_ctx* ctx, airgs_state* saved, const float* target, float* loss_out,
                             float* g_means, float* g_log_scales, float* g_quats, float* g_opacity_logit,
                             float* g_sh, float* importance_w, uint32_t* importance_cnt);

/* Optional outputs of the adjoint, for render_backward_ex. */
typedef struct {
  const float* dL_drgb;     /* dL/d(rgb) laid out like rgb_out (ignored when target is set) */
  const float* target;      /* nullable: L1 of Eq. 1 against this image, fused (as render_backward_l1) */
  float* loss_out;          /* nullable device float: the L1 loss when target is set */
  float* g_means;           /* device gradients, overwritten (required) */
  float* g_log_scales;
  float* g_quats;
  float* g_opacity_logit;
  float* g_sh;
  float* importance_w;      /* nullable, += blend weight (with importance_cnt) */
  uint32_t* importance_cnt;
  float* densify_grad;      /* nullable, += sum over views of |dL/d mean2d| in pixels (with densify_views) */
  uint32_t* densify_views;  /* nullable, += number of views in which the Gaussian is visible */
} airgs_backward_args;

/* render_backward_ex: the adjoint with every optional output; densify_grad and
 * densify_views are the statistics of the densification step of keyframe
 * reconstruction (Sec. III-B: Gaussians with large screen-space gradients are
 * cloned or split). */
int airgs_render_backward_ex(airgs_ctx* ctx, airgs_state* saved, const airgs_backward_args* args);

/* mask_out[i] = 1 where densify_views[i] > 0 and the mean screen-space gradient
 * densify_grad[i] / densify_views[i] exceeds threshold (the paper leaves the
 * threshold open), else 0.  All device arrays of length n. */
int airgs_densify_select(airgs_ctx* ctx, const float* densify_grad, const uint32_t* densify_views, int64_t n,
                         float threshold, uint8_t* mask_out);

/* Output of airgs_densify_apply: device buffers with room for `capacity`
 * Gaussians each (capacity >= 2 n: every input Gaussian yields at most two
 * outputs), laid out as airgs_gaussians with the same sh_degree. */
typedef struct {
  int64_t capacity;
  float* means;          /* device [capacity][3] */
  float* log_scales;     /* device [capacity][3] */
  float* quats;          /* device [capacity][4], 16-byte aligned */
  float* opacity_logit;  /* device [capacity] */
  float* sh;             /* device [capacity][K][3] */
  uint32_t* parent;      /* nullable device [capacity]: the input index of each output Gaussian */
  int64_t* n_out;        /* device: the number of output Gaussians (written) */
} airgs_densify_out;

/* densify_apply: the clone / split / discard step of keyframe reconstruction
 * (Sec. III-B: Gaussians in high-gradient regions are cloned or split, and
 * Gaussians of low opacity are discarded), with the clone and split rules of
 * the adaptive density control of 3D Gaussian Splatting.  For each input
 * Gaussian i (g, device):
 *   select[i] != 0 and every log_scale <= log(size_threshold): kept, plus an identical copy;
 *   select[i] != 0 otherwise: replaced by two children j = 0, 1 with
 *     mean = mean_i + R(q_i/|q_i|) diag(exp(log_scale_i)) z[i][j],
 *     log_scale = log_scale_i - log(split_factor), quaternion, opacity logit and SH copied;
 *   select[i] == 0: kept;
 *   opacity_logit[i] < logit(min_opacity): discarded, with its copy or children
 *     (min_opacity 0 discards nothing).
 * The comparisons are float32, against log(size_threshold) and
 * logit(min_opacity) rounded to float32 once.  select: device uint8 [n] (for
 * example from airgs_densify_select); z: device float [n][2][3], standard normal
 * samples the caller draws (only the rows of split Gaussians are read).
 * Output rows: the kept originals, then the copies, then the children (two per
 * split Gaussian), each group in input order; *out->n_out receives the count
 * (asynchronously, like every output).  Arguments: size_threshold > 0,
 * split_factor > 0, 0 <= min_opacity < 1 (else AIRGS_E_ARG);
 * out->capacity < 2 n is AIRGS_E_CAPACITY.  The output buffers must not overlap
 * the inputs. */
int airgs_densify_apply(airgs_ctx* ctx, const airgs_gaussians* g, const uint8_t* select, const float* z,
                        float size_threshold, float split_factor, float min_opacity, const airgs_densify_out* out);

/* gaussian_importance: the per-Gaussian blend weight and blended-pair count of
 * the current frame over n_views cameras, without colour output (the usage
 * frequency of Sec. III-C).  w_out [n] float and cnt_out [n] uint32 are
 * overwritten (device). */
int airgs_gaussian_importance(airgs_ctx* ctx, const airgs_camera* cams, int n_views, float* w_out,
                              uint32_t* cnt_out);

/* Usage-frequency pruning p(.) of Sec. III-C.  keep_out[i] = 0 for the
 * n_prune Gaussians with the smallest blend weight importance[i] (the usage
 * frequency airgs_gaussian_importance or the render calls accumulate), 1 for
 * the others; equal weights prune the lower index first, negative or NaN
 * weights rank lowest.  importance: device float [n]; keep_out: device uint8
 * [n].  0 <= n_prune <= n. */
int airgs_prune_mask(airgs_ctx* ctx, const float* importance, int64_t n, int64_t n_prune, uint8_t* keep_out);

/* Pruned differential delta of Sec. III-C, d'_t = p(D_t - D'_{t-1}): for every
 * Gaussian i and channel c of channel-major device float arrays [channels][n],
 *   d_out = keep[i] ? D_t - D_sent : 0,   then   D_sent += d_out,
 * so D_sent goes from the record D'_{t-1} of what was transmitted to D'_t.
 * Channels are treated additively (the paper's GS_{t+1} = GS_t + d_{t+1}).
 * nonzero_out (device uint64, nullable) receives the number of Gaussians whose
 * transmitted delta has a non-zero channel (the delta's size in Gaussians). */
int airgs_prune_delta(airgs_ctx* ctx, int64_t n, int channels, const float* D_t, float* D_sent, const uint8_t* keep,
                      float* d_out, uint64_t* nonzero_out);

/* apply_frame_delta: as airgs_apply_frame_update with an already decoded
 * float delta (device, channel-major [7][n]: dx, dy, dz, qw, qx, qy, qz). */
int airgs_apply_frame_delta(airgs_ctx* ctx, const float* delta, int mode, int64_t frame_id);

/* Per-view sum of squared differences of two images laid out like rgb_out
 * (device float), written to sse_out[n_views] (device double, overwritten);
 * the PSNR of a pruning level is 10 log10(3 H W / sse) for images in [0, 1]. */
int airgs_image_sse(airgs_ctx* ctx, const airgs_camera* cams, int n_views, const float* a, const float* b,
                    double* sse_out);

/* The 3DGS training loss of Eq. 1, L = (1 - lambda) L1 + lambda (1 - SSIM)
 * (lambda = 0.2 in Sec. IV-A), over all views, and its gradient with respect
 * to the rendered image, to feed airgs_render_backward.  SSIM per (view,
 * channel) with an 11x11 Gaussian window (sigma 1.5, normalised, zero padding,
 * output the size of the image), C1 = 0.01^2, C2 = 0.03^2, averaged over
 * views, pixels and channels; L1 is the mean absolute difference.
 *   rgb, target   device float laid out like rgb_out
 *   loss_out      device double[3] (nullable): L, L1, SSIM
 *   dL_drgb_out   device float laid out like rgb_out (overwritten)
 * Returns once the work is queued on the context's stream (the per-plane table
 * is staged from host memory before the call returns); the outputs are valid
 * in stream order, like those of airgs_render. */
int airgs_l3dgs_loss(airgs_ctx* ctx, const airgs_camera* cams, int n_views, const float* rgb, const float* target,
                     float lambda, double* loss_out, float* dL_drgb_out);

/* Release a state returned by a render call (its device memory is returned to
 * the context's pool once the stream passes this point). */
int airgs_release_state(airgs_ctx* ctx, airgs_state* state);

/* Counters of the render that produced `state` (synchronises on the stream). */
int airgs_state_stats(airgs_ctx* ctx, const airgs_state* state, airgs_stats* out);

/* Inspection of a state for parity tests (device outputs, caller-owned):
 *   view-local projection of each Gaussian: mean2d [n][2], depth [n],
 *   radius [n] (0 when culled);
 *   the view's tile lists: ranges [tiles][2] int64 (start, end) relative to the
 *   view's first entry, ids [entries] int32 (Gaussian index per list entry).
 * airgs_state_view_info returns the view's tile count and list length. */
int airgs_state_view_info(airgs_ctx* ctx, const airgs_state* state, int view, int64_t* n_tiles,
                          int64_t* n_entries);
int airgs_state_projection(airgs_ctx* ctx, const airgs_state* state, int view, float* mean2d, float* depth,
                           int32_t* radius);
int airgs_state_tile_lists(airgs_ctx* ctx, const airgs_state* state, int view, int64_t* ranges, int32_t* ids);

/* Stable LSD radix sort of (key, value) pairs by the key bits [0, key_bits),
 * the sort the tile ordering uses: keys_in/vals_in are device uint32 [n];
 * results go to keys_out/vals_out (device, distinct from the inputs).
 * Allocates its scratch from the context's pool. */
int airgs_sort_pairs(airgs_ctx* ctx, const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                     uint32_t* vals_out, int64_t n, int key_bits);

/* Allocation-free variant of airgs_sort_pairs, for callers that cannot
 * allocate device memory while they run (cudaMalloc / cudaFree can
 * synchronise the whole device and stall other streams; engine plug-ins and
 * real-time loops often run under a memory budget owned by their host).  The
 * paper has no counterpart: this is a service of the library, not a step of
 * the method.
 *   keys_in, vals_in    device uint32 [n], read only
 *   keys_out, vals_out  device uint32 [n], the pairs stably sorted by key bits
 *                       [0, key_bits); must not overlap the inputs
 *   stream              cudaStream_t the work is enqueued on (NULL = legacy)
 * Needs no context and calls no allocator: its scratch is a fixed device
 * array of 2 * AIRGS_NOALLOC_SORT_MAX_PAIRS + 262144 uint32 words (about 9 MB)
 * that every GPU loading the library holds until the process exits.  Every
 * call looks up that array's device address on the current device (a host-side
 * lookup that allocates nothing, so the address stays right after
 * cudaDeviceReset or under another context); the first call in a context may
 * load the library's device code, so make it before any stream capture.  All
 * calls share the array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  Returns AIRGS_E_CAPACITY if n > AIRGS_NOALLOC_SORT_MAX_PAIRS,
 * AIRGS_E_ARG for bad arguments, AIRGS_E_CUDA if a launch fails. */
#define AIRGS_NOALLOC_SORT_MAX_PAIRS (1 << 20)
int airgs_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                             uint32_t* vals_out, int64_t n, int key_bits, void* stream);

/* Autotune the kernel shape for this workload (n Gaussians of the current
 * frame, the given cameras): a coordinate search over the compiled shapes --
 * first the blend backward's (staged entries per batch, warps per SM), then
 * the blend forward's, then the radix sort's keys per thread, then the
 * emission's instances per thread -- timing the
 * training step as it runs (render with saved state, then the fused L1
 * backward with usage-frequency accumulation, against a constant target) with
 * CUDA events on the context's stream, best of 3 repetitions after one
 * warm-up.  Shape 0 is always among the candidates, so the choice is never
 * slower than it by the timing.  The choice is cached per (n, total pixels,
 * n_views), used by later renders of that workload when kernel_shape is -1,
 * and written to the config's cache path if set.  *shape receives the choice;
 * ms_default / ms_best (nullable) the step times of shape 0 and of the
 * choice.  Synchronises the context's stream. */
int airgs_autotune(airgs_ctx* ctx, const airgs_camera* cams, int n_views, int* shape, float* ms_default,
                   float* ms_best);

/* Per-stage device timing.  With profiling level AIRGS_PROFILE_ALL, each
 * pipeline stage (decode, projection, depth sort, scan+emit, tile sort, ranges,
 * blend forward, blend backward, projection backward) is bracketed by CUDA
 * events on the context's stream; with AIRGS_PROFILE_BLEND only the two blend
 * stages are (two event pairs per training step instead of nine, so the rest of
 * the pipeline runs as it does unprofiled); with either level the blend kernels
 * also add their evaluated pairs to a context counter.  airgs_set_profiling
 * returns AIRGS_E_ARG for any other level than the three below.
 * airgs_stage_times synchronises, writes the summed milliseconds and the
 * number of timed launches of each stage since the previous readout into
 * ms[AIRGS_NUM_STAGES] / launches[AIRGS_NUM_STAGES], and into pairs[4] (each
 * nullable) the forward and backward pair totals of the definition (list
 * entries up to termination / below n_contrib) followed by the forward and
 * backward lane evaluations the blend kernels actually issued (32 per 8x4
 * pixel block they evaluate); then clears them. */
#define AIRGS_NUM_STAGES 9
#define AIRGS_PROFILE_OFF 0
#define AIRGS_PROFILE_ALL 1
#define AIRGS_PROFILE_BLEND 2
int airgs_set_profiling(airgs_ctx* ctx, int enabled);
int airgs_stage_times(airgs_ctx* ctx, double* ms, int64_t* launches, int64_t* pairs);
const char* airgs_stage_name(int stage);

/* Measured FP32 throughput of the context's GPU (an FMA probe, 16 independent
 * chains per thread, 8 CTAs of 256 threads per SM, fastest of three timed
 * runs) in TFLOP/s -> *tflops.  Synchronises the context's stream.  The
 * measurement aid for the blend kernels' roofline; the paper has no
 * counterpart.  Returns AIRGS_E_ARG for a null pointer, AIRGS_E_OOM or
 * AIRGS_E_CUDA on failure. */
int airgs_measure_fp32_peak(airgs_ctx* ctx, double* tflops);

/* Measured shared-memory load throughput of the context's GPU, in TB/s, into
 * *tbs (host pointer): conflict-free 16-byte shared loads from every SM, timed
 * with CUDA events on the context's stream (synchronous).  A measurement aid
 * for the blend kernels' shared-memory roofline; the paper has no counterpart.
 * Returns AIRGS_E_ARG for a null pointer, AIRGS_E_OOM or AIRGS_E_CUDA on
 * failure. */
int airgs_measure_smem_peak(airgs_ctx* ctx, double* tbs);

/* Process-wide number of kernel launches the library has issued. */
int64_t airgs_kernel_launch_count(void);

/* Number of compiled kernel shapes and a short name of each ("fwd B/W bwd
 * B/W keys K run R": staged entries per batch and warps per SM of the blend
 * forward and backward, radix keys per thread of the instance sort, instances
 * per thread of the emission).  Shape 0 is the default. */
int airgs_shape_count(void);
const char* airgs_shape_name(int shape);

#ifdef __cplusplus
}
#endif

#endif /* AIRGS_H */
