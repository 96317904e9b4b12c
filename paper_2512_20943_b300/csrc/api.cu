// C ABI of the AirGS splatting library: context, device memory, and the
// render / backward / update pipelines built from the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "airgs.h"
#include "airgs_internal.cuh"
#include "kernels.h"

using namespace airgs;

static std::atomic<int64_t> g_launches{0};
void airgs::count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Stages timed with CUDA events on the context's stream when profiling is on.
enum Stage {
  ST_DECODE = 0,
  ST_PROJECT,
  ST_DEPTH_SORT,
  ST_EMIT,
  ST_TILE_SORT,
  ST_RANGES,
  ST_BLEND_FWD,
  ST_BLEND_BWD,
  ST_PROJECT_BWD,
  ST_COUNT
};
static const char* kStageNames[ST_COUNT] = {"decode_apply", "project_sh",  "depth_sort",  "scan_emit",  "tile_sort",
                                            "tile_ranges",  "blend_fwd",   "blend_bwd",   "project_bwd"};

struct airgs_ctx {
  airgs_config cfg;
  std::string autotune_path;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 148;
  int l2_bytes = 126 << 20;
  cudaMemPool_t pool = nullptr;
  // anchor GC_k and the current frame state
  int64_t n = 0;
  int sh_degree = -1;
  float *a_means = nullptr, *a_log_scales = nullptr, *a_quats = nullptr, *a_opacity = nullptr, *a_sh = nullptr;
  float *c_means = nullptr, *c_quats = nullptr;
  int64_t frame_id = -1;
  uint64_t* h_pinned = nullptr;  // small pinned host buffer for counters
  // pinned staging of the cameras a render uploads (two slots, each reused once
  // the copy out of it has run: a copy from pinned memory is a plain DMA)
  CamDev* h_cam_ring = nullptr;  // [2][AIRGS_MAX_VIEWS]
  cudaEvent_t cam_copied[2] = {nullptr, nullptr};
  int cam_slot = 0;
  cudaEvent_t count_ready = nullptr;  // the instance count has reached h_pinned
  std::string last_error;
  std::map<std::string, int> tuned;  // autotune choices
  // profiling: (stage, start, end) event triples awaiting readout
  int profiling = AIRGS_PROFILE_OFF;
  unsigned long long* d_pair_total = nullptr;  // [4] forward, backward pairs; forward, backward issued evaluations
  std::vector<cudaEvent_t> event_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
};

struct airgs_state {
  int n_views = 0;
  int64_t n = 0;
  int sh_degree = 0;
  const float *means = nullptr, *log_scales = nullptr, *quats = nullptr, *opacity = nullptr, *sh = nullptr;
  std::vector<CamDev> h_cams;
  CamDev* d_cams = nullptr;
  ProjRec* proj = nullptr;     // [V][N]
  uint32_t* ids = nullptr;     // sorted instance values
  uint2* ranges = nullptr;     // [tiles]
  int32_t* ncontrib = nullptr; // [pixels]
  uint2* hl = nullptr;         // half-tile lists, nullable (lists of 2^28 entries or more: the full lists)
  uint2* hranges = nullptr;    // [2][tiles]
  uint32_t* order = nullptr;   // [2 tiles] queue order of the blend kernels' half-tile items (with hl)
  GradRec* grad = nullptr;     // [V][N] blend-backward accumulators, zeroed during the render (saved states)
  bool grad_zeroed = false;    // grad holds zeros (not yet used by a backward)
  // [5] device counters, 8 bytes each: forward pairs, forward work queue,
  // backward pairs, backward work queue (int in the low half; the backward's
  // two are adjacent, so one memset resets them), tile instances
  unsigned long long* counters = nullptr;
  const float* rgb = nullptr;  // caller's forward output
  // tile instances; -1 while only the device counter holds the count (a render
  // that did not wait for it: n_inst_bound bounds it)
  int64_t n_inst = 0, n_inst_bound = 0, n_tiles = 0, n_pixels = 0;
  int shape = 0;               // kernel shape (shape_parts) the render ran and the backward runs
  std::vector<void*> owned;    // device allocations to free on release
};

// ------------------------------------------------------------------ helpers
namespace {

int fail(airgs_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->last_error = buf;
  return code;
}

// Batches of at most this many (view, Gaussian) pairs take the per-tile ordering by default (sort_mode -1):
// measured on a 2k-Gaussian, 128x128 render, 0.68 ms against 0.94 ms with the radix ordering.
constexpr int64_t kSmallOrdering = 65536;
// A per-tile ordering whose instance count is bounded by at most this many entries (every Gaussian of a view in
// every tile of it) and whose lists cannot outgrow one CTA's sort (at most kTileSortBig Gaussians) sizes its
// instance arrays by that bound instead of reading the count back: the render then never waits for the device.
constexpr int64_t kNoWaitInstances = 1ll << 22;
// The blend kernels' queue is ordered longest list first while it holds at most this many items per resident warp
// (32 per SM): with few items per warp the last long ones set the kernel's end (streaming step, 18 per warp: 2.5 %
// faster); with many, the tail is short anyway and the tile order keeps neighbouring tiles, which share Gaussians,
// in flight together.
constexpr int64_t kOrderMaxItemsPerWarp = 64;

// Groups of the blend queue's order: as many views as keep a group's projection and gradient records within half
// of L2, except the last group, which holds at least kOrderGroupItemsPerWarp items per resident warp (the longest
// lists are about three times the mean: the last group's longest items then start well before its end).
// Streaming step (8 views of 300k Gaussians): groups of 2, 2 and 4 views; with 2 groups of 4 views the backward took
// 1.845 ms with 1.03 GB of DRAM traffic, with 4 groups of 2 (4 items per warp in the last) 1.855 ms and 0.78 GB,
// with one group 1.845 ms and 1.32 GB.
constexpr int64_t kOrderGroupItemsPerWarp = 8;
void order_groups(const airgs_ctx* ctx, int64_t n, int n_views, int64_t n_tiles, int* views_per_group,
                  int* last_views) {
  const int64_t per_view = n * (int64_t)(sizeof(ProjRec) + sizeof(GradRec));
  const int64_t vpg = per_view > 0 ? (int64_t)ctx->l2_bytes / 2 / per_view : n_views;
  const int64_t items_per_view = 2 * n_tiles / (n_views > 0 ? n_views : 1);
  const int64_t need = kOrderGroupItemsPerWarp * 32ll * ctx->num_sms;
  const int64_t last = items_per_view > 0 ? (need + items_per_view - 1) / items_per_view : n_views;
  *views_per_group = (int)std::max<int64_t>(1, std::min<int64_t>(vpg, n_views));
  *last_views = (int)std::max<int64_t>(*views_per_group, std::min<int64_t>(last, n_views));
}

#define CK(expr)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (expr);                                                                      \
    if (e_ != cudaSuccess) return fail(ctx, AIRGS_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

template <class T>
int dalloc(airgs_ctx* ctx, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMallocFromPoolAsync((void**)p, count * sizeof(T), ctx->pool, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, AIRGS_E_OOM, "device allocation of %zu bytes failed: %s", count * sizeof(T),
                cudaGetErrorString(e));
  }
  return AIRGS_OK;
}

void dfree(airgs_ctx* ctx, void* p) {
  if (p) cudaFreeAsync(p, ctx->stream);
}

void free_anchor(airgs_ctx* ctx) {
  for (float** p : {&ctx->a_means, &ctx->a_log_scales, &ctx->a_quats, &ctx->a_opacity, &ctx->a_sh, &ctx->c_means,
                    &ctx->c_quats}) {
    dfree(ctx, *p);
    *p = nullptr;
  }
  ctx->n = 0;
  ctx->sh_degree = -1;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

int build_cams(airgs_ctx* ctx, const airgs_camera* cams, int n_views, std::vector<CamDev>& out, int64_t& n_tiles,
               int64_t& n_pixels) {
  if (!cams || n_views <= 0 || n_views > AIRGS_MAX_VIEWS)
    return fail(ctx, AIRGS_E_ARG, "n_views must be in [1, %d]", AIRGS_MAX_VIEWS);
  out.resize(n_views);
  n_tiles = 0;
  n_pixels = 0;
  for (int v = 0; v < n_views; ++v) {
    const airgs_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 65536 || c.height > 65536 || !(c.fx > 0) || !(c.fy > 0))
      return fail(ctx, AIRGS_E_ARG, "camera %d: bad size or focal length", v);
    CamDev& d = out[v];
    for (int r = 0; r < 3; ++r) {
      for (int k = 0; k < 3; ++k) d.R[3 * r + k] = c.viewmat[4 * r + k];
      d.t[r] = c.viewmat[4 * r + 3];
    }
    for (int k = 0; k < 3; ++k)
      d.campos[k] = -(d.R[k] * d.t[0] + d.R[3 + k] * d.t[1] + d.R[6 + k] * d.t[2]);
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    d.znear = c.near_plane;
    d.limx = 1.3f * (float)c.width / (2.f * c.fx);
    d.limy = 1.3f * (float)c.height / (2.f * c.fy);
    d.W = c.width;
    d.H = c.height;
    d.TW = (c.width + kTile - 1) / kTile;
    d.TH = (c.height + kTile - 1) / kTile;
    d.tile_base = n_tiles;
    d.pix_base = n_pixels;
    n_tiles += (int64_t)d.TW * d.TH;
    n_pixels += (int64_t)c.width * c.height;
  }
  if (n_tiles >= (1ll << 30)) return fail(ctx, AIRGS_E_CAPACITY, "too many tiles (%lld)", (long long)n_tiles);
  return AIRGS_OK;
}

int check_gaussians(airgs_ctx* ctx, const airgs_gaussians* g) {
  if (!g || g->n < 0 || g->n >= (1ll << 31)) return fail(ctx, AIRGS_E_ARG, "Gaussian count out of range");
  if (g->sh_degree < 0 || g->sh_degree > 3) return fail(ctx, AIRGS_E_ARG, "sh_degree must be 0..3");
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logit || !g->sh))
    return fail(ctx, AIRGS_E_ARG, "null Gaussian parameter pointer");
  if (g->n > 0 && !aligned16(g->quats)) return fail(ctx, AIRGS_E_ARG, "quats must be 16-byte aligned");
  return AIRGS_OK;
}

RasterParams raster_params(const airgs_config& c) {
  RasterParams rp;
  rp.dilation = c.dilation;
  rp.alpha_max = c.alpha_max;
  rp.alpha_min = c.alpha_min;
  rp.T_min = c.T_min;
  for (int k = 0; k < 3; ++k) rp.bg[k] = c.bg[k];
  return rp;
}

int bits_for(int64_t count) {
  int b = 0;
  while ((1ll << b) < count) ++b;
  return std::max(b, 1);
}

void release_state(airgs_ctx* ctx, airgs_state* s) {
  if (!s) return;
  for (void* p : s->owned) dfree(ctx, p);
  delete s;
}

cudaEvent_t take_event(airgs_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// RAII stage timer: records a start event now and an end event at scope exit.
struct StageScope {
  airgs_ctx* ctx;
  int stage;
  cudaEvent_t e0 = nullptr;
  StageScope(airgs_ctx* c, int s) : ctx(c), stage(s) {
    if (ctx->profiling == AIRGS_PROFILE_ALL ||
        (ctx->profiling == AIRGS_PROFILE_BLEND && (s == ST_BLEND_FWD || s == ST_BLEND_BWD))) {
      e0 = take_event(ctx);
      cudaEventRecord(e0, ctx->stream);
    }
  }
  ~StageScope() {
    if (e0) {
      cudaEvent_t e1 = take_event(ctx);
      cudaEventRecord(e1, ctx->stream);
      ctx->pending.push_back({stage, {e0, e1}});
    }
  }
};

}  // namespace

const char* airgs::shape_name(int shape) {
  struct Names {
    char s[kShapes][48];
    Names() {
      const int fwd[kFwdShapes][2] = {{32, 28}, {16, 28}, {64, 28}, {32, 32}, {32, 24}};
      const int bwd[kBwdShapes][2] = {{32, 32}, {16, 32}, {64, 32}, {32, 28}, {32, 24}};
      for (int i = 0; i < kShapes; ++i) {
        const ShapeParts p = shape_parts(i);
        snprintf(s[i], sizeof(s[i]), "fwd %d/%d bwd %d/%d keys %d run %d", fwd[p.fwd][0], fwd[p.fwd][1],
                 bwd[p.bwd][0], bwd[p.bwd][1], sort_keys_of(p.sort), emit_run_of(p.emit));
      }
    }
  };
  static const Names names;  // built once (thread-safe initialisation of a local static)
  return (shape >= 0 && shape < kShapes) ? names.s[shape] : "";
}

namespace {

std::string tune_key(int64_t n, int64_t pixels, int views) {
  std::ostringstream os;
  os << n << ":" << pixels << ":" << views;
  return os.str();
}

int choose_shape(airgs_ctx* ctx, int64_t n, int64_t pixels, int views) {
  if (ctx->cfg.kernel_shape >= 0 && ctx->cfg.kernel_shape < kShapes) return ctx->cfg.kernel_shape;
  auto it = ctx->tuned.find(tune_key(n, pixels, views));
  if (it != ctx->tuned.end()) return it->second;
  return 0;  // the default shape unless tuned otherwise
}

// Forward pipeline: project -> depth sort -> emit -> tile sort -> ranges -> blend.
int render_impl(airgs_ctx* ctx, const airgs_gaussians* g, const airgs_camera* cams, int n_views, float* rgb_out,
                float* T_out, int32_t* nc_out, float* imp_w, uint32_t* imp_cnt, airgs_state** saved,
                int forced_shape) {
  if (saved) *saved = nullptr;
  int rc = check_gaussians(ctx, g);
  if (rc) return rc;
  if (!rgb_out) return fail(ctx, AIRGS_E_ARG, "rgb_out is required");
  if ((imp_w == nullptr) != (imp_cnt == nullptr))
    return fail(ctx, AIRGS_E_ARG, "importance_w and importance_cnt go together");
  airgs_state* s = new (std::nothrow) airgs_state();
  if (!s) return fail(ctx, AIRGS_E_OOM, "host allocation failed");
  struct Guard {
    airgs_ctx* c;
    airgs_state* s;
    bool keep = false;
    ~Guard() {
      if (!keep) release_state(c, s);
    }
  } guard{ctx, s};

  rc = build_cams(ctx, cams, n_views, s->h_cams, s->n_tiles, s->n_pixels);
  if (rc) return rc;
  const int64_t N = g->n, V = n_views;
  s->n_views = n_views;
  s->n = N;
  s->sh_degree = g->sh_degree;
  s->means = g->means;
  s->log_scales = g->log_scales;
  s->quats = g->quats;
  s->opacity = g->opacity_logit;
  s->sh = g->sh;
  s->rgb = rgb_out;
  s->shape = forced_shape >= 0 ? forced_shape : choose_shape(ctx, N, s->n_pixels, n_views);
  const ShapeParts parts = shape_parts(s->shape);
  cudaStream_t st = ctx->stream;

#define ALLOC(ptr, count)                      \
  do {                                         \
    int r_ = dalloc(ctx, &(ptr), (count));     \
    if (r_) return r_;                         \
    s->owned.push_back((void*)(ptr));          \
  } while (0)
  // A state saved for a backward gets its gradient accumulators here, zeroed
  // while the host waits for the instance count (the GPU would otherwise idle
  // through that round trip); the backward then skips its own memset.
#define PREFILL_GRAD()                                                                  \
  do {                                                                                  \
    if (saved && !s->grad && N > 0) {                                                   \
      ALLOC(s->grad, V * N);                                                            \
      CK(cudaMemsetAsync(s->grad, 0, (size_t)V * N * sizeof(GradRec), st));            \
      s->grad_zeroed = true;                                                            \
    }                                                                                   \
  } while (0)
  ALLOC(s->d_cams, V);
  ALLOC(s->proj, V * N);
  ALLOC(s->ranges, s->n_tiles);
  ALLOC(s->ncontrib, s->n_pixels);
  ALLOC(s->counters, 5);
  {
    const int slot = ctx->cam_slot;
    CK(cudaEventSynchronize(ctx->cam_copied[slot]));  // the slot's previous copy (complete unless just enqueued)
    CamDev* staged = ctx->h_cam_ring + (size_t)slot * AIRGS_MAX_VIEWS;
    std::copy(s->h_cams.begin(), s->h_cams.end(), staged);
    CK(cudaMemcpyAsync(s->d_cams, staged, V * sizeof(CamDev), cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ctx->cam_copied[slot], st));
    ctx->cam_slot = slot ^ 1;
  }
  CK(cudaMemsetAsync(s->counters, 0, 5 * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(s->ranges, 0, s->n_tiles * sizeof(uint2), st));
  RasterParams rp = raster_params(ctx->cfg);

  // temporaries of the ordering stage
  std::vector<void*> tmp;
  struct TmpGuard {
    airgs_ctx* c;
    std::vector<void*>& t;
    ~TmpGuard() {
      for (void* p : t) dfree(c, p);
    }
  } tguard{ctx, tmp};
#define TALLOC(ptr, count)                     \
  do {                                         \
    int r_ = dalloc(ctx, &(ptr), (count));     \
    if (r_) return r_;                         \
    tmp.push_back((void*)(ptr));               \
  } while (0)

  int64_t n_inst = 0;
  if (N > 0) {
    uint32_t *dkeys, *tiles, *tile_counts = nullptr;
    TALLOC(dkeys, V * N);
    TALLOC(tiles, V * N);
    // ordering path: per-tile lists sorted in shared memory on request, or by default for small batches,
    // where the radix path's fixed cost (4 + 2 passes of 3 launches) dominates; the radix path otherwise
    const bool per_tile = ctx->cfg.sort_mode == 1 || (ctx->cfg.sort_mode == -1 && V * N <= kSmallOrdering);
    // unless the caller asks for n_contrib (positions in the definition's lists), a Gaussian is listed only in
    // tiles of its rectangle where it can reach alpha_min: the dropped entries are skipped by every pixel of their
    // tile, so images, T, blend weights and the backward's replay (which walks the same lists) are unchanged.  A
    // state saved for a backward (training: small footprints, where the exact row bands cost more to compute than
    // they save) takes the alpha_min box; a render without state (serving: large footprints) the exact bands.
    const int cull = (ctx->cfg.cull_lists == 0 || nc_out || per_tile) ? kCullNone : (saved ? kCullBox : kCullBands);
    if (per_tile) {
      TALLOC(tile_counts, s->n_tiles);
      CK(cudaMemsetAsync(tile_counts, 0, s->n_tiles * sizeof(uint32_t), st));
    }
    {
      StageScope sc(ctx, ST_PROJECT);
      CK(launch_project(st, N, g->sh_degree, g->means, g->log_scales, g->quats, g->opacity_logit, g->sh, s->d_cams,
                        n_views, rp, s->proj, dkeys, tiles, tile_counts, cull));
    }
    bool use_radix = !per_tile;
    // no wait for the instance count: an upper bound that keeps the arrays small, and lists that fit one CTA
    int64_t bound = 0;
    for (const CamDev& c : s->h_cams) bound += N * (int64_t)c.TW * c.TH;
    const bool no_wait = per_tile && N <= kTileSortBig && bound <= kNoWaitInstances;
    if (per_tile && no_wait) {
      // per-tile lists as below, sized by the bound; the count stays on the device (counters[4])
      const int64_t chunks = (int64_t)tile_offsets_chunks(s->n_tiles);
      uint64_t* csum;
      uint32_t *cursor, *big_list, *info;
      TALLOC(csum, chunks + 1);
      TALLOC(cursor, s->n_tiles);
      TALLOC(big_list, s->n_tiles);
      TALLOC(info, 4);
      CK(cudaMemsetAsync(info, 0, 4 * sizeof(uint32_t), st));
      {
        StageScope sc(ctx, ST_EMIT);
        CK(launch_tile_offsets(st, tile_counts, s->n_tiles, csum, s->ranges, cursor, big_list, info));
      }
      CK(cudaMemcpyAsync(s->counters + 4, csum + chunks, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
      PREFILL_GRAD();
      s->n_inst = -1;
      s->n_inst_bound = bound;
      if (bound > 0) {
        uint2* ipairs;
        uint32_t* ivals;
        TALLOC(ipairs, bound);
        ALLOC(ivals, bound);
        {
          StageScope sc(ctx, ST_EMIT);
          CK(launch_scatter(st, V * N, N, s->proj, s->d_cams, dkeys, cursor, ipairs));
        }
        {
          StageScope sc(ctx, ST_TILE_SORT);
          // lists longer than one 256-thread CTA's share: at most bound / kTileSortSmall of them
          const int64_t big_max = std::min<int64_t>(s->n_tiles, bound / kTileSortSmall);
          CK(launch_sort_tiles(st, s->n_tiles, s->ranges, big_list, big_max, ipairs, ivals, info + 1));
        }
        s->ids = ivals;
      }
    } else if (per_tile) {
      // per-tile lists: offsets from the counts, scatter, sort each list in shared memory
      const int64_t chunks = (int64_t)tile_offsets_chunks(s->n_tiles);
      uint64_t* csum;
      uint32_t *cursor, *big_list, *info;
      TALLOC(csum, chunks + 1);
      TALLOC(cursor, s->n_tiles);
      TALLOC(big_list, s->n_tiles);
      TALLOC(info, 4);
      CK(cudaMemsetAsync(info, 0, 4 * sizeof(uint32_t), st));
      {
        StageScope sc(ctx, ST_EMIT);
        CK(launch_tile_offsets(st, tile_counts, s->n_tiles, csum, s->ranges, cursor, big_list, info));
      }
      CK(cudaMemcpyAsync(ctx->h_pinned, csum + chunks, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(ctx->h_pinned + 1, info, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
      CK(cudaEventRecord(ctx->count_ready, st));
      PREFILL_GRAD();
      CK(cudaEventSynchronize(ctx->count_ready));
      n_inst = (int64_t)ctx->h_pinned[0];
      const uint32_t longest = (uint32_t)(ctx->h_pinned[1] & 0xFFFFFFFFu);
      const int64_t n_big = (int64_t)(ctx->h_pinned[1] >> 32);
      if (n_inst >= (int64_t)0xFFFFFFFFll)
        return fail(ctx, AIRGS_E_CAPACITY, "%lld tile instances exceed the 32-bit list limit", (long long)n_inst);
      s->n_inst = n_inst;
      if (longest > (uint32_t)kTileSortBig) {
        use_radix = true;  // a list too long for one CTA: order globally instead
        CK(cudaMemsetAsync(s->ranges, 0, s->n_tiles * sizeof(uint2), st));
      } else if (n_inst > 0) {
        uint2* ipairs;
        uint32_t* ivals;
        TALLOC(ipairs, n_inst);
        ALLOC(ivals, n_inst);
        {
          StageScope sc(ctx, ST_EMIT);
          CK(launch_scatter(st, V * N, N, s->proj, s->d_cams, dkeys, cursor, ipairs));
        }
        {
          StageScope sc(ctx, ST_TILE_SORT);
          CK(launch_sort_tiles(st, s->n_tiles, s->ranges, big_list, n_big, ipairs, ivals, nullptr));
        }
        s->ids = ivals;
      }
    }
    if (use_radix) {
      uint32_t *keys_b, *vals_a, *vals_b, *counts_sorted, *rs_scratch;
      uint64_t* chunk;
      TALLOC(keys_b, V * N);
      TALLOC(vals_a, V * N);
      TALLOC(vals_b, V * N);
      TALLOC(counts_sorted, V * N);
      TALLOC(rs_scratch, radix_scratch_bytes(N, n_views, ctx->num_sms) / sizeof(uint32_t) + 1);
      int64_t n_chunks = emit_chunks(V * N);
      TALLOC(chunk, n_chunks + 1);
      bool in_b = false;
      {
        StageScope sc(ctx, ST_DEPTH_SORT);
        CK(radix_sort_pairs(st, ctx->num_sms, dkeys, vals_a, keys_b, vals_b, N, n_views, 32, true, rs_scratch,
                            &in_b));
      }
      const uint32_t* order = in_b ? vals_b : vals_a;
      int64_t nc2 = 0;
      {
        StageScope sc(ctx, ST_EMIT);
        CK(launch_count_gather(st, V * N, N, order, tiles, counts_sorted, chunk, &nc2));
        CK(launch_scan_spans(st, chunk, nc2, chunk + n_chunks));
      }
      CK(cudaMemcpyAsync(ctx->h_pinned, chunk + n_chunks, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
      CK(cudaEventRecord(ctx->count_ready, st));
      PREFILL_GRAD();
      CK(cudaEventSynchronize(ctx->count_ready));
      n_inst = (int64_t)ctx->h_pinned[0];
      if (n_inst >= (int64_t)0xFFFF0000ll)
        return fail(ctx, AIRGS_E_CAPACITY, "%lld tile instances exceed the 32-bit list limit", (long long)n_inst);
      s->n_inst = n_inst;
      if (n_inst > 0) {
        uint32_t *ikeys_a, *ikeys_b, *ivals_b, *ivals_a, *rs2, *pieces;
        TALLOC(ikeys_a, n_inst);
        TALLOC(ikeys_b, n_inst);
        TALLOC(ivals_b, n_inst);
        ALLOC(ivals_a, n_inst);  // may end up holding the sorted values
        const int sort_keys = sort_keys_of(parts.sort);
        TALLOC(rs2, radix_scratch_bytes(n_inst, 1, ctx->num_sms, sort_keys) / sizeof(uint32_t) + 1);
        {
          StageScope sc(ctx, ST_EMIT);
          TALLOC(pieces, emit_piece_words(V * N, n_inst));
          CK(launch_emit(st, V * N, N, order, counts_sorted, chunk, n_inst, pieces, s->proj, s->d_cams,
                         ctx->cfg.alpha_min, s->n_tiles, cull, emit_run_of(parts.emit), ikeys_a, ivals_a));
        }
        bool in_b2 = false;
        {
          StageScope sc(ctx, ST_TILE_SORT);
          CK(radix_sort_pairs(st, ctx->num_sms, ikeys_a, ivals_a, ikeys_b, ivals_b, n_inst, 1,
                              bits_for(s->n_tiles), false, rs2, &in_b2, sort_keys));
        }
        const uint32_t* skeys = in_b2 ? ikeys_b : ikeys_a;
        if (in_b2) {
          // keep the sorted values: move ivals_b into the state, ivals_a to the temporaries
          s->owned.back() = ivals_b;
          tmp.erase(std::find(tmp.begin(), tmp.end(), (void*)ivals_b));
          tmp.push_back(ivals_a);
          s->ids = ivals_b;
        } else {
          s->ids = ivals_a;
        }
        const bool half_lists = n_inst < (1ll << 28);
        if (!half_lists) {  // (the half-list pass writes the ranges itself)
          StageScope sc(ctx, ST_RANGES);
          CK(launch_tile_ranges(st, n_inst, skeys, s->ranges));
        }
        if (half_lists) {
          // compacted half-tile lists for the half-tile culling kernels (list positions fit 28 bits;
          // otherwise the kernels walk the full lists and test the blocks themselves)
          const int64_t hchunks = (int64_t)half_list_chunks(n_inst);
          uint8_t* hflags;
          uint64_t* hsums;
          TALLOC(hflags, n_inst);
          TALLOC(hsums, 2 * (hchunks + 1));
          ALLOC(s->hl, 2 * n_inst);
          ALLOC(s->hranges, 2 * s->n_tiles);
          CK(cudaMemsetAsync(s->hranges, 0, 2 * s->n_tiles * sizeof(uint2), st));
          StageScope sc(ctx, ST_RANGES);
          CK(launch_half_lists(st, skeys, s->ids, s->ranges, s->d_cams, n_views, s->proj, N, n_inst,
                               ctx->cfg.alpha_min, s->n_tiles, hflags, hsums, s->hl, s->hranges));
          if (2 * s->n_tiles <= kOrderMaxItemsPerWarp * 32ll * ctx->num_sms) {
            uint32_t* oscratch;
            TALLOC(oscratch, item_order_words(n_views));
            ALLOC(s->order, 2 * s->n_tiles);
            int vpg = 1, last_views = 1;
            order_groups(ctx, N, n_views, s->n_tiles, &vpg, &last_views);
            CK(launch_item_order(st, ctx->num_sms, s->hranges, s->d_cams, n_views, vpg, last_views, s->n_tiles,
                                 oscratch, s->order));
          }
        }
      }
    }
  }

  BlendArgs a;
  a.proj = s->proj;
  a.n = N;
  a.ids = s->ids;
  a.ranges = s->ranges;
  a.cams = s->d_cams;
  a.n_views = n_views;
  a.n_tiles = s->n_tiles;
  a.rp = rp;
  a.work_counter = reinterpret_cast<int*>(s->counters + 1);
  a.pair_counter = s->counters;
  a.pair_total = ctx->profiling ? ctx->d_pair_total : nullptr;
  a.exec_total = ctx->profiling ? ctx->d_pair_total + 2 : nullptr;
  a.hl = s->hl;
  a.hl_mut = s->hl;
  a.hranges = s->hranges;
  a.work_order = s->order;
  FwdOut o;
  o.rgb = rgb_out;
  o.T = T_out;
  o.ncontrib = s->ncontrib;
  o.ncontrib_user = nc_out;
  o.imp_w = imp_w;
  o.imp_cnt = imp_cnt;
  {
    StageScope sc(ctx, ST_BLEND_FWD);
    CK(launch_blend_fwd(st, parts.fwd, ctx->num_sms, a, o));
  }
#undef PREFILL_GRAD
#undef ALLOC
#undef TALLOC
  if (saved) {
    guard.keep = true;
    *saved = s;
  }
  return AIRGS_OK;
}

int backward_impl(airgs_ctx* ctx, airgs_state* s, const float* dL, const float* target, float* loss_out,
                  float* g_means, float* g_log_scales, float* g_quats, float* g_opacity, float* g_sh, float* imp_w,
                  uint32_t* imp_cnt, float* dens_grad = nullptr, uint32_t* dens_views = nullptr) {
  if (!s) return fail(ctx, AIRGS_E_STATE, "null state");
  if (!dL && !target) return fail(ctx, AIRGS_E_ARG, "dL_drgb or target required");
  if (s->n > 0 && (!g_means || !g_log_scales || !g_quats || !g_opacity || !g_sh))
    return fail(ctx, AIRGS_E_ARG, "null gradient pointer");
  if (s->n > 0 && !aligned16(g_quats)) return fail(ctx, AIRGS_E_ARG, "g_quats must be 16-byte aligned");
  if ((imp_w == nullptr) != (imp_cnt == nullptr))
    return fail(ctx, AIRGS_E_ARG, "importance_w and importance_cnt go together");
  if ((dens_grad == nullptr) != (dens_views == nullptr))
    return fail(ctx, AIRGS_E_ARG, "densify_grad and densify_views go together");
  cudaStream_t st = ctx->stream;
  if (loss_out) CK(cudaMemsetAsync(loss_out, 0, sizeof(float), st));
  if (s->n == 0) return AIRGS_OK;
  // the accumulators the render zeroed for this state, else a temporary
  GradRec* grad = s->grad;
  struct G {
    airgs_ctx* c;
    void* p;
    ~G() { dfree(c, p); }
  } gguard{ctx, nullptr};
  if (!grad) {
    int rc = dalloc(ctx, &grad, (size_t)s->n_views * s->n);
    if (rc) return rc;
    gguard.p = grad;
  }
  if (!(grad == s->grad && s->grad_zeroed))
    CK(cudaMemsetAsync(grad, 0, (size_t)s->n_views * s->n * sizeof(GradRec), st));
  if (grad == s->grad) s->grad_zeroed = false;  // a second backward of the state zeroes them again
  CK(cudaMemsetAsync(s->counters + 2, 0, 2 * sizeof(unsigned long long), st));
  BlendArgs a;
  a.proj = s->proj;
  a.n = s->n;
  a.ids = s->ids;
  a.ranges = s->ranges;
  a.cams = s->d_cams;
  a.n_views = s->n_views;
  a.n_tiles = s->n_tiles;
  a.rp = raster_params(ctx->cfg);
  a.work_counter = reinterpret_cast<int*>(s->counters + 3);
  a.pair_counter = s->counters + 2;
  a.pair_total = ctx->profiling ? ctx->d_pair_total + 1 : nullptr;
  a.exec_total = ctx->profiling ? ctx->d_pair_total + 3 : nullptr;
  a.hl = s->hl;
  a.hl_mut = s->hl;
  a.hranges = s->hranges;
  a.work_order = s->order;
  BwdIn in;
  in.rgb = s->rgb;
  in.dL = dL;
  in.target = target;
  in.inv_norm = (float)(1.0 / (3.0 * (double)s->n_pixels));
  in.loss = loss_out;
  in.ncontrib = s->ncontrib;
  in.grad = grad;
  in.imp_w = imp_w;
  in.imp_cnt = imp_cnt;
  if (s->n_inst > 0 || (s->n_inst < 0 && s->n_inst_bound > 0)) {
    StageScope sc(ctx, ST_BLEND_BWD);
    CK(launch_blend_bwd(st, shape_parts(s->shape).bwd, ctx->num_sms, a, in));
  }
  StageScope sc(ctx, ST_PROJECT_BWD);
  CK(launch_project_bwd(st, s->n, s->sh_degree, s->means, s->log_scales, s->quats, s->opacity, s->sh, s->d_cams,
                        s->n_views, s->proj, grad, g_means, g_log_scales, g_quats, g_opacity, g_sh, dens_grad,
                        dens_views, imp_w, imp_cnt));
  return AIRGS_OK;
}

airgs_gaussians frame_gaussians(const airgs_ctx* ctx) {
  airgs_gaussians g;
  g.n = ctx->n;
  g.sh_degree = ctx->sh_degree;
  g.means = ctx->c_means;
  g.log_scales = ctx->a_log_scales;
  g.quats = ctx->c_quats;
  g.opacity_logit = ctx->a_opacity;
  g.sh = ctx->a_sh;
  return g;
}

__global__ void k_extract_projection(const ProjRec* proj, int64_t n, float* mean2d, float* depth, int32_t* radius) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ProjRec r = proj[i];
  if (mean2d) {
    mean2d[2 * i] = r.a.x;
    mean2d[2 * i + 1] = r.a.y;
  }
  if (depth) depth[i] = r.c.y;
  if (radius) radius[i] = __float_as_int(r.c.z);
}

void load_tune_cache(airgs_ctx* ctx) {
  if (ctx->autotune_path.empty()) return;
  std::ifstream f(ctx->autotune_path);
  std::string key;
  int v;
  while (f >> key >> v)
    if (v >= 0 && v < kShapes) ctx->tuned[key] = v;
}

void save_tune_cache(airgs_ctx* ctx) {
  if (ctx->autotune_path.empty()) return;
  std::ofstream f(ctx->autotune_path, std::ios::trunc);
  for (auto& kv : ctx->tuned) f << kv.first << " " << kv.second << "\n";
}

}  // namespace

// ------------------------------------------------------------------ ABI
extern "C" {

void airgs_default_config(airgs_config* c) {
  if (!c) return;
  c->dilation = 0.3f;
  c->alpha_max = 0.99f;
  c->alpha_min = 1.0f / 255.0f;
  c->T_min = 1e-4f;
  c->bg[0] = c->bg[1] = c->bg[2] = 0.f;
  c->kernel_shape = -1;
  c->sort_mode = -1;
  c->autotune_cache = nullptr;
  c->cull_lists = 1;
}

int airgs_create(airgs_ctx** out, const airgs_config* cfg, void* stream) {
  if (!out) return AIRGS_E_ARG;
  *out = nullptr;
  airgs_ctx* ctx = new (std::nothrow) airgs_ctx();
  if (!ctx) return AIRGS_E_OOM;
  airgs_default_config(&ctx->cfg);
  if (cfg) {
    ctx->cfg = *cfg;
    if (cfg->autotune_cache) ctx->autotune_path = cfg->autotune_cache;
    ctx->cfg.autotune_cache = nullptr;
  }
  if (!(ctx->cfg.alpha_max > 0 && ctx->cfg.alpha_max < 1) || !(ctx->cfg.alpha_min >= 0) || !(ctx->cfg.T_min >= 0) ||
      !(ctx->cfg.dilation >= 0)) {
    delete ctx;
    return AIRGS_E_ARG;
  }
  ctx->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->l2_bytes, cudaDevAttrL2CacheSize, ctx->device);
  if (e == cudaSuccess) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    e = cudaMemPoolCreate(&ctx->pool, &props);
  }
  if (e == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_pinned, 128);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_cam_ring, 2 * AIRGS_MAX_VIEWS * sizeof(CamDev));
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ctx->cam_copied[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->count_ready, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (cudaEvent_t ev : ctx->cam_copied)
      if (ev) cudaEventDestroy(ev);
    if (ctx->count_ready) cudaEventDestroy(ctx->count_ready);
    if (ctx->h_cam_ring) cudaFreeHost(ctx->h_cam_ring);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    delete ctx;
    return AIRGS_E_CUDA;
  }
  load_tune_cache(ctx);
  *out = ctx;
  return AIRGS_OK;
}

int airgs_destroy(airgs_ctx* ctx) {
  if (!ctx) return AIRGS_E_ARG;
  free_anchor(ctx);
  dfree(ctx, ctx->d_pair_total);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->h_cam_ring) cudaFreeHost(ctx->h_cam_ring);
  for (cudaEvent_t ev : ctx->cam_copied)
    if (ev) cudaEventDestroy(ev);
  if (ctx->count_ready) cudaEventDestroy(ctx->count_ready);
  for (auto& p : ctx->pending) ctx->event_pool.insert(ctx->event_pool.end(), {p.second.first, p.second.second});
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
  return AIRGS_OK;
}

int airgs_set_stream(airgs_ctx* ctx, void* stream) {
  if (!ctx) return AIRGS_E_ARG;
  ctx->stream = (cudaStream_t)stream;
  return AIRGS_OK;
}

int airgs_sync(airgs_ctx* ctx) {
  if (!ctx) return AIRGS_E_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  return AIRGS_OK;
}

const char* airgs_last_error(const airgs_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int airgs_set_anchor(airgs_ctx* ctx, int64_t n, int sh_degree, const float* means, const float* log_scales,
                     const float* quats, const float* opacity_logit, const float* sh) {
  if (!ctx) return AIRGS_E_ARG;
  airgs_gaussians g{n, sh_degree, means, log_scales, quats, opacity_logit, sh};
  int rc = check_gaussians(ctx, &g);
  if (rc) return rc;
  free_anchor(ctx);
  int K = (sh_degree + 1) * (sh_degree + 1);
  if ((rc = dalloc(ctx, &ctx->a_means, 3 * n)) || (rc = dalloc(ctx, &ctx->a_log_scales, 3 * n)) ||
      (rc = dalloc(ctx, &ctx->a_quats, 4 * n)) || (rc = dalloc(ctx, &ctx->a_opacity, n)) ||
      (rc = dalloc(ctx, &ctx->a_sh, (size_t)K * 3 * n)) || (rc = dalloc(ctx, &ctx->c_means, 3 * n)) ||
      (rc = dalloc(ctx, &ctx->c_quats, 4 * n))) {
    free_anchor(ctx);
    return rc;
  }
  cudaStream_t st = ctx->stream;
  if (n > 0) {
    CK(cudaMemcpyAsync(ctx->a_means, means, 12 * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->a_log_scales, log_scales, 12 * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->a_quats, quats, 16 * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->a_opacity, opacity_logit, 4 * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->a_sh, sh, (size_t)K * 12 * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->c_means, means, 12 * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->c_quats, quats, 16 * n, cudaMemcpyDeviceToDevice, st));
  }
  ctx->n = n;
  ctx->sh_degree = sh_degree;
  ctx->frame_id = -1;
  return AIRGS_OK;
}

int airgs_apply_frame_update(airgs_ctx* ctx, const uint16_t* map, int map_w, int map_h, const float* lo,
                             const float* hi, int mode, int64_t frame_id) {
  if (!ctx) return AIRGS_E_ARG;
  if (ctx->sh_degree < 0) return fail(ctx, AIRGS_E_STATE, "set_anchor first");
  if (!map || !lo || !hi || map_w <= 0 || map_h <= 0) return fail(ctx, AIRGS_E_ARG, "bad update map arguments");
  if ((int64_t)map_w * map_h < ctx->n)
    return fail(ctx, AIRGS_E_ARG, "map has %lld pixels for %lld Gaussians", (long long)map_w * map_h,
                (long long)ctx->n);
  int base = mode & 1, quat_add = (mode & AIRGS_QUAT_ADD) ? 1 : 0;
  if (mode & ~3) return fail(ctx, AIRGS_E_ARG, "unknown mode bits");
  const float* bm = base == AIRGS_DELTA_ANCHOR ? ctx->a_means : ctx->c_means;
  const float* bq = base == AIRGS_DELTA_ANCHOR ? ctx->a_quats : ctx->c_quats;
  StageScope sc(ctx, ST_DECODE);
  CK(launch_decode_apply(ctx->stream, ctx->n, map, (int64_t)map_w * map_h, lo, hi, quat_add, bm, bq, ctx->c_means,
                         ctx->c_quats));
  ctx->frame_id = frame_id;
  return AIRGS_OK;
}

int airgs_get_frame_state(airgs_ctx* ctx, float* means_out, float* quats_out) {
  if (!ctx) return AIRGS_E_ARG;
  if (ctx->sh_degree < 0) return fail(ctx, AIRGS_E_STATE, "set_anchor first");
  if (ctx->n == 0) return AIRGS_OK;
  if (means_out) CK(cudaMemcpyAsync(means_out, ctx->c_means, 12 * ctx->n, cudaMemcpyDeviceToDevice, ctx->stream));
  if (quats_out) CK(cudaMemcpyAsync(quats_out, ctx->c_quats, 16 * ctx->n, cudaMemcpyDeviceToDevice, ctx->stream));
  return AIRGS_OK;
}

int airgs_render(airgs_ctx* ctx, const airgs_camera* cams, int n_views, float* rgb_out, float* T_out,
                 int32_t* n_contrib_out, float* importance_w, uint32_t* importance_cnt, airgs_state** saved) {
  if (!ctx) return AIRGS_E_ARG;
  if (ctx->sh_degree < 0) return fail(ctx, AIRGS_E_STATE, "set_anchor first");
  airgs_gaussians g = frame_gaussians(ctx);
  return render_impl(ctx, &g, cams, n_views, rgb_out, T_out, n_contrib_out, importance_w, importance_cnt, saved, -1);
}

int airgs_render_gaussians(airgs_ctx* ctx, const airgs_gaussians* g, const airgs_camera* cams, int n_views,
                           float* rgb_out, float* T_out, int32_t* n_contrib_out, float* importance_w,
                           uint32_t* importance_cnt, airgs_state** saved) {
  if (!ctx) return AIRGS_E_ARG;
  return render_impl(ctx, g, cams, n_views, rgb_out, T_out, n_contrib_out, importance_w, importance_cnt, saved, -1);
}

int airgs_render_backward(airgs_ctx* ctx, airgs_state* saved, const float* dL_drgb, float* g_means,
                          float* g_log_scales, float* g_quats, float* g_opacity_logit, float* g_sh,
                          float* importance_w, uint32_t* importance_cnt) {
  if (!ctx) return AIRGS_E_ARG;
  if (!dL_drgb) return fail(ctx, AIRGS_E_ARG, "dL_drgb is required");
  return backward_impl(ctx, saved, dL_drgb, nullptr, nullptr, g_means, g_log_scales, g_quats, g_opacity_logit, g_sh,
                       importance_w, importance_cnt);
}

int airgs_render_backward_l1(airgs_ctx* ctx, airgs_state* saved, const float* target, float* loss_out,
                             float* g_means, float* g_log_scales, float* g_quats, float* g_opacity_logit,
                             float* g_sh, float* importance_w, uint32_t* importance_cnt) {
  if (!ctx) return AIRGS_E_ARG;
  if (!target) return fail(ctx, AIRGS_E_ARG, "target is required");
  return backward_impl(ctx, saved, nullptr, target, loss_out, g_means, g_log_scales, g_quats, g_opacity_logit, g_sh,
                       importance_w, importance_cnt);
}

int airgs_render_backward_ex(airgs_ctx* ctx, airgs_state* saved, const airgs_backward_args* a) {
  if (!ctx) return AIRGS_E_ARG;
  if (!a) return fail(ctx, AIRGS_E_ARG, "null arguments");
  if (!a->dL_drgb && !a->target) return fail(ctx, AIRGS_E_ARG, "dL_drgb or target required");
  return backward_impl(ctx, saved, a->target ? nullptr : a->dL_drgb, a->target, a->loss_out, a->g_means,
                       a->g_log_scales, a->g_quats, a->g_opacity_logit, a->g_sh, a->importance_w, a->importance_cnt,
                       a->densify_grad, a->densify_views);
}

int airgs_densify_select(airgs_ctx* ctx, const float* densify_grad, const uint32_t* densify_views, int64_t n,
                         float threshold, uint8_t* mask_out) {
  if (!ctx) return AIRGS_E_ARG;
  if (n < 0 || (n > 0 && (!densify_grad || !densify_views || !mask_out)))
    return fail(ctx, AIRGS_E_ARG, "bad densify_select arguments");
  CK(launch_densify_select(ctx->stream, n, densify_grad, densify_views, threshold, mask_out));
  return AIRGS_OK;
}

int airgs_densify_apply(airgs_ctx* ctx, const airgs_gaussians* g, const uint8_t* select, const float* z,
                        float size_threshold, float split_factor, float min_opacity, const airgs_densify_out* out) {
  if (!ctx) return AIRGS_E_ARG;
  int rc = check_gaussians(ctx, g);
  if (rc) return rc;
  if (!out || !out->n_out) return fail(ctx, AIRGS_E_ARG, "out and out->n_out are required");
  if (!(size_threshold > 0.f) || !std::isfinite(size_threshold) || !(split_factor > 0.f) ||
      !std::isfinite(split_factor) || !(min_opacity >= 0.f && min_opacity < 1.f))
    return fail(ctx, AIRGS_E_ARG, "densify_apply: size_threshold > 0, split_factor > 0, 0 <= min_opacity < 1");
  const int64_t n = g->n;
  if (n > 0 && (!select || !z)) return fail(ctx, AIRGS_E_ARG, "densify_apply: select and z are required");
  if (out->capacity < 2 * n)
    return fail(ctx, AIRGS_E_CAPACITY, "densify_apply: capacity %lld below 2 n = %lld", (long long)out->capacity,
                (long long)(2 * n));
  if (n > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logit || !out->sh))
    return fail(ctx, AIRGS_E_ARG, "densify_apply: null output pointer");
  if (n > 0 && !aligned16(out->quats)) return fail(ctx, AIRGS_E_ARG, "densify_apply: out->quats must be 16-byte aligned");
  const float ls_thr = (float)std::log((double)size_threshold);
  const float ls_div = (float)std::log((double)split_factor);
  const float lo_thr =
      min_opacity > 0.f ? (float)std::log((double)min_opacity / (1.0 - (double)min_opacity)) : -INFINITY;
  uint8_t* cls = nullptr;
  uint3* tiles = nullptr;
  uint32_t* totals = nullptr;
  if (n > 0 && ((rc = dalloc(ctx, &cls, n)) || (rc = dalloc(ctx, &tiles, densify_tiles(n))) ||
                (rc = dalloc(ctx, &totals, 4)))) {
    for (void* p : {(void*)cls, (void*)tiles}) dfree(ctx, p);
    return rc;
  }
  cudaError_t e = launch_densify_apply(ctx->stream, n, g->sh_degree, g->means, g->log_scales, g->quats,
                                       g->opacity_logit, g->sh, select, z, ls_thr, ls_div, lo_thr, cls, tiles, totals,
                                       out->means, out->log_scales, out->quats, out->opacity_logit, out->sh,
                                       out->parent, out->n_out);
  for (void* p : {(void*)cls, (void*)tiles, (void*)totals}) dfree(ctx, p);
  if (e != cudaSuccess) return fail(ctx, AIRGS_E_CUDA, "densify_apply: %s", cudaGetErrorString(e));
  return AIRGS_OK;
}

int airgs_gaussian_importance(airgs_ctx* ctx, const airgs_camera* cams, int n_views, float* w_out,
                              uint32_t* cnt_out) {
  if (!ctx) return AIRGS_E_ARG;
  if (ctx->sh_degree < 0) return fail(ctx, AIRGS_E_STATE, "set_anchor first");
  if (!w_out || !cnt_out) return fail(ctx, AIRGS_E_ARG, "w_out and cnt_out are required");
  std::vector<CamDev> tmp;
  int64_t nt = 0, np = 0;
  int rc = build_cams(ctx, cams, n_views, tmp, nt, np);
  if (rc) return rc;
  if (ctx->n > 0) {
    CK(cudaMemsetAsync(w_out, 0, 4 * ctx->n, ctx->stream));
    CK(cudaMemsetAsync(cnt_out, 0, 4 * ctx->n, ctx->stream));
  }
  float* rgb = nullptr;
  rc = dalloc(ctx, &rgb, 3 * np);
  if (rc) return rc;
  airgs_gaussians g = frame_gaussians(ctx);
  rc = render_impl(ctx, &g, cams, n_views, rgb, nullptr, nullptr, w_out, cnt_out, nullptr, -1);
  dfree(ctx, rgb);
  return rc;
}

int airgs_release_state(airgs_ctx* ctx, airgs_state* state) {
  if (!ctx) return AIRGS_E_ARG;
  release_state(ctx, state);
  return AIRGS_OK;
}

int airgs_state_stats(airgs_ctx* ctx, const airgs_state* s, airgs_stats* out) {
  if (!ctx || !s || !out) return AIRGS_E_ARG;
  CK(cudaMemcpyAsync(ctx->h_pinned, s->counters, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  out->n_instances = s->n_inst >= 0 ? s->n_inst : (int64_t)ctx->h_pinned[4];
  out->n_tiles = s->n_tiles;
  out->n_pixels = s->n_pixels;
  out->pairs_forward = (int64_t)ctx->h_pinned[0];
  out->pairs_backward = (int64_t)ctx->h_pinned[2];
  out->kernel_shape = s->shape;
  return AIRGS_OK;
}

int airgs_state_view_info(airgs_ctx* ctx, const airgs_state* s, int view, int64_t* n_tiles, int64_t* n_entries) {
  if (!ctx || !s || view < 0 || view >= s->n_views) return AIRGS_E_ARG;
  const CamDev& c = s->h_cams[view];
  int64_t nt = (int64_t)c.TW * c.TH;
  if (n_tiles) *n_tiles = nt;
  if (n_entries) {
    std::vector<uint2> r(nt);
    CK(cudaMemcpyAsync(r.data(), s->ranges + c.tile_base, nt * sizeof(uint2), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    int64_t cnt = 0;
    for (auto& x : r) cnt += (int64_t)x.y - x.x;
    *n_entries = cnt;
  }
  return AIRGS_OK;
}

int airgs_state_projection(airgs_ctx* ctx, const airgs_state* s, int view, float* mean2d, float* depth,
                           int32_t* radius) {
  if (!ctx || !s || view < 0 || view >= s->n_views) return AIRGS_E_ARG;
  if (s->n == 0) return AIRGS_OK;
  k_extract_projection<<<(unsigned)((s->n + 255) / 256), 256, 0, ctx->stream>>>(s->proj + (size_t)view * s->n, s->n,
                                                                                  mean2d, depth, radius);
  CK(cudaGetLastError());
  return AIRGS_OK;
}

int airgs_state_tile_lists(airgs_ctx* ctx, const airgs_state* s, int view, int64_t* ranges, int32_t* ids) {
  if (!ctx || !s || view < 0 || view >= s->n_views) return AIRGS_E_ARG;
  const CamDev& c = s->h_cams[view];
  int64_t nt = (int64_t)c.TW * c.TH;
  std::vector<uint2> r(nt);
  CK(cudaMemcpyAsync(r.data(), s->ranges + c.tile_base, nt * sizeof(uint2), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  // the view's entries are contiguous (tile ids are view-major)
  int64_t first = -1;
  for (auto& x : r)
    if (x.y > x.x) {
      first = x.x;
      break;
    }
  std::vector<int64_t> rel(2 * nt, 0);
  int64_t total = 0;
  for (int64_t t = 0; t < nt; ++t) {
    if (r[t].y > r[t].x) {
      rel[2 * t] = (int64_t)r[t].x - first;
      rel[2 * t + 1] = (int64_t)r[t].y - first;
      total = std::max(total, rel[2 * t + 1]);
    } else {
      rel[2 * t] = rel[2 * t + 1] = total;  // empty tile: an empty range at the current end
    }
  }
  if (ranges) {
    CK(cudaMemcpyAsync(ranges, rel.data(), rel.size() * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
  }
  if (ids && total > 0)
    CK(cudaMemcpyAsync(ids, s->ids + first, total * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return AIRGS_OK;
}

int airgs_sort_pairs(airgs_ctx* ctx, const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                     uint32_t* vals_out, int64_t n, int key_bits) {
  if (!ctx) return AIRGS_E_ARG;
  if (n < 0 || n >= (1ll << 32) || key_bits < 1 || key_bits > 32 || !keys_in || !vals_in || !keys_out || !vals_out)
    return fail(ctx, AIRGS_E_ARG, "bad sort arguments");
  if (n == 0) return AIRGS_OK;
  cudaStream_t st = ctx->stream;
  uint32_t *ka = nullptr, *va = nullptr, *kb = nullptr, *vb = nullptr, *scr = nullptr;
  int rc;
  if ((rc = dalloc(ctx, &ka, n)) || (rc = dalloc(ctx, &va, n)) || (rc = dalloc(ctx, &kb, n)) ||
      (rc = dalloc(ctx, &vb, n)) ||
      (rc = dalloc(ctx, &scr, radix_scratch_bytes(n, 1, ctx->num_sms) / sizeof(uint32_t) + 1))) {
    for (void* p : {(void*)ka, (void*)va, (void*)kb, (void*)vb}) dfree(ctx, p);
    return rc;
  }
  bool in_b = false;
  cudaError_t e = cudaMemcpyAsync(ka, keys_in, 4 * n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(va, vals_in, 4 * n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = radix_sort_pairs(st, ctx->num_sms, ka, va, kb, vb, n, 1, key_bits, false, scr, &in_b);
  if (e == cudaSuccess) e = cudaMemcpyAsync(keys_out, in_b ? kb : ka, 4 * n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vals_out, in_b ? vb : va, 4 * n, cudaMemcpyDeviceToDevice, st);
  for (void* p : {(void*)ka, (void*)va, (void*)kb, (void*)vb, (void*)scr}) dfree(ctx, p);
  if (e != cudaSuccess) return fail(ctx, AIRGS_E_CUDA, "sort: %s", cudaGetErrorString(e));
  return AIRGS_OK;
}

int airgs_autotune(airgs_ctx* ctx, const airgs_camera* cams, int n_views, int* shape, float* ms_default,
                   float* ms_best) {
  if (!ctx) return AIRGS_E_ARG;
  if (ctx->sh_degree < 0) return fail(ctx, AIRGS_E_STATE, "set_anchor first");
  std::vector<CamDev> tmp;
  int64_t nt = 0, np = 0;
  int rc = build_cams(ctx, cams, n_views, tmp, nt, np);
  if (rc) return rc;
  airgs_gaussians g = frame_gaussians(ctx);
  const int K = (ctx->sh_degree + 1) * (ctx->sh_degree + 1);
  const int64_t n = std::max<int64_t>(ctx->n, 1);
  // the buffers of a training step: image, a constant target, parameter gradients, usage frequency, loss
  float *rgb = nullptr, *target = nullptr, *gm = nullptr, *gl = nullptr, *gq = nullptr, *go = nullptr,
        *gs = nullptr, *impw = nullptr, *loss = nullptr;
  uint32_t* impc = nullptr;
  struct Free {
    airgs_ctx* c;
    std::vector<void*> p;
    ~Free() {
      for (void* q : p) dfree(c, q);
    }
  } fr{ctx, {}};
  const bool oom = (rc = dalloc(ctx, &rgb, 3 * np)) || (rc = dalloc(ctx, &target, 3 * np)) ||
                  (rc = dalloc(ctx, &gm, 3 * n)) || (rc = dalloc(ctx, &gl, 3 * n)) || (rc = dalloc(ctx, &gq, 4 * n)) ||
                  (rc = dalloc(ctx, &go, n)) || (rc = dalloc(ctx, &gs, (size_t)K * 3 * n)) ||
                  (rc = dalloc(ctx, &impw, n)) || (rc = dalloc(ctx, &impc, n)) || (rc = dalloc(ctx, &loss, 1));
  fr.p = {rgb, target, gm, gl, gq, go, gs, impw, impc, loss};  // the ones allocated return to the pool on any exit
  if (oom) return rc;
  CK(cudaMemsetAsync(target, 0x3F, 12 * np, ctx->stream));  // every channel 0x3F3F3F3F = 0.747
  CK(cudaMemsetAsync(impw, 0, 4 * n, ctx->stream));
  CK(cudaMemsetAsync(impc, 0, 4 * n, ctx->stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // one training step with the given shape: best of 3 timed repetitions after a warm-up
  auto time_shape = [&](int shp, float& ms) -> int {
    ms = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      airgs_state* s = nullptr;
      cudaEventRecord(e0, ctx->stream);
      int r = render_impl(ctx, &g, cams, n_views, rgb, nullptr, nullptr, nullptr, nullptr, &s, shp);
      if (r == AIRGS_OK) r = backward_impl(ctx, s, nullptr, target, loss, gm, gl, gq, go, gs, impw, impc);
      cudaEventRecord(e1, ctx->stream);
      const cudaError_t e = cudaEventSynchronize(e1);
      release_state(ctx, s);
      if (r != AIRGS_OK) return r;
      if (e != cudaSuccess) return fail(ctx, AIRGS_E_CUDA, "autotune: %s", cudaGetErrorString(e));
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) ms = std::min(ms, t);
    }
    return AIRGS_OK;
  };
  // coordinate search from shape 0: the backward's shapes, then the forward's,
  // then the sort's keys per thread, then the emission's run length, each with
  // the other parts at the best so far
  ShapeParts best{0, 0, 0, 0};
  float best_ms = 0.f, def_ms = 0.f;
  rc = time_shape(0, def_ms);
  best_ms = def_ms;
  for (int axis = 0; axis < 4 && rc == AIRGS_OK; ++axis) {
    const int count = axis == 0 ? kBwdShapes : axis == 1 ? kFwdShapes : axis == 2 ? kSortShapes : kEmitShapes;
    const ShapeParts base = best;
    for (int c = 0; c < count && rc == AIRGS_OK; ++c) {
      ShapeParts p = base;
      int& slot = axis == 0 ? p.bwd : axis == 1 ? p.fwd : axis == 2 ? p.sort : p.emit;
      if (slot == c) continue;  // already timed
      slot = c;
      float ms = 0.f;
      rc = time_shape(shape_index(p.fwd, p.bwd, p.sort, p.emit), ms);
      if (rc == AIRGS_OK && ms < best_ms) {
        best_ms = ms;
        best = p;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const int chosen = shape_index(best.fwd, best.bwd, best.sort, best.emit);
  ctx->tuned[tune_key(ctx->n, np, n_views)] = chosen;
  save_tune_cache(ctx);
  if (shape) *shape = chosen;
  if (ms_default) *ms_default = def_ms;
  if (ms_best) *ms_best = best_ms;
  return AIRGS_OK;
}

int airgs_prune_mask(airgs_ctx* ctx, const float* importance, int64_t n, int64_t n_prune, uint8_t* keep_out) {
  if (!ctx) return AIRGS_E_ARG;
  if (n < 0 || n >= (1ll << 32) || n_prune < 0 || n_prune > n || (n > 0 && (!importance || !keep_out)))
    return fail(ctx, AIRGS_E_ARG, "bad prune_mask arguments");
  if (n == 0) return AIRGS_OK;
  uint32_t *ka = nullptr, *va = nullptr, *kb = nullptr, *vb = nullptr, *scr = nullptr;
  int rc;
  if ((rc = dalloc(ctx, &ka, n)) || (rc = dalloc(ctx, &va, n)) || (rc = dalloc(ctx, &kb, n)) ||
      (rc = dalloc(ctx, &vb, n)) ||
      (rc = dalloc(ctx, &scr, radix_scratch_bytes(n, 1, ctx->num_sms) / sizeof(uint32_t) + 1))) {
    for (void* p : {(void*)ka, (void*)va, (void*)kb, (void*)vb}) dfree(ctx, p);
    return rc;
  }
  cudaError_t e = launch_prune_mask(ctx->stream, ctx->num_sms, n, n_prune, importance, ka, va, kb, vb, scr, keep_out);
  for (void* p : {(void*)ka, (void*)va, (void*)kb, (void*)vb, (void*)scr}) dfree(ctx, p);
  if (e != cudaSuccess) return fail(ctx, AIRGS_E_CUDA, "prune_mask: %s", cudaGetErrorString(e));
  return AIRGS_OK;
}

int airgs_prune_delta(airgs_ctx* ctx, int64_t n, int channels, const float* D_t, float* D_sent, const uint8_t* keep,
                      float* d_out, uint64_t* nonzero_out) {
  if (!ctx) return AIRGS_E_ARG;
  if (n < 0 || channels < 1 || channels > 64 || (n > 0 && (!D_t || !D_sent || !keep || !d_out)))
    return fail(ctx, AIRGS_E_ARG, "bad prune_delta arguments");
  if (nonzero_out) CK(cudaMemsetAsync(nonzero_out, 0, sizeof(uint64_t), ctx->stream));
  CK(launch_prune_delta(ctx->stream, n, channels, D_t, D_sent, keep, d_out, (unsigned long long*)nonzero_out));
  return AIRGS_OK;
}

int airgs_apply_frame_delta(airgs_ctx* ctx, const float* delta, int mode, int64_t frame_id) {
  if (!ctx) return AIRGS_E_ARG;
  if (ctx->sh_degree < 0) return fail(ctx, AIRGS_E_STATE, "set_anchor first");
  if (!delta && ctx->n > 0) return fail(ctx, AIRGS_E_ARG, "null delta");
  if (mode & ~3) return fail(ctx, AIRGS_E_ARG, "unknown mode bits");
  const int base = mode & 1, quat_add = (mode & AIRGS_QUAT_ADD) ? 1 : 0;
  const float* bm = base == AIRGS_DELTA_ANCHOR ? ctx->a_means : ctx->c_means;
  const float* bq = base == AIRGS_DELTA_ANCHOR ? ctx->a_quats : ctx->c_quats;
  StageScope sc(ctx, ST_DECODE);
  CK(launch_apply_delta(ctx->stream, ctx->n, delta, quat_add, bm, bq, ctx->c_means, ctx->c_quats));
  ctx->frame_id = frame_id;
  return AIRGS_OK;
}

int airgs_image_sse(airgs_ctx* ctx, const airgs_camera* cams, int n_views, const float* a, const float* b,
                    double* sse_out) {
  if (!ctx) return AIRGS_E_ARG;
  std::vector<CamDev> tmp;
  int64_t nt = 0, np = 0;
  int rc = build_cams(ctx, cams, n_views, tmp, nt, np);
  if (rc) return rc;
  if (!a || !b || !sse_out) return fail(ctx, AIRGS_E_ARG, "null image pointer");
  std::vector<int64_t> off(n_views + 1, 0);
  for (int v = 0; v < n_views; ++v) off[v + 1] = off[v] + 3 * (int64_t)tmp[v].W * tmp[v].H;
  int64_t* d_off = nullptr;
  if ((rc = dalloc(ctx, &d_off, n_views + 1))) return rc;
  cudaError_t e = cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sse_out, 0, n_views * sizeof(double), ctx->stream);
  if (e == cudaSuccess) e = launch_sq_err(ctx->stream, a, b, d_off, n_views, sse_out);
  // the offsets are read by the kernel before the stream-ordered free
  dfree(ctx, d_off);
  if (e != cudaSuccess) return fail(ctx, AIRGS_E_CUDA, "image_sse: %s", cudaGetErrorString(e));
  return AIRGS_OK;
}

int airgs_l3dgs_loss(airgs_ctx* ctx, const airgs_camera* cams, int n_views, const float* rgb, const float* target,
                     float lambda, double* loss_out, float* dL_drgb_out) {
  if (!ctx) return AIRGS_E_ARG;
  std::vector<CamDev> tmp;
  int64_t nt = 0, np = 0;
  int rc = build_cams(ctx, cams, n_views, tmp, nt, np);
  if (rc) return rc;
  if (!rgb || !target || !dL_drgb_out) return fail(ctx, AIRGS_E_ARG, "null image pointer");
  if (!(lambda >= 0.f && lambda <= 1.f)) return fail(ctx, AIRGS_E_ARG, "lambda must be in [0, 1]");
  const int n_planes = 3 * n_views;
  std::vector<int64_t> off(n_planes + 1, 0), tile_base(n_planes + 1, 0);
  std::vector<int> w(n_planes), h(n_planes);
  for (int v = 0; v < n_views; ++v)
    for (int c = 0; c < 3; ++c) {
      const int p = 3 * v + c;
      w[p] = tmp[v].W;
      h[p] = tmp[v].H;
      off[p + 1] = off[p] + (int64_t)tmp[v].W * tmp[v].H;
      tile_base[p + 1] = tile_base[p] + ssim_tiles(tmp[v].W, tmp[v].H);
    }
  const int64_t total = off[n_planes];
  int64_t *d_off = nullptr, *d_tb = nullptr;
  int *d_w = nullptr, *d_h = nullptr;
  double* sums = nullptr;
  if ((rc = dalloc(ctx, &d_off, n_planes + 1)) || (rc = dalloc(ctx, &d_tb, n_planes + 1)) ||
      (rc = dalloc(ctx, &d_w, n_planes)) || (rc = dalloc(ctx, &d_h, n_planes)) || (rc = dalloc(ctx, &sums, 5))) {
    for (void* p : {(void*)d_off, (void*)d_tb, (void*)d_w, (void*)d_h, (void*)sums}) dfree(ctx, p);
    return rc;
  }
  cudaStream_t st = ctx->stream;
  // pageable sources: each copy returns once its bytes are staged, so the host arrays may go after the calls
  cudaError_t e = cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tb, tile_base.data(), tile_base.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, w.data(), w.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_h, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, 5 * sizeof(double), st);
  if (e == cudaSuccess)
    e = launch_ssim_loss(st, d_off, d_w, d_h, d_tb, n_planes, total, tile_base[n_planes], rgb, target, lambda, sums,
                         dL_drgb_out);
  if (e == cudaSuccess && loss_out)
    e = cudaMemcpyAsync(loss_out, sums + 2, 3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  // device temporaries return to the pool in stream order
  for (void* p : {(void*)d_off, (void*)d_tb, (void*)d_w, (void*)d_h, (void*)sums}) dfree(ctx, p);
  if (e != cudaSuccess) return fail(ctx, AIRGS_E_CUDA, "l3dgs_loss: %s", cudaGetErrorString(e));
  return AIRGS_OK;
}

int airgs_set_profiling(airgs_ctx* ctx, int enabled) {
  if (!ctx) return AIRGS_E_ARG;
  if (enabled != AIRGS_PROFILE_OFF && enabled != AIRGS_PROFILE_ALL && enabled != AIRGS_PROFILE_BLEND)
    return fail(ctx, AIRGS_E_ARG, "profiling level %d: expected 0 (off), 1 (every stage) or 2 (blend stages)",
                enabled);
  if (enabled && !ctx->d_pair_total) {
    int rc = dalloc(ctx, &ctx->d_pair_total, 4);
    if (rc) return rc;
    CK(cudaMemsetAsync(ctx->d_pair_total, 0, 4 * sizeof(unsigned long long), ctx->stream));
  }
  ctx->profiling = enabled;
  return AIRGS_OK;
}

int airgs_stage_times(airgs_ctx* ctx, double* ms, int64_t* launches, int64_t* pairs) {
  if (!ctx) return AIRGS_E_ARG;
  if (pairs) {
    pairs[0] = pairs[1] = pairs[2] = pairs[3] = 0;
    if (ctx->d_pair_total) {
      CK(cudaMemcpyAsync(ctx->h_pinned + 2, ctx->d_pair_total, 4 * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                         ctx->stream));
      CK(cudaMemsetAsync(ctx->d_pair_total, 0, 4 * sizeof(unsigned long long), ctx->stream));
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (pairs && ctx->d_pair_total)
    for (int k = 0; k < 4; ++k) pairs[k] = (int64_t)ctx->h_pinned[2 + k];
  for (int k = 0; k < ST_COUNT; ++k) {
    if (ms) ms[k] = 0.0;
    if (launches) launches[k] = 0;
  }
  for (auto& p : ctx->pending) {
    float t = 0.f;
    cudaEventElapsedTime(&t, p.second.first, p.second.second);
    if (ms) ms[p.first] += t;
    if (launches) launches[p.first] += 1;
    ctx->event_pool.push_back(p.second.first);
    ctx->event_pool.push_back(p.second.second);
  }
  ctx->pending.clear();
  return AIRGS_OK;
}

const char* airgs_stage_name(int stage) { return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : ""; }

int airgs_measure_fp32_peak(airgs_ctx* ctx, double* tflops) {
  if (!ctx || !tflops) return AIRGS_E_ARG;
  float* scratch = nullptr;
  int rc = dalloc(ctx, &scratch, fp32_probe_words(ctx->num_sms));
  if (rc) return rc;
  const cudaError_t e = measure_fp32_peak(ctx->stream, ctx->num_sms, scratch, tflops);
  dfree(ctx, scratch);
  if (e != cudaSuccess) return fail(ctx, AIRGS_E_CUDA, "fp32 probe: %s", cudaGetErrorString(e));
  return AIRGS_OK;
}

int airgs_measure_smem_peak(airgs_ctx* ctx, double* tbs) {
  if (!ctx || !tbs) return AIRGS_E_ARG;
  float* scratch = nullptr;
  int rc = dalloc(ctx, &scratch, smem_probe_words(ctx->num_sms));
  if (rc) return rc;
  const cudaError_t e = measure_smem_peak(ctx->stream, ctx->num_sms, scratch, tbs);
  dfree(ctx, scratch);
  if (e != cudaSuccess) return fail(ctx, AIRGS_E_CUDA, "shared-memory probe: %s", cudaGetErrorString(e));
  return AIRGS_OK;
}

int64_t airgs_kernel_launch_count(void) { return g_launches.load(); }

int airgs_shape_count(void) { return kShapes; }
const char* airgs_shape_name(int shape) { return shape_name(shape); }

}  // extern "C"
