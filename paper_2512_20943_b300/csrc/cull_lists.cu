// Half-tile blend lists (sm_103a).
//
// When an instance is emitted it is tested once against the two 16x8 halves of
// its tile: the Gaussian's alpha >= alpha_min box (the same conservative box the
// blend kernels use per 8x4 block) either meets a half or cannot blend anywhere
// in it; the two flags ride in the key's top bits through the tile sort.  Each half gets its own compacted list of
// (Gaussian id, position in the tile's full list) in the full list's order, so
// the half-tile blend kernels stage only entries that can matter while still
// reporting and replaying positions of the definition's list.
#include "airgs_internal.cuh"
#include "kernels.h"
#include "launch.cuh"

namespace airgs {

#ifndef AIRGS_HL_THREADS
#define AIRGS_HL_THREADS 256  // measured best of 256, 512, 1024
#endif
constexpr int HL_THREADS = AIRGS_HL_THREADS;
constexpr int HL_ITEMS = 4;
constexpr int HL_CHUNK = HL_THREADS * HL_ITEMS;

size_t half_list_chunks(int64_t n_inst) { return (size_t)((n_inst + HL_CHUNK - 1) / HL_CHUNK); }

struct HalfArgs {
  const uint32_t* keys;  // sorted tile ids
  const uint32_t* ids;   // sorted Gaussian ids
  const uint2* ranges;   // full tile ranges (k_half_sums writes them, k_half_compact reads them)
  uint2* ranges_out;
  const CamDev* cams;
  int n_views;
  const ProjRec* proj;
  int64_t n;
  int64_t n_inst;
  float log2_amin;
};

// Also writes each tile's [start, end) in the sorted list (the tile-ranges
// pass): consecutive threads hold consecutive entries, so the neighbouring keys
// come by shuffle (the warp's end lanes load theirs).
__global__ void __launch_bounds__(HL_THREADS) k_half_sums(HalfArgs h, uint8_t* __restrict__ flags,
                                                          uint64_t* __restrict__ sums_top,
                                                          uint64_t* __restrict__ sums_bot) {
  wait_prior_grid();
  __shared__ uint32_t s_t[HL_THREADS / 32], s_b[HL_THREADS / 32];
  const int64_t c0 = (int64_t)blockIdx.x * HL_CHUNK;
  const int lane = threadIdx.x & 31;
  uint32_t nt = 0, nb = 0;
  uint32_t key[HL_ITEMS];
#pragma unroll
  for (int k = 0; k < HL_ITEMS; ++k) {
    const int64_t p = c0 + k * HL_THREADS + threadIdx.x;
    key[k] = p < h.n_inst ? h.keys[p] : 0u;
  }
#pragma unroll
  for (int k = 0; k < HL_ITEMS; ++k) {
    const int64_t p = c0 + k * HL_THREADS + threadIdx.x;
    const uint32_t tile = key[k] & kKeyTileMask;
    uint32_t prev = __shfl_up_sync(0xffffffffu, tile, 1), next = __shfl_down_sync(0xffffffffu, tile, 1);
    if (p < h.n_inst) {
      if (lane == 0 && p > 0) prev = h.keys[p - 1] & kKeyTileMask;
      if (lane == 31 && p + 1 < h.n_inst) next = h.keys[p + 1] & kKeyTileMask;
      if (p == 0 || prev != tile) h.ranges_out[tile].x = (uint32_t)p;
      if (p + 1 == h.n_inst || next != tile) h.ranges_out[tile].y = (uint32_t)(p + 1);
      const unsigned f = key[k] >> kKeyHalfShift;
      flags[p] = (uint8_t)f;
      nt += f & 1u;
      nb += f >> 1;
    }
  }
  nt = __reduce_add_sync(0xffffffffu, nt);
  nb = __reduce_add_sync(0xffffffffu, nb);
  if ((threadIdx.x & 31) == 0) {
    s_t[threadIdx.x >> 5] = nt;
    s_b[threadIdx.x >> 5] = nb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t a = 0, b = 0;
    for (int w = 0; w < HL_THREADS / 32; ++w) {
      a += s_t[w];
      b += s_b[w];
    }
    sums_top[blockIdx.x] = a;
    sums_bot[blockIdx.x] = b;
  }
}

// Exclusive block scan of two counters (blocked: thread t owns HL_ITEMS consecutive entries).
__global__ void __launch_bounds__(HL_THREADS) k_half_compact(HalfArgs h, const uint8_t* __restrict__ flags,
                                                             const uint64_t* __restrict__ off_top,
                                                             const uint64_t* __restrict__ off_bot,
                                                             uint64_t bot_base, uint2* __restrict__ hl,
                                                             uint2* __restrict__ hranges, int64_t n_tiles) {
  wait_prior_grid();
  __shared__ uint32_t s_t[HL_THREADS / 32], s_b[HL_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t p0 = (int64_t)blockIdx.x * HL_CHUNK + (int64_t)tid * HL_ITEMS;
  // every global load this thread needs is issued before the scan, so that
  // their latencies overlap it (the ranges wait only for the keys)
  const uint64_t cta_top = off_top[blockIdx.x], cta_bot = off_bot[blockIdx.x];
  uint32_t tiles[HL_ITEMS], gids[HL_ITEMS];
  uint2 rgs[HL_ITEMS];
#pragma unroll
  for (int k = 0; k < HL_ITEMS; ++k) {
    const int64_t p = p0 + k;
    tiles[k] = p < h.n_inst ? h.keys[p] & kKeyTileMask : 0u;
    gids[k] = p < h.n_inst ? h.ids[p] : 0u;
  }
#pragma unroll
  for (int k = 0; k < HL_ITEMS; ++k) rgs[k] = p0 + k < h.n_inst ? h.ranges[tiles[k]] : make_uint2(0u, 0u);
  unsigned f[HL_ITEMS];
  uint32_t lt = 0, lb = 0;
#pragma unroll
  for (int k = 0; k < HL_ITEMS; ++k) {
    f[k] = (p0 + k < h.n_inst) ? flags[p0 + k] : 0u;
    lt += f[k] & 1u;
    lb += f[k] >> 1;
  }
  uint32_t xt = lt, xb = lb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t yt = __shfl_up_sync(0xffffffffu, xt, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
    if (lane >= o) {
      xt += yt;
      xb += yb;
    }
  }
  if (lane == 31) {
    s_t[warp] = xt;
    s_b[warp] = xb;
  }
  __syncthreads();
  uint32_t wt = 0, wb = 0;
  for (int w = 0; w < warp; ++w) {
    wt += s_t[w];
    wb += s_b[w];
  }
  uint64_t ot = cta_top + wt + xt - lt;
  uint64_t ob = bot_base + cta_bot + wb + xb - lb;
#pragma unroll
  for (int k = 0; k < HL_ITEMS; ++k) {
    const int64_t p = p0 + k;
    if (p >= h.n_inst) break;
    const uint32_t tile = tiles[k];
    const uint32_t start = rgs[k].x;
    const uint32_t pos = (uint32_t)(p - start);
    const bool first = p == start, last = p + 1 == rgs[k].y;
    const uint32_t gid = gids[k];
    if (first) {
      hranges[tile].x = (uint32_t)ot;
      hranges[n_tiles + tile].x = (uint32_t)ob;
    }
    if (f[k] & 1u) hl[ot++] = make_uint2(gid, pos);
    if (f[k] & 2u) hl[ob++] = make_uint2(gid, pos);
    if (last) {
      hranges[tile].y = (uint32_t)ot;
      hranges[n_tiles + tile].y = (uint32_t)ob;
    }
  }
}

cudaError_t launch_half_lists(cudaStream_t st, const uint32_t* keys, const uint32_t* ids, uint2* ranges,
                              const CamDev* cams, int n_views, const ProjRec* proj, int64_t n, int64_t n_inst,
                              float alpha_min, int64_t n_tiles, uint8_t* flags, uint64_t* sums, uint2* hl,
                              uint2* hranges) {
  if (n_inst == 0) return cudaSuccess;
  const int64_t chunks = (int64_t)half_list_chunks(n_inst);
  HalfArgs h{keys, ids, ranges, ranges, cams, n_views, proj, n, n_inst, log2f(alpha_min)};
  uint64_t* st_ = sums;               // [chunks + 1] top
  uint64_t* sb_ = sums + chunks + 1;  // [chunks + 1] bottom
  cudaError_t e = launch_serialised(k_half_sums, dim3((unsigned)chunks), dim3(HL_THREADS), 0, st, h, flags, st_, sb_);
  if (e == cudaSuccess) e = launch_scan_spans(st, st_, chunks, st_ + chunks, sb_, sb_ + chunks);
  if (e != cudaSuccess) return e;
  e = launch_serialised(k_half_compact, dim3((unsigned)chunks), dim3(HL_THREADS), 0, st, h, (const uint8_t*)flags,
                        (const uint64_t*)st_, (const uint64_t*)sb_, (uint64_t)n_inst, hl, hranges, n_tiles);
  count_launches(2);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// ---------------------------------------------------------------- work order
// The blend kernels take their (half tile) items from an atomic queue, one warp
// per item.  Item costs vary several-fold (the half-list length), and with the
// queue in tile order a long item taken near the end keeps its SM busy while
// the others idle.  The order below hands out the items of each group of
// consecutive views (work indices are view-major) longest list first (in bins
// of a quarter octave): every group, the last one included, ends on short items,
// and the items in flight together come from one group, whose Gaussian
// records stay in L2.  The last group may hold more views than the others (it
// alone decides the kernel's end, so it needs enough items per warp).

// Bin of a half-list length L: 0 for an empty list, else 1 + 4 floor(log2 L)
// + the two bits below the leading one (quarter octaves: 0.17 % faster blend
// kernels than half octaves on the streaming step).
__device__ __forceinline__ int order_bin(uint32_t L) {
  if (L == 0u) return 0;
  const int msb = 31 - __clz(L);
  const int sub = msb > 1 ? (int)((L >> (msb - 2)) & 3u) : (msb == 1 ? (int)((L & 1u) << 1) : 0);
  return min(1 + 4 * msb + sub, kOrderBins - 1);
}

struct OrderArgs {
  const uint2* hranges;  // [2][tiles]
  const CamDev* cams;
  int n_views;
  int views_per_group;
  int n_groups;
  int64_t n_tiles;
};

// Group-major bin index of work item w (group g, bin b: g kOrderBins + b).
__device__ __forceinline__ int order_key(const OrderArgs& o, int64_t w) {
  const int64_t tile = w >> 1;
  const uint2 r = o.hranges[(w & 1) * o.n_tiles + tile];
  int lo = 0, hi = o.n_views - 1;  // the view owning the tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int64_t)__ldg(&o.cams[mid].tile_base) <= tile) lo = mid;
    else hi = mid - 1;
  }
  const int g = min(lo / o.views_per_group, o.n_groups - 1);
  return g * kOrderBins + order_bin(r.y - r.x);
}

// Adds one to counter[key] for every lane of the warp (one atomic per distinct
// key, of the number of lanes holding it); returns the lane's rank among them
// plus the counter's previous value.  Lanes with key < 0 take no part.
__device__ __forceinline__ uint32_t warp_count(uint32_t* counter, int key, bool want_rank) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(peers) - 1;
  uint32_t first = 0u;
  if (lane == leader && key >= 0) first = atomicAdd(&counter[key], (uint32_t)__popc(peers));
  if (!want_rank) return 0u;
  first = __shfl_sync(0xffffffffu, first, leader);
  return first + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(256) k_order_hist(OrderArgs o, uint32_t* __restrict__ hist) {
  wait_prior_grid();
  const int64_t n_work = 2 * o.n_tiles, stride = (int64_t)gridDim.x * blockDim.x;
  // every lane of a warp runs the same iterations (the warp votes take all lanes)
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < n_work; w0 += stride) {
    const int64_t w = w0 + (threadIdx.x & 31);
    warp_count(hist, w < n_work ? order_key(o, w) : -1, false);
  }
}

// base[g][b]: the group's first work index plus the items of its bins above b.
__global__ void __launch_bounds__(32) k_order_base(OrderArgs o, const uint32_t* __restrict__ hist,
                                                   uint32_t* __restrict__ base) {
  wait_prior_grid();
  static_assert(kOrderBins == 64, "two bins per lane");
  const int g = blockIdx.x, lane = threadIdx.x;
  const uint32_t* h = hist + (size_t)g * kOrderBins;
  const uint32_t h0 = h[2 * lane], h1 = h[2 * lane + 1];
  uint32_t x = h0 + h1;  // inclusive suffix sum over lanes >= this one
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_down_sync(0xffffffffu, x, off);
    if (lane + off < 32) x += y;
  }
  const uint32_t start = 2u * __ldg(&o.cams[g * o.views_per_group].tile_base);
  base[(size_t)g * kOrderBins + 2 * lane + 1] = start + x - h0 - h1;
  base[(size_t)g * kOrderBins + 2 * lane] = start + x - h0;
}

__global__ void __launch_bounds__(256) k_order_scatter(OrderArgs o, const uint32_t* __restrict__ base,
                                                       uint32_t* __restrict__ cursor, uint32_t* __restrict__ order) {
  wait_prior_grid();
  const int64_t n_work = 2 * o.n_tiles, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < n_work; w0 += stride) {
    const int64_t w = w0 + (threadIdx.x & 31);
    const int key = w < n_work ? order_key(o, w) : -1;
    const uint32_t rank = warp_count(cursor, key, true);
    if (key >= 0) order[base[key] + rank] = (uint32_t)w;
  }
}

size_t item_order_words(int n_views) { return (size_t)3 * kOrderBins * (n_views > 0 ? n_views : 1); }

cudaError_t launch_item_order(cudaStream_t st, int num_sms, const uint2* hranges, const CamDev* cams, int n_views,
                              int views_per_group, int last_views, int64_t n_tiles, uint32_t* scratch,
                              uint32_t* order) {
  if (n_tiles <= 0 || n_views <= 0) return cudaSuccess;
  if (views_per_group < 1) views_per_group = 1;
  if (views_per_group > n_views) views_per_group = n_views;
  if (last_views < views_per_group) last_views = views_per_group;
  if (last_views > n_views) last_views = n_views;
  // groups of views_per_group views before the last one, which takes the rest
  // (at least last_views views)
  OrderArgs o{hranges, cams, n_views, views_per_group, (n_views - last_views) / views_per_group + 1, n_tiles};
  const size_t words = (size_t)o.n_groups * kOrderBins;
  uint32_t *hist = scratch, *cursor = scratch + words, *base = scratch + 2 * words;
  cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * words * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (2 * n_tiles + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 2 * (int64_t)num_sms ? blocks : 2 * (int64_t)num_sms);
  e = launch_serialised(k_order_hist, dim3(grid), dim3(256), 0, st, o, hist);
  if (e == cudaSuccess)
    e = launch_serialised(k_order_base, dim3((unsigned)o.n_groups), dim3(32), 0, st, o, (const uint32_t*)hist, base);
  if (e == cudaSuccess)
    e = launch_serialised(k_order_scatter, dim3(grid), dim3(256), 0, st, o, (const uint32_t*)base, cursor, order);
  count_launches(3);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace airgs
