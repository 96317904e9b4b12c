// Binning and ordering of (tile, Gaussian) instances (sm_103a).
//
// The order the blend needs is (view, tile, depth, Gaussian index).  It is
// built in two stable stages instead of one wide-key sort:
//   1. per view, a stable LSD radix sort of the N depth keys (float bits of the
//      camera-space z; culled Gaussians carry 0xFFFFFFFF and sort last), with
//      the Gaussian index as value -> order (view, depth, index);
//   2. instances are emitted in that order (k_count_gather, k_scan_spans,
//      k_emit) and stably radix-sorted by their global tile id, whose
//      ceil(log2(tiles)) bits are all the second sort has to look at.
// Then k_tile_ranges marks each tile's [start, end).
//
// The radix sort is reduce-then-scan, 8-bit digits: k_rs_upsweep counts digits
// per CTA, k_rs_spine scans the counts of each segment (digit-major, so each
// CTA's run of a digit lands after the previous CTAs' runs: stability), and
// k_rs_downsweep ranks each 2048-key tile stably in shared memory (warp
// match/popc per 32-key round) and writes it out digit-contiguously, which
// keeps the global writes coalesced.
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;   // keys per thread per tile
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_RADIX = 256;

struct SortGeom {
  int64_t seg_len;    // keys per segment
  int n_seg;          // segments (views), each sorted independently
  int64_t tiles_seg;  // RS_TILE-key tiles per segment
  int ctas_seg;       // CTAs per segment
  int64_t tiles_cta;  // tiles handled by one CTA (contiguous)
};

__device__ __forceinline__ void cta_range(const SortGeom& g, int cta, int& seg, int64_t& t0, int64_t& t1) {
  seg = cta / g.ctas_seg;
  int c = cta % g.ctas_seg;
  t0 = (int64_t)c * g.tiles_cta;
  t1 = min(t0 + g.tiles_cta, g.tiles_seg);
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_upsweep(const uint32_t* __restrict__ keys, SortGeom g, int shift,
                                                          uint32_t* __restrict__ counts) {
  __shared__ uint32_t hist[RS_WARPS][RS_RADIX];
  int tid = threadIdx.x, warp = tid >> 5;
  for (int k = tid; k < RS_WARPS * RS_RADIX; k += RS_THREADS) (&hist[0][0])[k] = 0;
  __syncthreads();
  int seg;
  int64_t t0, t1;
  cta_range(g, blockIdx.x, seg, t0, t1);
  int64_t base = (int64_t)seg * g.seg_len;
  int64_t e0 = t0 * RS_TILE, e1 = min(t1 * RS_TILE, g.seg_len);
  for (int64_t e = e0 + tid; e < e1; e += RS_THREADS) {
    uint32_t d = (__ldg(keys + base + e) >> shift) & 0xFF;
    atomicAdd(&hist[warp][d], 1u);
  }
  __syncthreads();
  int c = blockIdx.x % g.ctas_seg;
  for (int d = tid; d < RS_RADIX; d += RS_THREADS) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) s += hist[w][d];
    counts[((size_t)seg * RS_RADIX + d) * g.ctas_seg + c] = s;
  }
}

// Exclusive scan of one segment's RS_RADIX * ctas_seg counts (in place).
__global__ void __launch_bounds__(1024) k_rs_spine(uint32_t* counts, int ctas_seg) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* c = counts + (size_t)blockIdx.x * RS_RADIX * ctas_seg;
  int64_t total = (int64_t)RS_RADIX * ctas_seg;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < total; base += 1024) {
    int64_t idx = base + tid;
    uint32_t v = idx < total ? c[idx] : 0;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t ws = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sums[lane] = ws;  // inclusive
    }
    __syncthreads();
    uint32_t excl = carry + (warp ? warp_sums[warp - 1] : 0) + x - v;
    if (idx < total) c[idx] = excl;
    __syncthreads();
    if (tid == 1023) carry = excl + v;
    __syncthreads();
  }
}

// vals_in == nullptr: the value of a key is its index within its segment.
__global__ void __launch_bounds__(RS_THREADS) k_rs_downsweep(const uint32_t* __restrict__ keys_in,
                                                            const uint32_t* __restrict__ vals_in,
                                                            uint32_t* __restrict__ keys_out,
                                                            uint32_t* __restrict__ vals_out, SortGeom g, int shift,
                                                            const uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_keys[RS_TILE];
  __shared__ uint32_t s_vals[RS_TILE];
  __shared__ uint32_t s_warp_cnt[RS_WARPS][RS_RADIX];  // per-warp digit counts, then per-warp offsets
  __shared__ uint32_t s_offset[RS_RADIX];               // running global offset of each digit
  __shared__ uint32_t s_local[RS_RADIX];                // tile-local start of each digit
  __shared__ uint32_t s_scan[RS_WARPS];

  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int seg;
  int64_t t0, t1;
  cta_range(g, blockIdx.x, seg, t0, t1);
  int64_t base = (int64_t)seg * g.seg_len;
  int c = blockIdx.x % g.ctas_seg;
  for (int d = tid; d < RS_RADIX; d += RS_THREADS) s_offset[d] = counts[((size_t)seg * RS_RADIX + d) * g.ctas_seg + c];
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  for (int64_t t = t0; t < t1; ++t) {
    int64_t e0 = t * RS_TILE;
    int tile_n = (int)min((int64_t)RS_TILE, g.seg_len - e0);
    for (int k = tid; k < RS_WARPS * RS_RADIX; k += RS_THREADS) (&s_warp_cnt[0][0])[k] = 0;
    __syncthreads();

    // warp w ranks tile positions [w*256, w*256 + 256), 32 per round, in order
    uint32_t key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
      int p = warp * (RS_ITEMS * 32) + j * 32 + lane;
      bool valid = p < tile_n;
      uint32_t k = valid ? __ldg(keys_in + base + e0 + p) : 0xFFFFFFFFu;
      val[j] = valid ? (vals_in ? __ldg(vals_in + base + e0 + p) : (uint32_t)(e0 + p)) : 0u;
      key[j] = k;
      uint32_t d = valid ? ((k >> shift) & 0xFF) : RS_RADIX;  // invalid keys form their own class
      uint32_t peers = __match_any_sync(0xffffffffu, d);
      uint32_t before = 0;
      if (valid) before = s_warp_cnt[warp][d];
      __syncwarp();
      if (valid && (peers & lanemask_lt) == 0) s_warp_cnt[warp][d] = before + __popc(peers);
      __syncwarp();
      rank[j] = before + __popc(peers & lanemask_lt);
    }
    __syncthreads();

    // per digit: offsets of each warp's run, tile total
    uint32_t tot = 0;
    {
      int d = tid;  // RS_THREADS == RS_RADIX
      for (int w = 0; w < RS_WARPS; ++w) {
        uint32_t cnt = s_warp_cnt[w][d];
        s_warp_cnt[w][d] = tot;
        tot += cnt;
      }
      // exclusive scan of the tile totals over digits
      uint32_t x = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_scan[warp] = x;
      __syncthreads();
      if (warp == 0) {
        uint32_t ws = lane < RS_WARPS ? s_scan[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
          if (lane >= o) ws += y;
        }
        if (lane < RS_WARPS) s_scan[lane] = ws;
      }
      __syncthreads();
      s_local[d] = (warp ? s_scan[warp - 1] : 0) + x - tot;
    }
    __syncthreads();

    // scatter into shared memory in digit order (stable)
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
      int p = warp * (RS_ITEMS * 32) + j * 32 + lane;
      if (p < tile_n) {
        uint32_t d = (key[j] >> shift) & 0xFF;
        uint32_t pos = s_local[d] + s_warp_cnt[warp][d] + rank[j];
        s_keys[pos] = key[j];
        s_vals[pos] = val[j];
      }
    }
    __syncthreads();

    // coalesced write-out: consecutive threads write consecutive positions of a digit run
    for (int p = tid; p < tile_n; p += RS_THREADS) {
      uint32_t k = s_keys[p];
      uint32_t d = (k >> shift) & 0xFF;
      uint32_t dst = s_offset[d] + (uint32_t)p - s_local[d];
      keys_out[base + dst] = k;
      vals_out[base + dst] = s_vals[p];
    }
    __syncthreads();
    s_offset[tid] += tot;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ instance emission
constexpr int EM_THREADS = 256;
constexpr int EM_ITEMS = 4;
constexpr int EM_CHUNK = EM_THREADS * EM_ITEMS;

// counts_sorted[p] = tiles_touched of the Gaussian at depth-order position p;
// chunk_sums[b] = sum over chunk b.
__global__ void __launch_bounds__(EM_THREADS) k_count_gather(int64_t total, int64_t n,
                                                            const uint32_t* __restrict__ order,
                                                            const uint32_t* __restrict__ tiles_touched,
                                                            uint32_t* __restrict__ counts_sorted,
                                                            uint64_t* __restrict__ chunk_sums) {
  __shared__ uint64_t s_w[EM_THREADS / 32];
  int64_t c0 = (int64_t)blockIdx.x * EM_CHUNK;
  uint64_t sum = 0;
#pragma unroll
  for (int j = 0; j < EM_ITEMS; ++j) {
    int64_t p = c0 + j * EM_THREADS + threadIdx.x;
    if (p < total) {
      int64_t v = p / n;
      uint32_t cnt = __ldg(tiles_touched + v * n + __ldg(order + p));
      counts_sorted[p] = cnt;
      sum += cnt;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t s = 0;
    for (int w = 0; w < EM_THREADS / 32; ++w) s += s_w[w];
    chunk_sums[blockIdx.x] = s;
  }
}

// Exclusive scan of the chunk sums (one CTA); total -> *total_out.
__global__ void __launch_bounds__(1024) k_scan_spans(uint64_t* sums, int64_t n_chunks, uint64_t* total_out) {
  __shared__ uint64_t warp_sums[32];
  __shared__ uint64_t carry;
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n_chunks; base += 1024) {
    int64_t idx = base + tid;
    uint64_t v = idx < n_chunks ? sums[idx] : 0;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t ws = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sums[lane] = ws;
    }
    __syncthreads();
    uint64_t excl = carry + (warp ? warp_sums[warp - 1] : 0) + x - v;
    if (idx < n_chunks) sums[idx] = excl;
    __syncthreads();
    if (tid == 1023) carry = excl + v;
    __syncthreads();
  }
  if (tid == 0) *total_out = carry;
}

// Emit every instance of every Gaussian in depth order: key = global tile id,
// value = Gaussian index.  Tiles of one Gaussian go out row-major.
__global__ void __launch_bounds__(EM_THREADS) k_emit(int64_t total, int64_t n, const uint32_t* __restrict__ order,
                                                    const uint32_t* __restrict__ counts_sorted,
                                                    const uint64_t* __restrict__ chunk_offsets,
                                                    const ProjRec* __restrict__ proj, const CamDev* __restrict__ cams,
                                                    float log2_amin, bool with_halves, uint32_t* __restrict__ keys,
                                                    uint32_t* __restrict__ vals) {
  __shared__ uint64_t s_w[EM_THREADS / 32];
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int64_t c0 = (int64_t)blockIdx.x * EM_CHUNK;
  // blocked arrangement: thread t owns positions c0 + t*EM_ITEMS .. +EM_ITEMS
  uint32_t cnt[EM_ITEMS];
  uint64_t local = 0;
#pragma unroll
  for (int j = 0; j < EM_ITEMS; ++j) {
    int64_t p = c0 + (int64_t)tid * EM_ITEMS + j;
    cnt[j] = p < total ? __ldg(counts_sorted + p) : 0u;
    local += cnt[j];
  }
  uint64_t x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  uint64_t woff = 0;
  for (int w = 0; w < warp; ++w) woff += s_w[w];
  uint64_t off = chunk_offsets[blockIdx.x] + woff + x - local;
#pragma unroll
  for (int j = 0; j < EM_ITEMS; ++j) {
    int64_t p = c0 + (int64_t)tid * EM_ITEMS + j;
    if (cnt[j]) {
      int v = (int)(p / n);
      uint32_t gid = __ldg(order + p);
      const CamDev& cam = cams[v];
      ProjRec rec = proj[(size_t)v * n + gid];
      int radius = __float_as_int(rec.c.z);
      int x0, y0, x1, y1;
      tile_rect(rec.a.x, rec.a.y, radius, cam.TW, cam.TH, x0, y0, x1, y1);
      uint32_t tb = (uint32_t)cam.tile_base;
      float hx = 0.f, hy = 0.f;
      const int kind = with_halves ? alpha_box(rec.a, rec.b, log2_amin, hx, hy) : 2;
      for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) {
          // with more than 2^24 tiles the sort reaches the top bits: keep them uniform
          const uint32_t halves = half_flags_of(rec.a, kind, hx, hy, (float)(tx * kTile), (float)(ty * kTile));
          keys[off] = (tb + (uint32_t)(ty * cam.TW + tx)) | (halves << kKeyHalfShift);
          vals[off] = gid;
          ++off;
        }
    }
  }
}

__global__ void k_tile_ranges(int64_t n_inst, const uint32_t* __restrict__ keys, uint2* __restrict__ ranges) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_inst) return;
  uint32_t k = keys[p] & kKeyTileMask;
  if (p == 0 || (keys[p - 1] & kKeyTileMask) != k) ranges[k].x = (uint32_t)p;
  if (p == n_inst - 1 || (keys[p + 1] & kKeyTileMask) != k) ranges[k].y = (uint32_t)(p + 1);
}

// ------------------------------------------------------------------ host side
static SortGeom make_geom(int64_t seg_len, int n_seg, int num_sms) {
  SortGeom g;
  g.seg_len = seg_len;
  g.n_seg = n_seg;
  g.tiles_seg = (seg_len + RS_TILE - 1) / RS_TILE;
  if (g.tiles_seg == 0) g.tiles_seg = 1;
  int target = max(1, (2 * num_sms + n_seg - 1) / n_seg);  // about two CTAs per SM overall
  g.tiles_cta = (g.tiles_seg + target - 1) / target;
  g.ctas_seg = (int)((g.tiles_seg + g.tiles_cta - 1) / g.tiles_cta);
  return g;
}

size_t radix_scratch_bytes(int64_t seg_len, int n_seg, int num_sms) {
  SortGeom g = make_geom(seg_len, n_seg, num_sms);
  return (size_t)n_seg * RS_RADIX * g.ctas_seg * sizeof(uint32_t);
}

// Sorts each of n_seg segments of seg_len keys by bits [0, key_bits), ping-
// ponging between (keys_a, vals_a) and (keys_b, vals_b); *result_in_b tells
// which pair holds the result.  With identity_vals the first pass takes the
// in-segment index as the value instead of reading vals_a (vals_a is still
// used as a buffer by later passes).
cudaError_t radix_sort_pairs(cudaStream_t st, int num_sms, uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b,
                             uint32_t* vals_b, int64_t seg_len, int n_seg, int key_bits, bool identity_vals,
                             uint32_t* scratch, bool* result_in_b) {
  *result_in_b = false;
  if (seg_len == 0 || n_seg == 0) return cudaSuccess;
  SortGeom g = make_geom(seg_len, n_seg, num_sms);
  int grid = g.ctas_seg * n_seg;
  int passes = (key_bits + 7) / 8;
  uint32_t *ki = keys_a, *vi = vals_a, *ko = keys_b, *vo = vals_b;
  for (int pass = 0; pass < passes; ++pass) {
    int shift = 8 * pass;
    k_rs_upsweep<<<grid, RS_THREADS, 0, st>>>(ki, g, shift, scratch);
    k_rs_spine<<<n_seg, 1024, 0, st>>>(scratch, g.ctas_seg);
    k_rs_downsweep<<<grid, RS_THREADS, 0, st>>>(ki, (pass == 0 && identity_vals) ? nullptr : vi, ko, vo, g, shift,
                                                 scratch);
    count_launches(3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint32_t* t = ki;
    ki = ko;
    ko = t;
    t = vi;
    vi = vo;
    vo = t;
    *result_in_b = !*result_in_b;
  }
  return cudaSuccess;
}

// One 8-bit pass (bits [shift, shift + 8)) of the same radix sort over a single
// segment, reading (keys_in, vals_in) and writing (keys_out, vals_out);
// `counts` must hold radix_scratch_bytes(n, 1, num_sms) bytes.
cudaError_t radix_sort_pass(cudaStream_t st, int num_sms, const uint32_t* keys_in, const uint32_t* vals_in,
                            uint32_t* keys_out, uint32_t* vals_out, int64_t n, int shift, uint32_t* counts) {
  if (n == 0) return cudaSuccess;
  SortGeom g = make_geom(n, 1, num_sms);
  k_rs_upsweep<<<g.ctas_seg, RS_THREADS, 0, st>>>(keys_in, g, shift, counts);
  k_rs_spine<<<1, 1024, 0, st>>>(counts, g.ctas_seg);
  k_rs_downsweep<<<g.ctas_seg, RS_THREADS, 0, st>>>(keys_in, vals_in, keys_out, vals_out, g, shift, counts);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_count_gather(cudaStream_t st, int64_t total, int64_t n, const uint32_t* order,
                                const uint32_t* tiles_touched, uint32_t* counts_sorted, uint64_t* chunk_sums,
                                int64_t* n_chunks) {
  *n_chunks = (total + EM_CHUNK - 1) / EM_CHUNK;
  if (total == 0) return cudaSuccess;
  k_count_gather<<<(unsigned)*n_chunks, EM_THREADS, 0, st>>>(total, n, order, tiles_touched, counts_sorted,
                                                             chunk_sums);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scan_spans(cudaStream_t st, uint64_t* sums, int64_t n_chunks, uint64_t* total_out) {
  k_scan_spans<<<1, 1024, 0, st>>>(sums, n_chunks, total_out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_emit(cudaStream_t st, int64_t total, int64_t n, const uint32_t* order,
                        const uint32_t* counts_sorted, const uint64_t* chunk_offsets, const ProjRec* proj,
                        const CamDev* cams, float alpha_min, int64_t n_tiles, uint32_t* keys, uint32_t* vals) {
  if (total == 0) return cudaSuccess;
  int64_t n_chunks = (total + EM_CHUNK - 1) / EM_CHUNK;
  k_emit<<<(unsigned)n_chunks, EM_THREADS, 0, st>>>(total, n, order, counts_sorted, chunk_offsets, proj, cams,
                                                     log2f(alpha_min), n_tiles <= (1ll << 24), keys, vals);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_tile_ranges(cudaStream_t st, int64_t n_inst, const uint32_t* keys, uint2* ranges) {
  if (n_inst == 0) return cudaSuccess;
  k_tile_ranges<<<(unsigned)((n_inst + 255) / 256), 256, 0, st>>>(n_inst, keys, ranges);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace airgs
