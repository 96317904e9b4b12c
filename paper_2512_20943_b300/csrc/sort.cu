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
// per CTA, k_rs_spine scans each (segment, digit) row of per-CTA counts with
// one warp per row (digit-major, so each CTA's run of a digit lands after the
// previous CTAs' runs: stability) and leaves the row totals, whose scan over
// digits every k_rs_downsweep CTA redoes in shared memory; k_rs_downsweep ranks
// each 2048-key tile stably in shared memory (warp match/popc per 32-key
// round) and writes it out digit-contiguously, which keeps the global writes
// coalesced.  About RS_CTAS_PER_SM CTAs per SM keep loads in flight.
#include "airgs_internal.cuh"
#include "kernels.h"
#include "launch.cuh"

namespace airgs {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
#ifndef AIRGS_RS_ITEMS
#define AIRGS_RS_ITEMS 8
#endif
#ifndef AIRGS_RS_ITEMS_SEG
#define AIRGS_RS_ITEMS_SEG 6  // measured best of 4, 6, 8 (more CTAs over the views' short segments)
#endif
constexpr int RS_ITEMS = AIRGS_RS_ITEMS;          // keys per thread per tile
constexpr int RS_ITEMS_SEG = AIRGS_RS_ITEMS_SEG;  // the same for a sort of several segments (the per-view depth sort)
constexpr int RS_RADIX = 256;
constexpr int RS_CTAS_PER_SM = 8;

// The radix kernels and the emission chain are launched with programmatic
// stream serialisation (launch.cuh): each waits for its predecessor first.
struct SortGeom {
  int64_t tile;       // keys per CTA tile (RS_THREADS x keys per thread)
  int64_t seg_len;    // keys per segment
  int n_seg;          // segments (views), each sorted independently
  int64_t tiles_seg;  // tiles per segment
  int ctas_seg;       // CTAs per segment
  int64_t tiles_cta;  // tiles handled by one CTA (contiguous)
};

__device__ __forceinline__ void cta_range(const SortGeom& g, int cta, int& seg, int64_t& t0, int64_t& t1) {
  seg = cta / g.ctas_seg;
  int c = cta % g.ctas_seg;
  t0 = (int64_t)c * g.tiles_cta;
  t1 = min(t0 + g.tiles_cta, g.tiles_seg);
}

// Digit of a pass: bits [shift, min(shift + 8, key_bits)) of the key, so that
// the bits above key_bits (flags kept in the same word) never take part.
static inline uint32_t radix_digit_mask(int key_bits, int shift) {
  const int w = key_bits - shift;
  return w >= 8 ? 0xFFu : (1u << w) - 1u;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_upsweep(const uint32_t* __restrict__ keys, SortGeom g, int shift,
                                                          uint32_t dmask, uint32_t* __restrict__ counts) {
  wait_prior_grid();
  const int64_t RS_TILE = g.tile;
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
    uint32_t d = (__ldg(keys + base + e) >> shift) & dmask;
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

// One warp per (segment, digit) row: exclusive scan of the row's per-CTA counts
// in place, row total -> totals[segment * RS_RADIX + digit].
__global__ void __launch_bounds__(256) k_rs_spine(uint32_t* counts, uint32_t* totals, int ctas_seg, int rows) {
  wait_prior_grid();
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= rows) return;
  uint32_t* c = counts + (size_t)row * ctas_seg;
  uint32_t carry = 0;
  for (int base = 0; base < ctas_seg; base += 32) {
    const int idx = base + lane;
    const uint32_t v = idx < ctas_seg ? c[idx] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (idx < ctas_seg) c[idx] = carry + x - v;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) totals[row] = carry;
}

// vals_in == nullptr: the value of a key is its index within its segment.
#ifndef AIRGS_RS_MINB
#define AIRGS_RS_MINB 5  // 48 registers, 5 CTAs per SM (measured best of 4 (unbounded), 5, 6, 8)
#endif
template <int RS_ITEMS>
__global__ void __launch_bounds__(RS_THREADS, AIRGS_RS_MINB) k_rs_downsweep(const uint32_t* __restrict__ keys_in,
                                                            const uint32_t* __restrict__ vals_in,
                                                            uint32_t* __restrict__ keys_out,
                                                            uint32_t* __restrict__ vals_out, SortGeom g, int shift,
                                                            uint32_t dmask, const uint32_t* __restrict__ counts,
                                                            const uint32_t* __restrict__ totals) {
  wait_prior_grid();
  constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
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
  {
    // digit bases of this segment: exclusive scan of the row totals (RS_THREADS == RS_RADIX)
    const uint32_t tot = totals[(size_t)seg * RS_RADIX + tid];
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_scan[warp] = x;
    __syncthreads();
    uint32_t wb = 0;
    for (int w = 0; w < warp; ++w) wb += s_scan[w];
    s_offset[tid] = wb + x - tot + counts[((size_t)seg * RS_RADIX + tid) * g.ctas_seg + c];
    __syncthreads();
  }
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  for (int64_t t = t0; t < t1; ++t) {
    int64_t e0 = t * RS_TILE;
    int tile_n = (int)min((int64_t)RS_TILE, g.seg_len - e0);
    for (int k = tid; k < RS_WARPS * RS_RADIX; k += RS_THREADS) (&s_warp_cnt[0][0])[k] = 0;
    __syncthreads();

    // warp w ranks tile positions [w*256, w*256 + 256), 32 per round, in order;
    // all of the thread's keys and values are loaded before the ranking, so the
    // loads overlap instead of each waiting behind the previous round's sync
    uint32_t key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
      const int p = warp * (RS_ITEMS * 32) + j * 32 + lane;
      const bool valid = p < tile_n;
      key[j] = valid ? __ldg(keys_in + base + e0 + p) : 0xFFFFFFFFu;
      val[j] = valid ? (vals_in ? __ldg(vals_in + base + e0 + p) : (uint32_t)(e0 + p)) : 0u;
    }
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
      const int p = warp * (RS_ITEMS * 32) + j * 32 + lane;
      const bool valid = p < tile_n;
      const uint32_t k = key[j];
      uint32_t d = valid ? ((k >> shift) & dmask) : RS_RADIX;  // invalid keys form their own class
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
        uint32_t d = (key[j] >> shift) & dmask;
        uint32_t pos = s_local[d] + s_warp_cnt[warp][d] + rank[j];
        s_keys[pos] = key[j];
        s_vals[pos] = val[j];
      }
    }
    __syncthreads();

    // coalesced write-out: consecutive threads write consecutive positions of a digit run
    for (int p = tid; p < tile_n; p += RS_THREADS) {
      uint32_t k = s_keys[p];
      uint32_t d = (k >> shift) & dmask;
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
#ifndef AIRGS_EM_ITEMS
#define AIRGS_EM_ITEMS 1  // 256-Gaussian chunks: 6 CTAs per SM (measured best of 1, 2)
#endif
constexpr int EM_ITEMS = AIRGS_EM_ITEMS;
constexpr int EM_CHUNK = EM_THREADS * EM_ITEMS;

int64_t emit_chunks(int64_t total) { return (total + EM_CHUNK - 1) / EM_CHUNK; }

// counts_sorted[p] = tiles_touched of the Gaussian at depth-order position p;
// chunk_sums[b] = sum over chunk b.
constexpr int CG_THREADS = 64;                    // a chunk's positions over 64 threads,
constexpr int CG_ITEMS = EM_CHUNK / CG_THREADS;   // so that each thread's gathers overlap
__global__ void __launch_bounds__(CG_THREADS) k_count_gather(int64_t total, int64_t n,
                                                            const uint32_t* __restrict__ order,
                                                            const uint32_t* __restrict__ tiles_touched,
                                                            uint32_t* __restrict__ counts_sorted,
                                                            uint64_t* __restrict__ chunk_sums) {
  wait_prior_grid();
  __shared__ uint64_t s_w[CG_THREADS / 32];
  const int64_t c0 = (int64_t)blockIdx.x * EM_CHUNK;
  uint32_t gid[CG_ITEMS];
#pragma unroll
  for (int j = 0; j < CG_ITEMS; ++j) {
    const int64_t p = c0 + j * CG_THREADS + threadIdx.x;
    gid[j] = p < total ? __ldg(order + p) : 0u;
  }
  uint32_t cnt[CG_ITEMS];
#pragma unroll
  for (int j = 0; j < CG_ITEMS; ++j) {
    const int64_t p = c0 + j * CG_THREADS + threadIdx.x;
    const int64_t v = total < (int64_t)0xFFFFFFFFll ? (int64_t)((uint32_t)p / (uint32_t)n) : p / n;
    cnt[j] = p < total ? __ldg(tiles_touched + v * n + gid[j]) : 0u;
  }
  uint64_t sum = 0;
#pragma unroll
  for (int j = 0; j < CG_ITEMS; ++j) {
    const int64_t p = c0 + j * CG_THREADS + threadIdx.x;
    if (p < total) counts_sorted[p] = cnt[j];
    sum += cnt[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t s = 0;
    for (int w = 0; w < CG_THREADS / 32; ++w) s += s_w[w];
    chunk_sums[blockIdx.x] = s;
  }
}

// Exclusive scan in place of one or two arrays of n_chunks chunk sums, one CTA
// per array (blockIdx.x picks it); each array's total -> its total pointer.
// Every thread scans SP_ITEMS consecutive values per round, so a round covers
// SP_THREADS x SP_ITEMS values and the CTA's serial rounds stay few.
constexpr int SP_THREADS = 1024;
constexpr int SP_ITEMS = 8;
__global__ void __launch_bounds__(SP_THREADS) k_scan_spans(uint64_t* sums0, uint64_t* sums1, int64_t n_chunks,
                                                          uint64_t* total0, uint64_t* total1) {
  wait_prior_grid();
  uint64_t* sums = blockIdx.x ? sums1 : sums0;
  __shared__ uint64_t warp_sums[SP_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t carry = 0;  // the same in every thread
  for (int64_t base = 0; base < n_chunks; base += (int64_t)SP_THREADS * SP_ITEMS) {
    const int64_t i0 = base + (int64_t)tid * SP_ITEMS;
    uint64_t v[SP_ITEMS];
    uint64_t local = 0;
#pragma unroll
    for (int j = 0; j < SP_ITEMS; ++j) {
      v[j] = i0 + j < n_chunks ? sums[i0 + j] : 0ull;
      local += v[j];
    }
    uint64_t x = local;  // inclusive scan of the thread totals within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t ws = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sums[lane] = ws;  // inclusive over the warps
    }
    __syncthreads();
    uint64_t run = carry + (warp ? warp_sums[warp - 1] : 0ull) + x - local;
#pragma unroll
    for (int j = 0; j < SP_ITEMS; ++j) {
      if (i0 + j < n_chunks) sums[i0 + j] = run;
      run += v[j];
    }
    carry += warp_sums[SP_THREADS / 32 - 1];
    __syncthreads();  // warp_sums is rewritten by the next round
  }
  if (tid == 0) *(blockIdx.x ? total1 : total0) = carry;
}

// Pieces of at most EM_PIECE instances per chunk: piece_off[c] = exclusive
// scan over chunks of ceil(instances of chunk c / EM_PIECE) (one CTA), total
// pieces in piece_off[n_chunks].  chunk_offsets holds the chunks' exclusive
// instance offsets with the total in chunk_offsets[n_chunks].
// RUN: instances per thread and piece (4, 8 or 16: a kernel-shape parameter);
// a piece is EM_THREADS x RUN instances, one CTA.
template <int RUN>
struct EmitGeom {
  static constexpr uint32_t PIECE = (uint32_t)EM_THREADS * RUN;  // instances per CTA
  static constexpr int STAGE = EM_THREADS * (RUN + 1);            // padded staging rows (no bank conflicts)
  static constexpr size_t SMEM = 3 * EM_CHUNK * sizeof(float4) + EM_CHUNK * sizeof(float2) +
                                 (2 * EM_CHUNK + 4) * sizeof(uint32_t) + 2 * STAGE * sizeof(uint32_t);
};
constexpr uint32_t EM_MIN_PIECE = EmitGeom<4>::PIECE;  // the smallest piece (bounds the piece count)

template <int RUN>
__global__ void __launch_bounds__(SP_THREADS) k_emit_pieces(const uint64_t* __restrict__ chunk_offsets,
                                                           int64_t n_chunks, uint32_t* __restrict__ piece_off) {
  wait_prior_grid();
  __shared__ uint32_t warp_sums[SP_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t carry = 0;  // the same in every thread
  for (int64_t base = 0; base < n_chunks; base += (int64_t)SP_THREADS * SP_ITEMS) {
    const int64_t c0 = base + (int64_t)tid * SP_ITEMS;
    uint32_t v[SP_ITEMS];
    uint32_t local = 0;
#pragma unroll
    for (int j = 0; j < SP_ITEMS; ++j) {
      const int64_t c = c0 + j;
      constexpr uint32_t PIECE = EmitGeom<RUN>::PIECE;
      v[j] = c < n_chunks ? (uint32_t)((chunk_offsets[c + 1] - chunk_offsets[c] + PIECE - 1) / PIECE) : 0u;
      local += v[j];
    }
    uint32_t x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t ws = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sums[lane] = ws;
    }
    __syncthreads();
    uint32_t run = carry + (warp ? warp_sums[warp - 1] : 0u) + x - local;
#pragma unroll
    for (int j = 0; j < SP_ITEMS; ++j) {
      if (c0 + j < n_chunks) piece_off[c0 + j] = run;
      run += v[j];
    }
    carry += warp_sums[SP_THREADS / 32 - 1];
    __syncthreads();
  }
  if (tid == 0) piece_off[n_chunks] = carry;
}

// piece_chunk[b] = the chunk that owns piece b (one thread per chunk).
__global__ void k_emit_piece_map(const uint32_t* __restrict__ piece_off, int64_t n_chunks,
                                 uint32_t* __restrict__ piece_chunk) {
  wait_prior_grid();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  for (uint32_t b = piece_off[c]; b < piece_off[c + 1]; ++b) piece_chunk[b] = (uint32_t)c;
}

// Emit every instance of every Gaussian in depth order: key = global tile id
// (plus the half flags in bits 30-31), value = Gaussian index; the tiles of one
// Gaussian go out row-major.  A CTA takes one piece (at most EM_PIECE
// instances) of a chunk of EM_CHUNK consecutive depth-order positions, so that
// no CTA carries much more work than another however uneven the counts are
// (nearby Gaussians, which come first in depth order, cover many tiles).  The
// CTA scans the chunk's counts into list offsets (thread t holds Gaussian t of
// the chunk, whose id it loads first so that the scan hides that load), finds
// the owners of the piece's first and last instances (each thread tests its own
// Gaussian's offset range), and describes the Gaussians that own the piece's
// instances in shared memory (first key, rectangle, alpha box and terms of the
// exact half test).  Thread t then
// produces the piece's instances t*EM_RUN .. +EM_RUN: one binary search for
// the owner of the first, then tile by tile (row-major stepping, no division
// past the first), moving to the next Gaussian when the offsets say so; the
// run goes to shared memory (rows padded to EM_RUN + 1 words) and the CTA
// writes the piece out coalesced.
template <int RUN>
__global__ void __launch_bounds__(EM_THREADS) k_emit(int64_t total, int64_t n, const uint32_t* __restrict__ order,
                                                    const uint32_t* __restrict__ counts_sorted,
                                                    const uint64_t* __restrict__ chunk_offsets,
                                                    const uint32_t* __restrict__ piece_off,
                                                    const uint32_t* __restrict__ piece_chunk, int64_t n_chunks,
                                                    const ProjRec* __restrict__ proj, const CamDev* __restrict__ cams,
                                                    float log2_amin, bool with_halves, int cull,
                                                    uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  wait_prior_grid();
  constexpr uint32_t EM_PIECE = EmitGeom<RUN>::PIECE;
  constexpr int EM_STAGE = EmitGeom<RUN>::STAGE;
  constexpr int EM_RUN = RUN;
  // dynamic shared memory (EmitGeom<RUN>::SMEM bytes):
  extern __shared__ float4 em_smem[];
  float4* s_box = em_smem;                   // centre, alpha-box half-widths (-inf: never, +inf: unbounded)
  float4* s_quad = s_box + EM_CHUNK;         // a2, b2, c2 (a2 = 0: no exact test), L = log2(o / alpha_min)
  uint4* s_rect = reinterpret_cast<uint4*>(s_quad + EM_CHUNK);  // first key, width | tile columns << 16,
                                                                // x0 | y0 << 16, Gaussian id
  float2* s_kxy = reinterpret_cast<float2*>(s_rect + EM_CHUNK);     // maximisers along a row / column
  uint32_t* s_off = reinterpret_cast<uint32_t*>(s_kxy + EM_CHUNK);  // [EM_CHUNK + 1] chunk-local first instances
  uint32_t* s_ext = s_off + EM_CHUNK + 4;                             // culled lists: tile columns | rows << 16
  uint32_t* s_key = s_ext + EM_CHUNK;                                 // [EM_STAGE] staged keys
  uint32_t* s_val = s_key + EM_STAGE;                                 // [EM_STAGE] staged values
  __shared__ uint32_t s_w[EM_THREADS / 32];
  __shared__ int s_g0, s_g1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t b = blockIdx.x;
  if (b >= piece_off[n_chunks]) return;  // the grid is an upper bound on the pieces
  const int64_t chunk = piece_chunk[b];
  const uint32_t piece = b - piece_off[chunk];
  const int64_t c0 = chunk * EM_CHUNK;
  // the chunk's Gaussian ids in depth order (thread t: Gaussian t), loaded now so
  // that describing the piece's Gaussians below waits for one global load
  static_assert(EM_ITEMS == 1 && EM_CHUNK == EM_THREADS, "one Gaussian per thread");
  const uint32_t my_gid = c0 + tid < total ? __ldg(order + c0 + tid) : 0u;
  // chunk offsets: blocked, thread t scans chunk positions t*EM_ITEMS .. +EM_ITEMS
  uint32_t cnt[EM_ITEMS];
  uint32_t local = 0;
#pragma unroll
  for (int j = 0; j < EM_ITEMS; ++j) {
    const int64_t p = c0 + (int64_t)tid * EM_ITEMS + j;
    cnt[j] = p < total ? __ldg(counts_sorted + p) : 0u;
    local += cnt[j];  // chunk totals stay below 2^32: the instance count was checked
  }
  uint32_t x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  uint32_t off = x - local;
  for (int w = 0; w < warp; ++w) off += s_w[w];
#pragma unroll
  for (int j = 0; j < EM_ITEMS; ++j) {
    s_off[tid * EM_ITEMS + j] = off;
    off += cnt[j];
  }
  if (tid == EM_THREADS - 1) s_off[EM_CHUNK] = off;
  __syncthreads();

  const uint32_t p0 = piece * EM_PIECE;
  const uint32_t p1 = (uint32_t)min((uint64_t)s_off[EM_CHUNK], (uint64_t)p0 + EM_PIECE);
  // the last Gaussian whose first instance is <= i owns instance i
  auto owner = [&](uint32_t i, int lo, int hi) {
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  {  // owners of the piece's first and last instances: the g with s_off[g] <= i < s_off[g + 1]
    const uint32_t lo = s_off[tid], hi = s_off[tid + 1];
    if (lo <= p0 && p0 < hi) s_g0 = tid;
    if (lo <= p1 - 1 && p1 - 1 < hi) s_g1 = tid;
  }
  __syncthreads();
  const int g0 = s_g0, g1 = s_g1;
  for (int g = tid; g <= g1; g += EM_THREADS) {
    if (g < g0 || s_off[g + 1] == s_off[g]) continue;  // not in the piece, or no instances
    const int64_t p = c0 + g;
    const int v = (total < (int64_t)0xFFFFFFFFll) ? (int)((uint32_t)p / (uint32_t)n) : (int)(p / n);
    const uint32_t gid = my_gid;
    const CamDev& cam = cams[v];
    const ProjRec* rec = proj + (size_t)v * n + gid;
    const float4 ra = __ldg(&rec->a), rb = __ldg(&rec->b);
    const int radius = __float_as_int(__ldg(&rec->c.z));
    int x0, y0, x1, y1;
    tile_rect(ra.x, ra.y, radius, cam.TW, cam.TH, x0, y0, x1, y1);
    if (cull == kCullBox) clip_rect_to_alpha_box(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, log2_amin, x0, y0, x1, y1);
    s_rect[g] = make_uint4((uint32_t)cam.tile_base + (uint32_t)(y0 * cam.TW + x0),
                           (uint32_t)(x1 - x0) | ((uint32_t)cam.TW << 16), (uint32_t)x0 | ((uint32_t)y0 << 16), gid);
    if (cull == kCullBands) {  // culled lists: the row-band terms the projection counted with, from the same record values
      const EllipseBands e = ellipse_bands(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, log2_amin);
      s_rect[g].x = (uint32_t)cam.tile_base;
      s_ext[g] = (uint32_t)cam.TW | ((uint32_t)(y1 - y0) << 16);
      s_box[g] = make_float4(e.mx, e.my, e.hx, e.hy);
      s_quad[g] = make_float4(e.kx, e.cpr, e.inv_na2, e.L);
      s_kxy[g] = make_float2(e.dyr, e.kind == 2 ? -1.f : e.eps);  // (no instances when kind is 0)
    } else if (with_halves) {
      float hx = 0.f, hy = 0.f;
      const int kind = alpha_box(ra, rb, log2_amin, hx, hy);
      if (kind == 0) hx = hy = -INFINITY;
      if (kind == 2) hx = hy = INFINITY;
      const bool exact = kind == 1 && ra.z < 0.f && rb.x < 0.f && 4.f * ra.z * rb.x > 1.0001f * ra.w * ra.w;
      s_box[g] = make_float4(ra.x, ra.y, hx, hy);
      s_quad[g] = make_float4(exact ? ra.z : 0.f, ra.w, rb.x, lg2_approx(rb.y) - log2_amin + 1e-3f);
      s_kxy[g] = exact ? make_float2(__fdividef(-ra.w, 2.f * ra.z), __fdividef(-ra.w, 2.f * rb.x)) : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  const uint32_t i0 = p0 + (uint32_t)tid * EM_RUN;
  const uint32_t i1 = min(i0 + (uint32_t)EM_RUN, p1);
  if (cull == kCullBands && i0 < i1) {
    // culled lists: walk the live tiles row by row exactly as the projection counted them
    auto bands_of = [&](int gg) {
      EllipseBands e;
      const float4 b4 = s_box[gg], q4 = s_quad[gg];
      const float2 k2 = s_kxy[gg];
      e.mx = b4.x;
      e.my = b4.y;
      e.hx = b4.z;
      e.hy = b4.w;
      e.kx = q4.x;
      e.cpr = q4.y;
      e.inv_na2 = q4.z;
      e.L = q4.w;
      e.dyr = k2.x;
      e.eps = k2.y;
      e.kind = k2.y < 0.f ? 2 : 1;
      return e;
    };
    int g = owner(i0, g0, g1);
    EllipseBands e = bands_of(g);
    uint4 r = s_rect[g];
    int x0 = (int)(r.z & 0xFFFFu), y0 = (int)(r.z >> 16), x1 = x0 + (int)(r.y & 0xFFFFu);
    int y1 = y0 + (int)(s_ext[g] >> 16), tw = (int)(s_ext[g] & 0xFFFFu);
    int ty = y0;
    LiveRow row = live_row(e, ty, x0, x1);
    uint32_t li = i0 - s_off[g];
    while (li >= (uint32_t)(row.hi - row.lo) && ty + 1 < y1) {
      li -= (uint32_t)(row.hi - row.lo);
      row = live_row(e, ++ty, x0, x1);
    }
    int tx = row.lo + (int)li;
    for (uint32_t i = i0; i < i1; ++i) {
      if (i >= s_off[g + 1]) {  // first instance of the next Gaussian with instances
        do {
          ++g;
        } while (i >= s_off[g + 1]);
        e = bands_of(g);
        r = s_rect[g];
        x0 = (int)(r.z & 0xFFFFu);
        y0 = (int)(r.z >> 16);
        x1 = x0 + (int)(r.y & 0xFFFFu);
        y1 = y0 + (int)(s_ext[g] >> 16);
        tw = (int)(s_ext[g] & 0xFFFFu);
        ty = y0;
        row = live_row(e, ty, x0, x1);
        while (row.hi == row.lo && ty + 1 < y1) row = live_row(e, ++ty, x0, x1);
        tx = row.lo;
      } else if (i != i0 && ++tx >= row.hi) {  // next live row
        do {
          row = live_row(e, ++ty, x0, x1);
        } while (row.hi == row.lo && ty + 1 < y1);
        tx = row.lo;
      }
      const uint32_t halves = with_halves ? live_row_halves(row, tx) : 3u;
      const int slot = tid * (EM_RUN + 1) + (int)(i - i0);
      s_key[slot] = (r.x + (uint32_t)(ty * tw + tx)) | (halves << kKeyHalfShift);
      s_val[slot] = r.w;
    }
  } else if (i0 < i1) {
    int g = owner(i0, g0, g1);
    uint4 r = s_rect[g];
    float4 bx = s_box[g], qd = s_quad[g];
    float2 kxy = s_kxy[g];
    uint32_t w = r.y & 0xFFFFu, tw = r.y >> 16;
    uint32_t qy, rx;
    {
      const uint32_t li = i0 - s_off[g];
      qy = li / w;
      rx = li - qy * w;
    }
    for (uint32_t i = i0; i < i1; ++i) {
      if (i >= s_off[g + 1]) {  // first instance of the next Gaussian with instances
        do {
          ++g;
        } while (i >= s_off[g + 1]);
        r = s_rect[g];
        bx = s_box[g];
        qd = s_quad[g];
        kxy = s_kxy[g];
        w = r.y & 0xFFFFu;
        tw = r.y >> 16;
        qy = rx = 0;
      }
      // with more than 2^24 tiles the sort reaches the top bits: keep them uniform
      uint32_t halves = 3u;
      if (with_halves) {
        const float X0 = (float)(((r.z & 0xFFFFu) + rx) * kTile), Y0 = (float)(((r.z >> 16) + qy) * kTile);
        halves = 0u;
        if (bx.x + bx.z >= X0 + 0.5f && bx.x - bx.z <= X0 + 15.5f) {
          if (bx.y + bx.w >= Y0 + 0.5f && bx.y - bx.w <= Y0 + 7.5f) halves |= 1u;
          if (bx.y + bx.w >= Y0 + 8.5f && bx.y - bx.w <= Y0 + 15.5f) halves |= 2u;
        }
        if (halves != 0u && qd.x < 0.f) {  // refine by the exact test of each half's rectangle (rect_max_power2)
          const float xlo = (X0 + 0.5f) - bx.x, xhi = xlo + 15.f;
#pragma unroll
          for (int k = 0; k < 2; ++k) {  // both halves tested, the result masked (no divergence)
            const float ylo = (Y0 + 8.f * k + 0.5f) - bx.y, yhi = ylo + 7.f;
            float S;
            const float pm = rect_max_power2(qd.x, qd.y, qd.z, kxy.x, kxy.y, xlo, xhi, ylo, yhi, S);
            if (pm < -qd.w - (0.01f + 1e-5f * S)) halves &= ~(1u << k);
          }
        }
      }
      const int slot = tid * (EM_RUN + 1) + (int)(i - i0);
      s_key[slot] = (r.x + qy * tw + rx) | (halves << kKeyHalfShift);
      s_val[slot] = r.w;
      if (++rx == w) {
        rx = 0;
        ++qy;
      }
    }
  }
  __syncthreads();
  const uint64_t base = chunk_offsets[chunk] + p0;
  const uint32_t np = p1 - p0;
  for (uint32_t k = tid; k < np; k += EM_THREADS) {
    const uint32_t slot = (k / EM_RUN) * (EM_RUN + 1) + (k % EM_RUN);
    keys[base + k] = s_key[slot];
    vals[base + k] = s_val[slot];
  }
}

__global__ void k_tile_ranges(int64_t n_inst, const uint32_t* __restrict__ keys, uint2* __restrict__ ranges) {
  wait_prior_grid();
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_inst) return;
  uint32_t k = keys[p] & kKeyTileMask;
  if (p == 0 || (keys[p - 1] & kKeyTileMask) != k) ranges[k].x = (uint32_t)p;
  if (p == n_inst - 1 || (keys[p + 1] & kKeyTileMask) != k) ranges[k].y = (uint32_t)(p + 1);
}

// ------------------------------------------------------------------ host side
// keys: keys per thread of a CTA tile (6, 8 or 12; 0 = the default for the
// segment count).
static int radix_keys(int n_seg, int keys) {
  if (keys == 6 || keys == 8 || keys == 12) return keys;
  return n_seg > 1 ? RS_ITEMS_SEG : RS_ITEMS;
}

static SortGeom make_geom(int64_t seg_len, int n_seg, int num_sms, int keys = 0) {
  SortGeom g;
  g.tile = (int64_t)RS_THREADS * radix_keys(n_seg, keys);
  g.seg_len = seg_len;
  g.n_seg = n_seg;
  g.tiles_seg = (seg_len + g.tile - 1) / g.tile;
  if (g.tiles_seg == 0) g.tiles_seg = 1;
  int target = max(1, (RS_CTAS_PER_SM * num_sms + n_seg - 1) / n_seg);
  g.tiles_cta = (g.tiles_seg + target - 1) / target;
  g.ctas_seg = (int)((g.tiles_seg + g.tiles_cta - 1) / g.tiles_cta);
  return g;
}

// counts [n_seg][RS_RADIX][ctas_seg], then totals [n_seg][RS_RADIX]
size_t radix_scratch_bytes(int64_t seg_len, int n_seg, int num_sms, int keys) {
  SortGeom g = make_geom(seg_len, n_seg, num_sms, keys);
  return (size_t)n_seg * RS_RADIX * (g.ctas_seg + 1) * sizeof(uint32_t);
}

// Sorts each of n_seg segments of seg_len keys by bits [0, key_bits), ping-
// ponging between (keys_a, vals_a) and (keys_b, vals_b); *result_in_b tells
// which pair holds the result.  With identity_vals the first pass takes the
// in-segment index as the value instead of reading vals_a (vals_a is still
// used as a buffer by later passes).
cudaError_t radix_sort_pairs(cudaStream_t st, int num_sms, uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b,
                             uint32_t* vals_b, int64_t seg_len, int n_seg, int key_bits, bool identity_vals,
                             uint32_t* scratch, bool* result_in_b, int keys) {
  *result_in_b = false;
  if (seg_len == 0 || n_seg == 0) return cudaSuccess;
  SortGeom g = make_geom(seg_len, n_seg, num_sms, keys);
  const int kpt = radix_keys(n_seg, keys);
  int grid = g.ctas_seg * n_seg;
  int passes = (key_bits + 7) / 8;
  uint32_t *ki = keys_a, *vi = vals_a, *ko = keys_b, *vo = vals_b;
  for (int pass = 0; pass < passes; ++pass) {
    int shift = 8 * pass;
    const uint32_t dmask = radix_digit_mask(key_bits, shift);
    uint32_t* totals = scratch + (size_t)n_seg * RS_RADIX * g.ctas_seg;
    const uint32_t* vin = (pass == 0 && identity_vals) ? nullptr : vi;
    cudaError_t e = launch_serialised(k_rs_upsweep, dim3(grid), dim3(RS_THREADS), 0, st, (const uint32_t*)ki, g, shift,
                                      dmask, scratch);
    if (e == cudaSuccess)
      e = launch_serialised(k_rs_spine, dim3((n_seg * RS_RADIX + 7) / 8), dim3(256), 0, st, scratch, totals, g.ctas_seg,
                            n_seg * RS_RADIX);
    if (e == cudaSuccess) {
      auto down = kpt == 12 ? k_rs_downsweep<12> : kpt == 8 ? k_rs_downsweep<8> : k_rs_downsweep<6>;
      e = launch_serialised(down, dim3(grid), dim3(RS_THREADS), 0, st, (const uint32_t*)ki, vin, ko, vo, g, shift,
                            dmask, (const uint32_t*)scratch, (const uint32_t*)totals);
    }
    count_launches(3);
    if (e == cudaSuccess) e = cudaGetLastError();
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

// One pass (the digit of bits [shift, min(shift + 8, key_bits))) of the same radix sort over a single
// segment, reading (keys_in, vals_in) and writing (keys_out, vals_out);
// `counts` must hold radix_scratch_bytes(n, 1, num_sms) bytes.
cudaError_t radix_sort_pass(cudaStream_t st, int num_sms, const uint32_t* keys_in, const uint32_t* vals_in,
                            uint32_t* keys_out, uint32_t* vals_out, int64_t n, int shift, int key_bits,
                            uint32_t* counts) {
  if (n == 0) return cudaSuccess;
  SortGeom g = make_geom(n, 1, num_sms);
  const uint32_t dmask = radix_digit_mask(key_bits, shift);
  uint32_t* totals = counts + (size_t)RS_RADIX * g.ctas_seg;
  cudaError_t e =
      launch_serialised(k_rs_upsweep, dim3(g.ctas_seg), dim3(RS_THREADS), 0, st, keys_in, g, shift, dmask, counts);
  if (e == cudaSuccess)
    e = launch_serialised(k_rs_spine, dim3((RS_RADIX + 7) / 8), dim3(256), 0, st, counts, totals, g.ctas_seg, RS_RADIX);
  if (e == cudaSuccess)
    e = launch_serialised(k_rs_downsweep<RS_ITEMS>, dim3(g.ctas_seg), dim3(RS_THREADS), 0, st, keys_in, vals_in,
                          keys_out, vals_out, g, shift, dmask, (const uint32_t*)counts, (const uint32_t*)totals);
  count_launches(3);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

cudaError_t launch_count_gather(cudaStream_t st, int64_t total, int64_t n, const uint32_t* order,
                                const uint32_t* tiles_touched, uint32_t* counts_sorted, uint64_t* chunk_sums,
                                int64_t* n_chunks) {
  *n_chunks = (total + EM_CHUNK - 1) / EM_CHUNK;
  if (total == 0) return cudaSuccess;
  cudaError_t e = launch_serialised(k_count_gather, dim3((unsigned)*n_chunks), dim3(CG_THREADS), 0, st, total, n,
                                    order, tiles_touched, counts_sorted, chunk_sums);
  count_launches(1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_scan_spans(cudaStream_t st, uint64_t* sums, int64_t n_chunks, uint64_t* total_out,
                              uint64_t* sums2, uint64_t* total_out2) {
  cudaError_t e = launch_serialised(k_scan_spans, dim3(sums2 ? 2 : 1), dim3(SP_THREADS), 0, st, sums, sums2, n_chunks,
                                    total_out, total_out2);
  count_launches(1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// piece offsets [n_chunks + 1], then the piece -> chunk map [n_inst / piece + n_chunks + 1]
// (sized for the smallest piece, so that every run length fits)
size_t emit_piece_words(int64_t total, int64_t n_inst) {
  const int64_t n_chunks = (total + EM_CHUNK - 1) / EM_CHUNK;
  return (size_t)(2 * n_chunks + n_inst / EM_MIN_PIECE + 2);
}

template <int RUN>
static cudaError_t emit_launch(cudaStream_t st, int64_t total, int64_t n, const uint32_t* order,
                               const uint32_t* counts_sorted, const uint64_t* chunk_offsets, int64_t n_inst,
                               uint32_t* piece_off, const ProjRec* proj, const CamDev* cams, float alpha_min,
                               int64_t n_tiles, int cull, uint32_t* keys, uint32_t* vals) {
  constexpr uint32_t PIECE = EmitGeom<RUN>::PIECE;
  constexpr size_t SMEM = EmitGeom<RUN>::SMEM;
  const int64_t n_chunks = (total + EM_CHUNK - 1) / EM_CHUNK;
  // sum over chunks of ceil(count / piece) <= n_inst / piece + n_chunks; surplus CTAs return at once
  const int64_t grid = n_chunks + n_inst / PIECE + 1;
  uint32_t* piece_chunk = piece_off + n_chunks + 1;
  cudaError_t e = launch_serialised(k_emit_pieces<RUN>, dim3(1), dim3(SP_THREADS), 0, st, chunk_offsets, n_chunks,
                                    piece_off);
  if (e == cudaSuccess)
    e = launch_serialised(k_emit_piece_map, dim3((unsigned)((n_chunks + 255) / 256)), dim3(256), 0, st,
                          (const uint32_t*)piece_off, n_chunks, piece_chunk);
  if (e != cudaSuccess) return e;
  // the attribute is per device: set it once for each device this process uses
  static bool smem_set[kMaxDevicesAttr] = {};
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= kMaxDevicesAttr || !smem_set[dev]) {
    e = cudaFuncSetAttribute(k_emit<RUN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e == cudaSuccess)  // several CTAs per SM rather than the largest L1
      e = cudaFuncSetAttribute(k_emit<RUN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (dev < kMaxDevicesAttr) smem_set[dev] = true;
  }
  e = launch_serialised(k_emit<RUN>, dim3((unsigned)grid), dim3(EM_THREADS), SMEM, st, total, n, order,
                        counts_sorted, chunk_offsets, (const uint32_t*)piece_off, (const uint32_t*)piece_chunk,
                        n_chunks, proj, cams, log2f(alpha_min), n_tiles <= (1ll << 24), cull, keys, vals);
  count_launches(3);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_emit(cudaStream_t st, int64_t total, int64_t n, const uint32_t* order,
                        const uint32_t* counts_sorted, const uint64_t* chunk_offsets, int64_t n_inst,
                        uint32_t* piece_off, const ProjRec* proj, const CamDev* cams, float alpha_min,
                        int64_t n_tiles, int cull, int run, uint32_t* keys, uint32_t* vals) {
  if (total == 0 || n_inst == 0) return cudaSuccess;
  if (run == 4)
    return emit_launch<4>(st, total, n, order, counts_sorted, chunk_offsets, n_inst, piece_off, proj, cams,
                          alpha_min, n_tiles, cull, keys, vals);
  if (run == 16)
    return emit_launch<16>(st, total, n, order, counts_sorted, chunk_offsets, n_inst, piece_off, proj, cams,
                           alpha_min, n_tiles, cull, keys, vals);
  return emit_launch<8>(st, total, n, order, counts_sorted, chunk_offsets, n_inst, piece_off, proj, cams, alpha_min,
                        n_tiles, cull, keys, vals);
}

cudaError_t launch_tile_ranges(cudaStream_t st, int64_t n_inst, const uint32_t* keys, uint2* ranges) {
  if (n_inst == 0) return cudaSuccess;
  cudaError_t e = launch_serialised(k_tile_ranges, dim3((unsigned)((n_inst + 255) / 256)), dim3(256), 0, st, n_inst,
                                    keys, ranges);
  count_launches(1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace airgs
