// Warp-per-tile blend kernels with exact block culling (sm_103a).
//
// A 16x16 tile is split into eight 8x4 pixel blocks; block k (bx = k & 1,
// by = k >> 1) gives lane l the pixel (8 bx + (l & 7), 4 by + (l >> 3)).  A warp
// owns either the whole tile (eight blocks) or one half of it (four blocks,
// each half an independent work item, so twice the warps fit per SM).
// Most (pixel, Gaussian) pairs of a tile list cannot contribute: a Gaussian is
// listed for every tile its 3-sigma square touches, but it blends only where
// alpha = o G >= alpha_min, i.e. inside the ellipse
//     Q(d) = -log2(e) power(d) <= L,   L = log2(o / alpha_min).
// When a batch is staged, each Gaussian's axis-aligned bounding box of that
// ellipse (half-widths sqrt(L (M^-1)_xx), sqrt(L (M^-1)_yy) for Q = d^T M d),
// widened by a safety margin far above the single-precision error of the
// per-pair test, is intersected with the eight blocks; the warp then evaluates
// only the blocks the box meets, with warp-uniform branches.  Pairs in skipped
// blocks are pairs whose alpha is below alpha_min, which the definition skips:
// results are bit-identical to the unculled variants.  Blocks whose pixels
// all stopped (forward) or whose pixels' n_contrib lie behind the current list
// position (backward) are skipped the same way.
//
// Per-pixel arithmetic uses the exact-replay helpers of airgs_internal.cuh; the
// backward reduces each Gaussian's ten sums once per tile with the 20-shuffle
// transpose butterfly and three red.global.add.v4.f32.
//
// COMPACT (variant 6): staging keeps only the list entries whose block mask is
// non-zero (ballot + prefix count), so the serial walk over a batch touches
// useful entries only; the backward also folds the live-block test into the
// staging, and defers each Gaussian's ten sums (plus its blended-pair count)
// into a per-warp shared-memory table of three Gaussians, reduced by one
// column sum per lane (a transpose through shared memory) and flushed with one
// scalar red.global.add per sum.
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

constexpr int NG_TILE = 8;     // 8x4 blocks per tile
#ifndef AIRGS_CULL_FWD_BATCH
#define AIRGS_CULL_FWD_BATCH 32  // measured best of 16, 24, 32, 64, 96, 128
#endif
#ifndef AIRGS_CULL_BWD_BATCH
#define AIRGS_CULL_BWD_BATCH 32  // measured best of 32, 64, 96
#endif
constexpr int CBATCH = AIRGS_CULL_BWD_BATCH;  // records the backward stages per batch
constexpr int FBATCH = AIRGS_CULL_FWD_BATCH;  // the forward's batch (its live blocks are refreshed per batch)
constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ int cull_fetch(int* counter) {
  int it = 0;
  if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(kAll, it, 0);
}


// Tile bases of the views as 32-bit values (global tile ids stay below 2^30).
__device__ __forceinline__ int view_of_tile32(const int* tile_base, int n_views, int tile) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_base[mid] <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Per staged list entry, read back with one 16-byte load: position in the
// tile's full list plus one, block mask, third colour channel, Gaussian id.
struct __align__(16) StageMeta {
  uint32_t pos1;
  unsigned mask;
  float c;
  uint32_t id;
};

// The same search over the cameras' own tile bases (read through the cache).
__device__ __forceinline__ int view_of_tile_cams(const CamDev* cams, int n_views, int tile) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)__ldg(&cams[mid].tile_base) <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Stages the list entries [b0, b0 + nb) of a tile (or half-tile) item into
// shared memory, keeping only those whose block mask is non-zero, in list
// order; returns how many were kept.  With LIVE (the backward) the mask is also
// restricted to the blocks whose largest n_contrib (gmax) lies beyond the
// entry's position, and `past` is set when an entry lies at or beyond maxnc
// (positions increase along the list, so no later batch can contribute).
// Half-list entries: the forward computes each staged entry's exact block mask
// and stores it in the entry's top bits; the backward reads it from there (every
// entry before maxnc was staged by the forward of the same state).  Each lane
// adds to `groups` the blocks its kept entries will evaluate (mask & alive, the
// blocks not yet terminated at the batch's start), the issued-work statistic.
template <int NG, bool LIVE>
__device__ __forceinline__ int stage_compact(const BlendArgs& a, bool use_hl, uint32_t b0, int nb, uint32_t list0,
                                             const ProjRec* projv, float log2_amin, float X0, float Y0,
                                             const int (&gmax)[NG], int maxnc, unsigned alive, float4* s_a,
                                             float4* s_b, StageMeta* s_meta, bool& past, uint32_t& groups) {
  const int lane = threadIdx.x & 31;
  int kept = 0;
  bool beyond = false;
  for (int j0 = 0; j0 < nb; j0 += 32) {
    const int j = j0 + lane;
    unsigned msk = 0u;
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga;
    float gc = 0.f;
    uint32_t id = 0u, pos = 0u;
    if (j < nb) {
      bool have_mask = false;
      if (use_hl) {
        const uint2 en = a.hl[b0 + j];  // not through the read-only cache: the forward writes the masks
        id = en.x;
        pos = en.y & kHlPosMask;
        msk = en.y >> kHlMaskShift;
        have_mask = LIVE;  // the backward reads the forward's masks
      } else {
        id = __ldg(a.ids + b0 + j);
        pos = b0 + j - list0;
      }
      if (LIVE && (int)pos >= maxnc) {
        beyond = true;
        msk = 0u;
      } else {
        if (LIVE) {
          unsigned live = 0u;
#pragma unroll
          for (int k = 0; k < NG; ++k) live |= ((int)pos < gmax[k] ? 1u : 0u) << k;
          msk = have_mask ? (msk & live) : live;
        } else if (!have_mask) {
          msk = (1u << NG) - 1u;
        }
        if (msk) {
          const ProjRec* r = projv + id;
          ga = __ldg(&r->a);
          gb = __ldg(&r->b);
          gc = __ldg(&r->c.x);
          if (!have_mask) msk &= block_mask_exact(ga, gb, log2_amin, X0, Y0, (1u << NG) - 1u);
        }
        if (!LIVE && use_hl) a.hl_mut[b0 + j].y = pos | (msk << kHlMaskShift);
      }
    }
    const unsigned bal = __ballot_sync(kAll, msk != 0u);
    if (msk) {
      const int d = kept + __popc(bal & ((1u << lane) - 1u));
      s_a[d] = ga;
      s_b[d] = gb;
      s_meta[d] = StageMeta{pos + 1u, msk, gc, id};
      groups += __popc(msk & alive);
    }
    kept += __popc(bal);
  }
  if (LIVE && __any_sync(kAll, beyond)) past = true;
  __syncwarp();
  return kept;
}

// ------------------------------------------------------------------ forward
// NG blocks per warp: 8 = the whole tile, 4 = one half (rows 8h .. 8h+7) of it,
// so that two warps with half the per-lane state share a tile independently.
#ifndef AIRGS_CULL_FWD_MINB
#define AIRGS_CULL_FWD_MINB 32  // 64 registers: the 32-block limit of 32-thread CTAs
#endif
template <int NG, bool IMP, bool COMPACT>
__global__ void __launch_bounds__(32, COMPACT ? AIRGS_CULL_FWD_MINB : 1) k_blend_fwd_cull(BlendArgs a, FwdOut out) {
  constexpr int PARTS = NG_TILE / NG;
  __shared__ float4 s_a[FBATCH];
  __shared__ float4 s_b[FBATCH];
  __shared__ StageMeta s_meta[FBATCH];
  __shared__ int s_tile_base[COMPACT ? 1 : AIRGS_MAX_VIEWS_DEV];  // COMPACT reads the bases from the cameras

  const int lane = threadIdx.x;
  if (!COMPACT)
    for (int v = lane; v < a.n_views; v += 32) s_tile_base[v] = (int)a.cams[v].tile_base;
  __syncwarp();
  const float alpha_max = a.rp.alpha_max, alpha_min = a.rp.alpha_min, T_min = a.rp.T_min;
  const float log2_amin = log2f(alpha_min);
  const int lx = lane & 7, ly = lane >> 3;
  unsigned long long pairs = 0, executed = 0;

  while (true) {
    const int work = cull_fetch(a.work_counter);
    if (work >= a.n_tiles * PARTS) break;
    const int item = work / PARTS, part = work % PARTS;
    const int v = COMPACT ? view_of_tile_cams(a.cams, a.n_views, item) : view_of_tile32(s_tile_base, a.n_views, item);
    const CamDev& cam = a.cams[v];
    const int lt = item - (COMPACT ? (int)__ldg(&a.cams[v].tile_base) : s_tile_base[v]);
    const int X0 = (lt % cam.TW) * kTile, Y0 = (lt / cam.TW) * kTile + part * (kTile / PARTS);
    const float pxb[2] = {(float)(X0 + lx) + 0.5f, (float)(X0 + 8 + lx) + 0.5f};
    float pyb[NG / 2];  // pixel-centre rows of the item's block rows
#pragma unroll
    for (int by = 0; by < NG / 2; ++by) pyb[by] = (float)(Y0 + 4 * by + ly) + 0.5f;
    float T[NG], C2[NG];
    float2 C01[NG];  // the first two colour channels, updated as one packed FMA
    // last: position + 1 of the last blended entry; stop_at: -1 while the pixel
    // is blending, else position + 1 of the entry that stopped it (0 for a pixel
    // outside the image)
    int last[NG], stop_at[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int x = X0 + 8 * (k & 1) + lx, y = Y0 + 4 * (k >> 1) + ly;
      T[k] = 1.f;
      C01[k] = make_float2(0.f, 0.f);
      C2[k] = 0.f;
      last[k] = 0;
      stop_at[k] = (x < cam.W && y < cam.H) ? -1 : 0;
    }
    const uint2 range = a.ranges[item];
    const bool use_hl = PARTS > 1 && a.hl != nullptr;  // this half's compacted list
    uint2 er = range;
    if (use_hl) er = a.hranges[(int64_t)part * a.n_tiles + item];
    const ProjRec* projv = a.proj + (size_t)v * a.n;
    uint32_t exec_groups = 0;  // warp-uniform (per-entry count) or per lane (COMPACT: counted while staging)

    for (uint32_t b0 = er.x; b0 < er.y; b0 += FBATCH) {
      unsigned live = 0;
#pragma unroll
      for (int k = 0; k < NG; ++k)
        if (__any_sync(kAll, stop_at[k] < 0)) live |= 1u << k;
      if (live == 0) break;
      int nb = (int)min((uint32_t)FBATCH, er.y - b0);
      if (COMPACT) {
        const int none[NG] = {};
        bool unused = false;
        nb = stage_compact<NG, false>(a, use_hl, b0, nb, range.x, projv, log2_amin, (float)X0, (float)Y0, none, 0,
                                      live, s_a, s_b, s_meta, unused, exec_groups);
      } else
      for (int j = lane; j < nb; j += 32) {
        uint32_t id, pos;
        if (use_hl) {
          const uint2 en = __ldg(a.hl + b0 + j);
          id = en.x;
          pos = en.y & kHlPosMask;
        } else {
          id = __ldg(a.ids + b0 + j);
          pos = b0 + j - range.x;
        }
        const ProjRec* r = projv + id;
        const float4 ga = __ldg(&r->a), gb = __ldg(&r->b);
        s_a[j] = ga;
        s_b[j] = gb;
        s_meta[j] = StageMeta{pos + 1u, block_mask(ga, gb, log2_amin, (float)X0, (float)Y0) & ((1u << NG) - 1u),
                              __ldg(&r->c.x), id};
      }
      __syncwarp();
      for (int j = 0; j < nb; ++j) {
        const StageMeta me = s_meta[j];
        const unsigned m = me.mask & live;
        if (m == 0) continue;
        if (!COMPACT) exec_groups += __popc(m);
        const float4 ga = s_a[j];
        const float4 gb = s_b[j];
        const float cb = me.c;
        const int pos1 = (int)me.pos1;
        const float dxb[2] = {__fsub_rn(ga.x, pxb[0]), __fsub_rn(ga.x, pxb[1])};
        float wsum = 0.f;
        int bcount = 0;
#pragma unroll
        for (int by = 0; by < NG / 2; ++by) {
          if (!((m >> (2 * by)) & 3u)) continue;  // warp-uniform
          float dy, b2dy, c2dy2;  // shared by the row's two blocks
          row_terms(ga.y, pyb[by], ga.w, gb.x, dy, b2dy, c2dy2);
#pragma unroll
        for (int bx = 0; bx < 2; ++bx) {
          const int k = 2 * by + bx;
          if (!((m >> k) & 1u)) continue;  // warp-uniform
          const float dx = dxb[bx];
          const float p2 = power2_of(dx, ga.z, b2dy, c2dy2);
          const float G = ex2_approx(p2);
          const float alpha = alpha_of(gb.y, G, alpha_max);
          const float Tn = transmit(T[k], alpha);
          const bool valid = (stop_at[k] < 0) && !(p2 > 0.f) && !(alpha < alpha_min);
          const bool stop = valid && (Tn < T_min);
          const bool blend = valid && !stop;
          const float w = __fmul_rn(alpha, T[k]);
          if (blend) {
            C01[k] = __ffma2_rn(make_float2(gb.z, gb.w), make_float2(w, w), C01[k]);
            C2[k] = __fmaf_rn(cb, w, C2[k]);
            T[k] = Tn;
            last[k] = pos1;
          }
          if (stop) stop_at[k] = pos1;
          if (IMP) {
            wsum += blend ? w : 0.f;
            bcount += blend ? 1 : 0;
          }
        }
        }
        if (IMP) {
          if (__any_sync(kAll, bcount > 0)) {
            float s = wsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kAll, s, o);
            const int c = __reduce_add_sync(kAll, bcount);
            if (lane == 0) {
              atomicAdd(out.imp_w + me.id, s);
              atomicAdd(out.imp_cnt + me.id, (uint32_t)c);
            }
          }
        }
      }
      __syncwarp();
    }
    executed += (COMPACT ? 1ull : 32ull) * exec_groups;
    const int64_t HW = (int64_t)cam.W * cam.H;
    float* rgb = out.rgb + 3 * cam.pix_base;
    const uint32_t len = range.y - range.x;
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int x = X0 + 8 * (k & 1) + lx, y = Y0 + 4 * (k >> 1) + ly;
      if (x < cam.W && y < cam.H) {
        // pairs of the definition: list entries up to and including the stop
        pairs += stop_at[k] > 0 ? (unsigned long long)stop_at[k] : (unsigned long long)len;
        const int64_t pix = (int64_t)y * cam.W + x;
        rgb[pix] = __fmaf_rn(T[k], a.rp.bg[0], C01[k].x);
        rgb[HW + pix] = __fmaf_rn(T[k], a.rp.bg[1], C01[k].y);
        rgb[2 * HW + pix] = __fmaf_rn(T[k], a.rp.bg[2], C2[k]);
        if (out.T) out.T[cam.pix_base + pix] = T[k];
        out.ncontrib[cam.pix_base + pix] = last[k];
        if (out.ncontrib_user) out.ncontrib_user[cam.pix_base + pix] = last[k];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kAll, pairs, o);
  if (COMPACT) {  // per-lane block counts: 32 lane evaluations per block
    for (int o = 16; o > 0; o >>= 1) executed += __shfl_xor_sync(kAll, executed, o);
    executed *= 32ull;
  }
  if (lane == 0) {
    if (pairs) {
      atomicAdd(a.pair_counter, pairs);
      if (a.pair_total) atomicAdd(a.pair_total, pairs);
    }
    if (a.exec_total && executed) atomicAdd(a.exec_total, executed);
  }
}

// ------------------------------------------------------------------ 16 -> 4 transpose reduction
__device__ __forceinline__ void cull_reduce16_to4(float (&v)[16], int lane) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool up = lane & 16;
    const float send = up ? v[k] : v[k + 8];
    const float keep = up ? v[k + 8] : v[k];
    v[k] = keep + __shfl_xor_sync(kAll, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = lane & 8;
    const float send = up ? v[k] : v[k + 4];
    const float keep = up ? v[k + 4] : v[k];
    v[k] = keep + __shfl_xor_sync(kAll, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 4;
    const float send = up ? v[k] : v[k + 2];
    const float keep = up ? v[k + 2] : v[k];
    v[k] = keep + __shfl_xor_sync(kAll, send, 4);
  }
  v[0] += __shfl_xor_sync(kAll, v[0], 1);
  v[1] += __shfl_xor_sync(kAll, v[1], 1);
  v[0] += __shfl_xor_sync(kAll, v[0], 2);
  v[1] += __shfl_xor_sync(kAll, v[1], 2);
  v[2] = __shfl_xor_sync(kAll, v[0], 4);
  v[3] = __shfl_xor_sync(kAll, v[1], 4);
}


// Deferred per-Gaussian reduction of the backward (COMPACT): rows 10 f + q of
// the table hold, per lane (column), sum q of the f-th deferred Gaussian,
//   0 S_x = sum t dx, 1 S_y = sum t dy, 2 sum t dx^2, 3 sum t dx dy, 4 sum t dy^2,
//   5 sum t, 6-8 colour, 9 blend weight,   t = dL/dalpha G on unclamped pairs,
// so that with power2 = a2 dx^2 + b2 dx dy + c2 dy^2 and dL/dpower = o t the
// mean gradient is o (2 a2 S_x + b2 S_y, b2 S_x + 2 c2 S_y) (times ln 2); row
// 30 holds the lanes' blended-pair counts of the three Gaussians packed in 8-bit
// fields (at most 4 pixels per lane and 128 per half tile, so the packed sums
// are integers below 2^24 and exact in single precision).  Lane s sums row s
// with eight 16-byte loads (rows padded to 36 floats: each 8-lane phase of a
// 16-byte load touches 32 different banks) and sends it with one scalar
// reduction.
constexpr int kDeferG = 3;
constexpr int kRedStride = 36;  // row stride (floats): 16-byte rows, conflict-free 8-lane phases of LDS.128

template <bool IMP>
__device__ __forceinline__ void flush_deferred(float (*s_red)[kRedStride], const uint32_t* s_fid, const float4* s_fcon,
                                               int nf,
                                               uint32_t cpack, GradRec* gradv, const BwdIn& in, int lane) {
  if (IMP) s_red[30][lane] = (float)cpack;
  __syncwarp();
  const int row = lane < 31 ? lane : 30;
  const float4* rp = reinterpret_cast<const float4*>(&s_red[row][0]);
  float4 s = rp[0];
  float2 s01 = make_float2(s.x, s.y), s23 = make_float2(s.z, s.w);
#pragma unroll
  for (int i = 1; i < 8; ++i) {  // column sums as packed FP32x2 additions
    const float4 u = rp[i];
    s01 = __fadd2_rn(s01, make_float2(u.x, u.y));
    s23 = __fadd2_rn(s23, make_float2(u.z, u.w));
  }
  const float2 s4 = __fadd2_rn(s01, s23);
  const float sum = s4.x + s4.y;
  const float other = __shfl_xor_sync(kAll, sum, 1);  // S_y for the S_x lane and vice versa
  const int f = lane / 10, q = lane - 10 * f;
  if (lane < 10 * nf && (IMP || q < 9)) {
    // GradRec floats 0-8: mean2d, conic A (x -1/2), B (x -1), C (x -1/2), opacity,
    // colour; sum 9 (the blend weight) goes to the importance weights.  One
    // branch-free coefficient pair per lane: value = ca sum + cb other.
    const uint32_t id = s_fid[f];
    const float4 cf = s_fcon[f];  // (a2, b2, c2, o)
    const float o = cf.w, lo = kLn2 * cf.w;
    const float ca = q == 0 ? 2.f * lo * cf.x : q == 1 ? 2.f * lo * cf.z : q == 3 ? -o : q < 5 ? -0.5f * o : 1.f;
    const float cb = q < 2 ? lo * cf.y : 0.f;
    const float val = fmaf(ca, sum, cb * other);
    float* dst = q < 9 ? reinterpret_cast<float*>(gradv + id) + q : in.imp_w + id;
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(dst), "f"(val) : "memory");
  }
  if (IMP) {
    const uint32_t packed = (uint32_t)__shfl_sync(kAll, sum, 30);
    if (lane < nf) {
      const uint32_t c = (packed >> (8 * lane)) & 0xFFu;
      asm volatile("red.global.add.u32 [%0], %1;" ::"l"(in.imp_cnt + s_fid[lane]), "r"(c) : "memory");
    }
  }
  __syncwarp();  // the table is refilled after this
}

// ------------------------------------------------------------------ backward
// Sums per (tile, Gaussian), scaled when flushed (see blend_warp.cu):
//   0 mx (x ln2), 1 my (x ln2), 2 A (x -1/2), 3 B (x -1), 4 C (x -1/2),
//   5 opacity, 6-8 colour, 9 blend weight.
#ifndef AIRGS_CULL_BWD_MINB
#define AIRGS_CULL_BWD_MINB 28  // 72 registers: 28 warps per SM (measured best of 20, 24, 26, 28, 30, 32)
#endif
template <int NG, bool L1, bool IMP, bool COMPACT>
__global__ void __launch_bounds__(32, COMPACT ? AIRGS_CULL_BWD_MINB : 1) k_blend_bwd_cull(BlendArgs a, BwdIn in) {
  constexpr int PARTS = NG_TILE / NG;
  static_assert(!COMPACT || NG * 32 < 256, "packed 8-bit pair counts");
  __shared__ __align__(16) float s_red[COMPACT ? 31 : 1][kRedStride];
  __shared__ uint32_t s_fid[kDeferG];
  __shared__ float4 s_fcon[kDeferG];  // (a2, b2, c2, o) of the deferred Gaussians
  __shared__ float4 s_a[CBATCH];
  __shared__ float4 s_b[CBATCH];
  __shared__ StageMeta s_meta[CBATCH];
  __shared__ int s_tile_base[COMPACT ? 1 : AIRGS_MAX_VIEWS_DEV];  // COMPACT reads the bases from the cameras

  const int lane = threadIdx.x;
  if (!COMPACT)
    for (int v = lane; v < a.n_views; v += 32) s_tile_base[v] = (int)a.cams[v].tile_base;
  __syncwarp();
  const float alpha_max = a.rp.alpha_max, alpha_min = a.rp.alpha_min;
  const float log2_amin = log2f(alpha_min);
  const int lx = lane & 7, ly = lane >> 3;
  unsigned long long pairs = 0, executed = 0;
  float loss_acc = 0.f;

  while (true) {
    const int work = cull_fetch(a.work_counter);
    if (work >= a.n_tiles * PARTS) break;
    const int item = work / PARTS, part = work % PARTS;
    const int v = COMPACT ? view_of_tile_cams(a.cams, a.n_views, item) : view_of_tile32(s_tile_base, a.n_views, item);
    const CamDev& cam = a.cams[v];
    const int lt = item - (COMPACT ? (int)__ldg(&a.cams[v].tile_base) : s_tile_base[v]);
    const int X0 = (lt % cam.TW) * kTile, Y0 = (lt / cam.TW) * kTile + part * (kTile / PARTS);
    const float pxb[2] = {(float)(X0 + lx) + 0.5f, (float)(X0 + 8 + lx) + 0.5f};
    float pyb[NG / 2];  // pixel-centre rows of the item's block rows
#pragma unroll
    for (int by = 0; by < NG / 2; ++by) pyb[by] = (float)(Y0 + 4 * by + ly) + 0.5f;
    const int64_t HW = (int64_t)cam.W * cam.H;
    const int64_t base3 = 3 * cam.pix_base;

    float T[NG], gP[NG], gC[NG], g0[NG], g1[NG], g2[NG];
    int nc[NG], gmax[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int x = X0 + 8 * (k & 1) + lx, y = Y0 + 4 * (k >> 1) + ly;
      T[k] = 1.f;
      gP[k] = 0.f;
      g0[k] = g1[k] = g2[k] = gC[k] = 0.f;
      nc[k] = 0;
      if (x < cam.W && y < cam.H) {
        const int64_t pix = (int64_t)y * cam.W + x;
        float cf[3], gg[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          cf[ch] = in.rgb[base3 + ch * HW + pix];
          if (L1) {
            const float d = cf[ch] - in.target[base3 + ch * HW + pix];
            gg[ch] = d > 0.f ? in.inv_norm : (d < 0.f ? -in.inv_norm : 0.f);
            loss_acc += fabsf(d);
          } else {
            gg[ch] = in.dL[base3 + ch * HW + pix];
          }
        }
        g0[k] = gg[0];
        g1[k] = gg[1];
        g2[k] = gg[2];
        gC[k] = gg[0] * cf[0] + gg[1] * cf[1] + gg[2] * cf[2];
        nc[k] = in.ncontrib[cam.pix_base + pix];
        pairs += (unsigned long long)nc[k];
      }
      gmax[k] = (int)__reduce_max_sync(kAll, (unsigned)nc[k]);  // warp-uniform
    }
    int maxnc = 0;
#pragma unroll
    for (int k = 0; k < NG; ++k) maxnc = max(maxnc, gmax[k]);
    const uint2 range = a.ranges[item];
    const bool use_hl = PARTS > 1 && a.hl != nullptr;  // this half's compacted list
    uint2 er = make_uint2(range.x, range.x + (uint32_t)maxnc);
    if (use_hl) er = a.hranges[(int64_t)part * a.n_tiles + item];
    const ProjRec* projv = a.proj + (size_t)v * a.n;
    GradRec* gradv = in.grad + (size_t)v * a.n;
    uint32_t exec_groups = 0;
    bool past_end = false;
    int ns = 0;          // deferred Gaussians in the table (COMPACT)
    uint32_t cpack = 0;  // this lane's packed pair counts of those

    for (uint32_t b0 = er.x; b0 < er.y && !past_end; b0 += CBATCH) {
      int nb = (int)min((uint32_t)CBATCH, er.y - b0);
      if (COMPACT) {
        nb = stage_compact<NG, true>(a, use_hl, b0, nb, range.x, projv, log2_amin, (float)X0, (float)Y0, gmax, maxnc,
                                     (1u << NG) - 1u, s_a, s_b, s_meta, past_end, exec_groups);
      } else
      for (int j = lane; j < nb; j += 32) {
        uint32_t id, pos;
        if (use_hl) {
          const uint2 en = __ldg(a.hl + b0 + j);
          id = en.x;
          pos = en.y & kHlPosMask;
        } else {
          id = __ldg(a.ids + b0 + j);
          pos = b0 + j - range.x;
        }
        const ProjRec* r = projv + id;
        const float4 ga = __ldg(&r->a), gb = __ldg(&r->b);
        s_a[j] = ga;
        s_b[j] = gb;
        s_meta[j] = StageMeta{pos + 1u, block_mask(ga, gb, log2_amin, (float)X0, (float)Y0) & ((1u << NG) - 1u),
                              __ldg(&r->c.x), id};
      }
      __syncwarp();
      for (int j = 0; j < nb; ++j) {
        const StageMeta me = s_meta[j];
        const int pos1 = (int)me.pos1;  // pair (pixel, entry) replayed iff pos1 <= n_contrib
        unsigned m = me.mask;
        if (!COMPACT) {
          if (pos1 > maxnc) {  // positions increase along the list
            past_end = true;
            break;
          }
          unsigned live = 0;
#pragma unroll
          for (int k = 0; k < NG; ++k) live |= (pos1 <= gmax[k] ? 1u : 0u) << k;
          m &= live;
          if (m == 0) continue;
          exec_groups += __popc(m);
        }
        const float4 ga = s_a[j];
        const float4 gb = s_b[j];
        const float cb = me.c;
        const float dxb[2] = {__fsub_rn(ga.x, pxb[0]), __fsub_rn(ga.x, pxb[1])};
        const float twoa2 = 2.f * ga.z;
        float acc[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = 0.f;
        int cnt = 0;
        if (!COMPACT) {
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          if (!((m >> k) & 1u)) continue;  // warp-uniform
          const float py = (float)(Y0 + 4 * (k >> 1) + ly) + 0.5f;
          float dy, b2dy, c2dy2;
          row_terms(ga.y, py, ga.w, gb.x, dy, b2dy, c2dy2);
          const float dx = dxb[k & 1];
          const float p2 = power2_of(dx, ga.z, b2dy, c2dy2);
          const float G = ex2_approx(p2);
          const float oG = __fmul_rn(gb.y, G);
          const float alpha = alpha_of(gb.y, G, alpha_max);
          const bool valid = (pos1 <= nc[k]) && !(p2 > 0.f) && !(alpha < alpha_min);
          const float ae = valid ? alpha : 0.f;
          const bool graded = valid && (oG <= alpha_max);
          const float w = __fmul_rn(ae, T[k]);
          const float gc = g0[k] * gb.z + g1[k] * gb.w + g2[k] * cb;
          acc[6] = fmaf(w, g0[k], acc[6]);
          acc[7] = fmaf(w, g1[k], acc[7]);
          acc[8] = fmaf(w, g2[k], acc[8]);
          gP[k] = fmaf(gc, w, gP[k]);
          const float om = __fsub_rn(1.0f, ae);
          const float dL_dalpha = T[k] * gc - __fdividef(gC[k] - gP[k], om);
          T[k] = __fmul_rn(T[k], om);
          const float dL_dpow = graded ? dL_dalpha * alpha : 0.f;
          acc[5] = fmaf(dL_dalpha, graded ? G : 0.f, acc[5]);
          acc[2] = fmaf(dL_dpow, dx * dx, acc[2]);
          acc[3] = fmaf(dL_dpow, dx * dy, acc[3]);
          acc[4] = fmaf(dL_dpow, dy * dy, acc[4]);
          acc[0] = fmaf(dL_dpow, fmaf(twoa2, dx, b2dy), acc[0]);
          acc[1] = fmaf(dL_dpow, fmaf(ga.w, dx, 2.f * gb.x * dy), acc[1]);
          if (IMP) acc[9] += w;
          cnt += valid ? 1 : 0;
        }
        } else {
        float2 a01 = make_float2(0.f, 0.f), a24 = a01, a67 = a01;
#pragma unroll
        for (int by = 0; by < NG / 2; ++by) {
          if (!((m >> (2 * by)) & 3u)) continue;  // warp-uniform
          float dy, b2dy, c2dy2;  // shared by the row's two blocks
          row_terms(ga.y, pyb[by], ga.w, gb.x, dy, b2dy, c2dy2);
#pragma unroll
        for (int bx = 0; bx < 2; ++bx) {
          const int k = 2 * by + bx;
          if (!((m >> k) & 1u)) continue;  // warp-uniform
          const float dx = dxb[bx];
          const float p2 = power2_of(dx, ga.z, b2dy, c2dy2);
          const float G = ex2_approx(p2);
          const float oG = __fmul_rn(gb.y, G);
          const float alpha = alpha_of(gb.y, G, alpha_max);
          const bool valid = (pos1 <= nc[k]) && !(p2 > 0.f) && !(alpha < alpha_min);
          const float ae = valid ? alpha : 0.f;
          const bool graded = valid && (oG <= alpha_max);
          const float w = __fmul_rn(ae, T[k]);
          const float gc = g0[k] * gb.z + g1[k] * gb.w + g2[k] * cb;
          // independent sums in pairs: one packed FP32x2 operation each
          a67 = __ffma2_rn(make_float2(w, w), make_float2(g0[k], g1[k]), a67);
          acc[8] = fmaf(w, g2[k], acc[8]);
          // gC[k] holds the colour still ahead of the replay, R = gC - gP
          gC[k] = fmaf(-gc, w, gC[k]);
          const float om = __fsub_rn(1.0f, ae);
          const float dL_dalpha = T[k] * gc - __fdividef(gC[k], om);
          T[k] = __fmul_rn(T[k], om);
          // t = dL/dalpha G on unclamped pairs; dL/dpower = o t, o applied at the flush
          const float tt = dL_dalpha * (graded ? G : 0.f);
          acc[5] += tt;
          const float2 d2 = make_float2(dx, dy);
          const float2 td = __fmul2_rn(make_float2(tt, tt), d2);  // (t dx, t dy)
          a01 = __fadd2_rn(a01, td);
          a24 = __ffma2_rn(td, d2, a24);                           // (t dx^2, t dy^2)
          acc[3] = fmaf(td.x, dy, acc[3]);
          if (IMP) acc[9] += w;
          cnt += valid ? 1 : 0;
        }
        }
        acc[0] = a01.x;
        acc[1] = a01.y;
        acc[2] = a24.x;
        acc[4] = a24.y;
        acc[6] = a67.x;
        acc[7] = a67.y;
        }
        if (COMPACT) {
          {  // every compacted entry has a live block: defer without a vote
#pragma unroll
            for (int q = 0; q < 10; ++q) s_red[ns * 10 + q][lane] = acc[q];
            if (IMP) cpack += (uint32_t)cnt << (8 * ns);
            // every lane stores the same values (one shared-memory word each, no branch)
            s_fid[ns] = me.id;
            s_fcon[ns] = make_float4(ga.z, ga.w, gb.x, gb.y);
            if (++ns == kDeferG) {
              flush_deferred<IMP>(s_red, s_fid, s_fcon, ns, cpack, gradv, in, lane);
              ns = 0;
              cpack = 0;
            }
          }
        } else if (__any_sync(kAll, cnt > 0)) {
          float vals[16];
#pragma unroll
          for (int q = 0; q < 10; ++q) vals[q] = acc[q];
#pragma unroll
          for (int q = 10; q < 16; ++q) vals[q] = 0.f;
          cull_reduce16_to4(vals, lane);
          const uint32_t id = me.id;
          float* gr = reinterpret_cast<float*>(gradv + id);
          if (lane == 0) red_add_v4(gr, vals[0] * kLn2, vals[1] * kLn2, -0.5f * vals[2], -vals[3]);
          if (lane == 8) red_add_v4(gr + 4, -0.5f * vals[0], vals[1], vals[2], vals[3]);
          if (lane == 16) {
            red_add_v4(gr + 8, vals[0], 0.f, 0.f, 0.f);
            if (IMP && vals[1] != 0.f) atomicAdd(in.imp_w + id, vals[1]);
          }
          if (IMP) {
            const int c = __reduce_add_sync(kAll, cnt);
            if (lane == 0 && c) atomicAdd(in.imp_cnt + id, (uint32_t)c);
          }
        }
      }
      __syncwarp();
    }
    if (COMPACT && ns > 0) flush_deferred<IMP>(s_red, s_fid, s_fcon, ns, cpack, gradv, in, lane);
    executed += (COMPACT ? 1ull : 32ull) * exec_groups;
  }
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kAll, pairs, o);
  if (COMPACT) {  // per-lane block counts: 32 lane evaluations per block
    for (int o = 16; o > 0; o >>= 1) executed += __shfl_xor_sync(kAll, executed, o);
    executed *= 32ull;
  }
  if (lane == 0) {
    if (pairs) {
      atomicAdd(a.pair_counter, pairs);
      if (a.pair_total) atomicAdd(a.pair_total, pairs);
    }
    if (a.exec_total && executed) atomicAdd(a.exec_total, executed);
  }
  if (L1 && in.loss) {
    for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(kAll, loss_acc, o);
    if (lane == 0) atomicAdd(in.loss, loss_acc * in.inv_norm);
  }
}

// ------------------------------------------------------------------ launchers
template <class K>
static int cull_grid(K kernel, int num_sms, int64_t items, cudaError_t& e) {
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 32, 0);
  int64_t g = (int64_t)(occ > 0 ? occ : 1) * num_sms;
  return (int)(items < g ? items : g);
}

// Shared memory is carved out to the maximum once per kernel, so that the
// occupancy the register count allows is not cut by the per-warp tables.
template <class K>
static cudaError_t prefer_shared(K kernel) {
  static bool done[kMaxDevicesAttr] = {};  // per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < kMaxDevicesAttr && done[dev]) return cudaSuccess;
  if (dev < kMaxDevicesAttr) done[dev] = true;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

template <int NG, bool IMP, bool COMPACT>
static cudaError_t fwd_cull(cudaStream_t st, int num_sms, const BlendArgs& a, const FwdOut& o) {
  cudaError_t e = prefer_shared(k_blend_fwd_cull<NG, IMP, COMPACT>);
  if (e != cudaSuccess) return e;
  int grid = cull_grid(k_blend_fwd_cull<NG, IMP, COMPACT>, num_sms, a.n_tiles * (NG_TILE / NG), e);
  if (e != cudaSuccess) return e;
  if (grid > 0) k_blend_fwd_cull<NG, IMP, COMPACT><<<grid, 32, 0, st>>>(a, o);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_blend_fwd_cull(cudaStream_t st, int num_sms, int blocks_per_warp, bool compact, const BlendArgs& a,
                                  const FwdOut& o) {
  const bool imp = o.imp_w != nullptr;
  if (compact)
    return imp ? fwd_cull<4, true, true>(st, num_sms, a, o) : fwd_cull<4, false, true>(st, num_sms, a, o);
  if (blocks_per_warp == 4)
    return imp ? fwd_cull<4, true, false>(st, num_sms, a, o) : fwd_cull<4, false, false>(st, num_sms, a, o);
  return imp ? fwd_cull<8, true, false>(st, num_sms, a, o) : fwd_cull<8, false, false>(st, num_sms, a, o);
}

template <int NG, bool L1, bool IMP, bool COMPACT>
static cudaError_t bwd_cull(cudaStream_t st, int num_sms, const BlendArgs& a, const BwdIn& in) {
  cudaError_t e = prefer_shared(k_blend_bwd_cull<NG, L1, IMP, COMPACT>);
  if (e != cudaSuccess) return e;
  int grid = cull_grid(k_blend_bwd_cull<NG, L1, IMP, COMPACT>, num_sms, a.n_tiles * (NG_TILE / NG), e);
  if (e != cudaSuccess) return e;
  if (grid > 0) k_blend_bwd_cull<NG, L1, IMP, COMPACT><<<grid, 32, 0, st>>>(a, in);
  count_launches(1);
  return cudaGetLastError();
}

template <int NG, bool COMPACT>
static cudaError_t bwd_cull_dispatch(cudaStream_t st, int num_sms, const BlendArgs& a, const BwdIn& in) {
  const bool l1 = in.target != nullptr, imp = in.imp_w != nullptr;
  if (l1)
    return imp ? bwd_cull<NG, true, true, COMPACT>(st, num_sms, a, in)
               : bwd_cull<NG, true, false, COMPACT>(st, num_sms, a, in);
  return imp ? bwd_cull<NG, false, true, COMPACT>(st, num_sms, a, in)
             : bwd_cull<NG, false, false, COMPACT>(st, num_sms, a, in);
}

cudaError_t launch_blend_bwd_cull(cudaStream_t st, int num_sms, int blocks_per_warp, bool compact, const BlendArgs& a,
                                  const BwdIn& in) {
  if (compact) return bwd_cull_dispatch<4, true>(st, num_sms, a, in);
  if (blocks_per_warp == 4) return bwd_cull_dispatch<4, false>(st, num_sms, a, in);
  return bwd_cull_dispatch<8, false>(st, num_sms, a, in);
}

}  // namespace airgs
