// Shared pieces of the blend kernels (sm_103a): the work queue, the view of a
// global tile, and the compacted staging of a half tile's list entries.
//
// A 16x16 tile is split into two 16x8 halves, each an independent work item of
// one warp, and a half into four 8x4 pixel blocks; block k (bx = k & 1,
// by = k >> 1) gives lane l the pixel (8 bx + (l & 7), 4 by + (l >> 3)).  Most
// (pixel, Gaussian) pairs of a tile list cannot contribute: a Gaussian is
// listed for every tile its 3-sigma square touches, but it blends only where
// alpha = o G >= alpha_min, i.e. inside the ellipse
//     Q(d) = -log2(e) power(d) <= L,   L = log2(o / alpha_min).
// Staging tests every list entry against the four blocks (block_mask_exact:
// the bounding box of that ellipse, then the quadratic's maximum over each
// block's pixel-centre rectangle, with a margin far above the single-precision
// error of the per-pair test) and keeps, in list order, only the entries with a
// non-zero block mask, so the serial walk over a batch touches useful entries
// only.  Pairs in skipped blocks have alpha below alpha_min, which the
// definition skips: results are bit-identical to walking every entry.
#pragma once

#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

constexpr unsigned kAll = 0xffffffffu;
constexpr int kBlocks = 4;  // 8x4 blocks per half tile

__device__ __forceinline__ int cull_fetch(int* counter) {
  int it = 0;
  if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(kAll, it, 0);
}

// The work item at queue position q (< the item count): through the queue
// order when there is one (every lane reads the same word).
__device__ __forceinline__ int queue_item(const uint32_t* order, int q) { return order ? (int)__ldg(order + q) : q; }

// View that owns a global tile id, from the cameras' tile bases (read through
// the read-only cache).
__device__ __forceinline__ int view_of_tile_cams(const CamDev* cams, int n_views, int tile) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)__ldg(&cams[mid].tile_base) <= tile) lo = mid;
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

// Stages the list entries [b0, b0 + nb) of a half-tile item into shared memory,
// keeping only those whose block mask is non-zero, in list order; returns how
// many were kept.  With LIVE (the backward) the mask is also restricted to the
// blocks whose largest n_contrib (gmax, in shared memory) lies beyond the
// entry's position, and `past` is set when an entry lies at or beyond maxnc
// (positions increase along the list, so no later batch can contribute).  Without
// LIVE (the forward) the exact test covers only the blocks in `alive` (some pixel
// still blending at the batch's start), so entries that reach only finished
// blocks are not staged.  Half-list entries: the forward stores each staged
// entry's exact block mask (restricted to `alive`) in the entry's top bits; the
// backward reads it from there (every entry before maxnc was staged by the
// forward of the same state, and a block finished before the entry's batch has
// no pixel whose n_contrib lies beyond the entry).  Each lane adds to `groups`
// the blocks its kept entries will evaluate (mask & alive), the issued-work
// statistic.
template <bool LIVE>
__device__ __forceinline__ int stage_compact(const BlendArgs& a, bool use_hl, uint32_t b0, int nb, uint32_t list0,
                                             const ProjRec* projv, float log2_amin, float X0, float Y0,
                                             const int* gmax, int maxnc, unsigned alive, float4* s_a,
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
          for (int k = 0; k < kBlocks; ++k) live |= ((int)pos < gmax[k] ? 1u : 0u) << k;
          msk = have_mask ? (msk & live) : live;
        } else if (!have_mask) {
          msk = alive;
        }
        if (msk) {
          const ProjRec* r = projv + id;
          ga = __ldg(&r->a);
          gb = __ldg(&r->b);
          gc = __ldg(&r->c.x);
          if (!have_mask)
            msk = LIVE ? (msk & block_mask_exact(ga, gb, log2_amin, X0, Y0, (1u << kBlocks) - 1u))
                       : block_mask_exact(ga, gb, log2_amin, X0, Y0, msk);
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

// Shared memory is carved out to the maximum once per kernel and device, so
// that the occupancy the register count allows is not cut by the per-warp
// tables.
template <class K>
cudaError_t prefer_shared(K kernel) {
  static bool done[kMaxDevicesAttr] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < kMaxDevicesAttr && done[dev]) return cudaSuccess;
  if (dev < kMaxDevicesAttr) done[dev] = true;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

// Persistent grid: as many one-warp CTAs as fit on the SMs, at most one per item.
template <class K>
int persistent_grid(K kernel, int num_sms, int64_t items, cudaError_t& e) {
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 32, 0);
  const int64_t g = (int64_t)(occ > 0 ? occ : 1) * num_sms;
  return (int)(items < g ? items : g);
}

}  // namespace airgs
