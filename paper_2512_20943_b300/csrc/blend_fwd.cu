// Blend forward (sm_103a): front-to-back alpha blending of each pixel's tile
// list, one warp per 16x8 half tile, persistent over an atomic queue of all
// (view, half tile) items of a batch.
//
// Per pixel p (sampled at (u + 0.5, v + 0.5)) and list entry i in order:
// d = p - mean2d_i, power = -1/2 (A dx^2 + C dy^2) - B dx dy (at most 0: the
// projection keeps only positive-definite conics, so the kernels have no
// power > 0 test, and a rounding excess near power = 0 blends as the exact
// value does); alpha = min(alpha_max, o_i e^power); skip if alpha < alpha_min; stop (i not
// blended) if T (1 - alpha) < T_min; else C += c_i alpha T, T <- T (1 - alpha).
// The kernel stores C + T bg, T_final and n_contrib (position + 1 of the last
// blended entry), and with IMP adds alpha T and 1 per blended pair to the
// Gaussian's usage weight and count.
//
// Each staged entry is tested against the blocks whose pixels are all still
// blending at the batch's start; the entry's exact block mask is stored into
// its half-list entry for the backward, which walks the same entries.  All
// per-pair arithmetic uses the exact-replay helpers of airgs_internal.cuh, so
// the backward reproduces every decision bit for bit.
#include "blend_common.cuh"

#include <cstddef>

namespace airgs {

template <bool IMP, int FB, int MINB>
__global__ void __launch_bounds__(32, MINB) k_blend_fwd(BlendArgs a, FwdOut out) {
  // the warp's shared memory as one block (16-byte records first)
  struct __align__(16) WarpSmem {
    float4 a[FB];
    float4 b[FB];
    StageMeta meta[FB];
    unsigned long long pairs;  // the warp's definition pairs (no register holds them through the blend)
  };
  static_assert(offsetof(WarpSmem, a) % 16 == 0 && offsetof(WarpSmem, b) % 16 == 0 &&
                    offsetof(WarpSmem, meta) % 16 == 0,
                "16-byte shared loads need 16-byte aligned records");
  __shared__ WarpSmem sw;
  float4* s_a = sw.a;
  float4* s_b = sw.b;
  StageMeta* s_meta = sw.meta;
  unsigned long long& s_pairs = sw.pairs;

  const int lane = threadIdx.x;
  const float alpha_max = a.rp.alpha_max, alpha_min = a.rp.alpha_min, T_min = a.rp.T_min;
  const float log2_amin = log2f(alpha_min);
  const int lx = lane & 7, ly = lane >> 3;
  uint32_t exec_groups = 0;  // per lane: blocks counted while staging
  if (lane == 0) s_pairs = 0ull;

  while (true) {
    const int q = cull_fetch(a.work_counter);
    if (q >= a.n_tiles * 2) break;
    const int work = queue_item(a.work_order, q);
    const int item = work >> 1, part = work & 1;
    const int v = view_of_tile_cams(a.cams, a.n_views, item);
    const CamDev& cam = a.cams[v];
    const int lt = item - (int)__ldg(&a.cams[v].tile_base);
    const int X0 = (lt % cam.TW) * kTile, Y0 = (lt / cam.TW) * kTile + part * (kTile / 2);
    const float pxb[2] = {(float)(X0 + lx) + 0.5f, (float)(X0 + 8 + lx) + 0.5f};
    const float pyb[2] = {(float)(Y0 + ly) + 0.5f, (float)(Y0 + 4 + ly) + 0.5f};  // the two block rows
    float T[kBlocks], C2[kBlocks];
    float2 C01[kBlocks];  // the first two colour channels, updated as one packed FMA
    // last: position + 1 of the last blended entry; stop_at: -1 while the pixel
    // is blending, else position + 1 of the entry that stopped it (0 for a pixel
    // outside the image)
    int last[kBlocks], stop_at[kBlocks];
#pragma unroll
    for (int k = 0; k < kBlocks; ++k) {
      const int x = X0 + 8 * (k & 1) + lx, y = Y0 + 4 * (k >> 1) + ly;
      T[k] = 1.f;
      C01[k] = make_float2(0.f, 0.f);
      C2[k] = 0.f;
      last[k] = 0;
      stop_at[k] = (x < cam.W && y < cam.H) ? -1 : 0;
    }
    const uint2 range = a.ranges[item];
    const bool use_hl = a.hl != nullptr;  // this half's compacted list
    uint2 er = range;
    if (use_hl) er = a.hranges[(int64_t)part * a.n_tiles + item];
    const ProjRec* projv = a.proj + (size_t)v * a.n;

    for (uint32_t b0 = er.x; b0 < er.y; b0 += FB) {
      unsigned live = 0;
#pragma unroll
      for (int k = 0; k < kBlocks; ++k)
        if (__any_sync(kAll, stop_at[k] < 0)) live |= 1u << k;
      if (live == 0) break;
      bool unused = false;
      const int nb = stage_compact<false>(a, use_hl, b0, (int)min((uint32_t)FB, er.y - b0), range.x, projv,
                                          log2_amin, (float)X0, (float)Y0, nullptr, 0, live, s_a, s_b, s_meta, unused,
                                          exec_groups);
      for (int j = 0; j < nb; ++j) {
        const StageMeta me = s_meta[j];
        const unsigned m = me.mask;  // staged against the blocks live at the batch's start: non-zero
        const float4 ga = s_a[j];
        const float4 gb = s_b[j];
        const float cb = me.c;
        const int pos1 = (int)me.pos1;
        const float dxb[2] = {__fsub_rn(ga.x, pxb[0]), __fsub_rn(ga.x, pxb[1])};
        float wsum = 0.f;
        int bcount = 0;
        // one block: the lane's pixel of block k (column bx) against the entry
        auto block = [&](int k, int bx, float dy, float b2dy, float c2dy2) {
          const float dx = dxb[bx];
          const float p2 = power2_of(dx, ga.z, b2dy, c2dy2);
          const float G = ex2_approx(p2);
          const float alpha = alpha_of(gb.y, G, alpha_max);
          const float w = blend_weight(alpha, T[k]);
          const float Tn = transmit(T[k], w);
          const bool valid = (stop_at[k] < 0) && !(alpha < alpha_min);
          const bool stop = valid && (Tn < T_min);
          const bool blend = valid && !stop;
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
        };
#pragma unroll
        for (int by = 0; by < 2; ++by) {
          // the row's live blocks (warp-uniform): both, or one of them
          const unsigned rm = (m >> (2 * by)) & 3u;
          if (!rm) continue;
          float dy, b2dy, c2dy2;  // shared by the row's two blocks
          row_terms(ga.y, pyb[by], ga.w, gb.x, dy, b2dy, c2dy2);
          if (rm == 3u) {
            block(2 * by, 0, dy, b2dy, c2dy2);
            block(2 * by + 1, 1, dy, b2dy, c2dy2);
          } else if (rm == 1u) {
            block(2 * by, 0, dy, b2dy, c2dy2);
          } else {
            block(2 * by + 1, 1, dy, b2dy, c2dy2);
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
    const int64_t HW = (int64_t)cam.W * cam.H;
    float* rgb = out.rgb + 3 * cam.pix_base;
    const uint32_t len = range.y - range.x;
    unsigned long long pairs = 0;
#pragma unroll
    for (int k = 0; k < kBlocks; ++k) {
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
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kAll, pairs, o);
    if (lane == 0) s_pairs += pairs;
  }
  unsigned long long executed = exec_groups;
  for (int o = 16; o > 0; o >>= 1) executed += __shfl_xor_sync(kAll, executed, o);
  __syncwarp();
  if (lane == 0) {
    if (a.exec_total && executed) atomicAdd(a.exec_total, 32ull * executed);  // 32 lane evaluations per block
    if (s_pairs) {
      atomicAdd(a.pair_counter, s_pairs);
      if (a.pair_total) atomicAdd(a.pair_total, s_pairs);
    }
  }
}

namespace {

template <bool IMP, int FB, int MINB>
cudaError_t fwd_launch(cudaStream_t st, int num_sms, const BlendArgs& a, const FwdOut& o) {
  cudaError_t e = prefer_shared(k_blend_fwd<IMP, FB, MINB>);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid(k_blend_fwd<IMP, FB, MINB>, num_sms, a.n_tiles * 2, e);
  if (e != cudaSuccess) return e;
  if (grid > 0) k_blend_fwd<IMP, FB, MINB><<<grid, 32, 0, st>>>(a, o);
  count_launches(1);
  return cudaGetLastError();
}

template <int FB, int MINB>
cudaError_t fwd_dispatch(cudaStream_t st, int num_sms, const BlendArgs& a, const FwdOut& o) {
  return o.imp_w ? fwd_launch<true, FB, MINB>(st, num_sms, a, o) : fwd_launch<false, FB, MINB>(st, num_sms, a, o);
}

}  // namespace

// The compiled forward shapes (kFwdShapes in kernels.h): staged entries per
// batch and warps per SM (the register bound).
cudaError_t launch_blend_fwd(cudaStream_t st, int shape, int num_sms, const BlendArgs& a, const FwdOut& o) {
  switch (shape) {
    case 1: return fwd_dispatch<16, 28>(st, num_sms, a, o);
    case 2: return fwd_dispatch<64, 28>(st, num_sms, a, o);
    case 3: return fwd_dispatch<32, 32>(st, num_sms, a, o);
    case 4: return fwd_dispatch<32, 24>(st, num_sms, a, o);
    default: return fwd_dispatch<32, 28>(st, num_sms, a, o);
  }
}

}  // namespace airgs
