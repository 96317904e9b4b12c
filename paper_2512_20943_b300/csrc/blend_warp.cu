// Warp-per-tile blend kernels (sm_103a): one warp owns a whole 16x16 tile,
// each lane 8 adjacent pixels of one row (lanes 2r, 2r+1 cover row r).
//
// Why: both blend kernels are issue-bound, so the cost that matters is
// instructions per (pixel, Gaussian) pair.  With 8 pixels per lane the per-
// Gaussian work (shared-memory loads, the conic's row terms, the loop) is
// spread over 8 pairs, the per-pixel update is branch-free (predicated), the
// batch staging needs only __syncwarp, and the backward reduces each
// Gaussian's ten gradient sums once per tile (not once per warp of a tile):
// a 20-shuffle transpose butterfly leaves four consecutive sums on lanes 0, 8,
// 16, 24, which issue three red.global.add.v4.f32 into the gradient record.
//
// Semantics are those of k_blend_fwd / k_blend_bwd (same exact-rounding
// helpers, same skip / stop decisions, NaN-safe in the same way); a forward and
// backward of the same variant replay identical decisions.
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

constexpr int WPX = 8;       // pixels per lane
constexpr int WBATCH = 64;   // records staged per batch (two per lane)
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int warp_fetch(int* counter) {
  int it = 0;
  if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(kFull, it, 0);
}

// ------------------------------------------------------------------ forward
template <bool IMP>
__global__ void __launch_bounds__(32) k_blend_fwd_warp(BlendArgs a, FwdOut out) {
  __shared__ float4 s_a[WBATCH];
  __shared__ float4 s_b[WBATCH];
  __shared__ float s_c[WBATCH];
  __shared__ uint32_t s_id[WBATCH];
  __shared__ int64_t s_tile_base[AIRGS_MAX_VIEWS_DEV];

  const int lane = threadIdx.x;
  for (int v = lane; v < a.n_views; v += 32) s_tile_base[v] = a.cams[v].tile_base;
  __syncwarp();
  const float alpha_max = a.rp.alpha_max, alpha_min = a.rp.alpha_min, T_min = a.rp.T_min;
  unsigned long long pairs = 0;

  while (true) {
    const int item = warp_fetch(a.work_counter);
    if (item >= a.n_tiles) break;
    const int v = view_of_tile(s_tile_base, a.n_views, item);
    const CamDev& cam = a.cams[v];
    const int lt = (int)(item - s_tile_base[v]);
    const int tx = lt % cam.TW, ty = lt / cam.TW;
    const int py_i = ty * kTile + (lane >> 1);
    const int px0 = tx * kTile + (lane & 1) * WPX;
    const float py = (float)py_i + 0.5f;
    float pxf[WPX], T[WPX], C0[WPX], C1[WPX], C2[WPX];
    int last[WPX];
    unsigned done = 0;
#pragma unroll
    for (int k = 0; k < WPX; ++k) {
      pxf[k] = (float)(px0 + k) + 0.5f;
      if (!((px0 + k) < cam.W && py_i < cam.H)) done |= 1u << k;
      T[k] = 1.f;
      C0[k] = C1[k] = C2[k] = 0.f;
      last[k] = 0;
    }
    const uint2 range = a.ranges[item];
    const ProjRec* projv = a.proj + (size_t)v * a.n;
    uint32_t evals = 0;

    for (uint32_t b0 = range.x; b0 < range.y; b0 += WBATCH) {
      if (__all_sync(kFull, done == 0xFFu)) break;
      const int nb = (int)min((uint32_t)WBATCH, range.y - b0);
      for (int j = lane; j < nb; j += 32) {
        const uint32_t id = __ldg(a.ids + b0 + j);
        const ProjRec* r = projv + id;
        s_a[j] = __ldg(&r->a);
        s_b[j] = __ldg(&r->b);
        s_c[j] = __ldg(&r->c.x);
        s_id[j] = id;
      }
      __syncwarp();
      const int pos_base = (int)(b0 - range.x) + 1;
      for (int j = 0; j < nb; ++j) {
        if (__all_sync(kFull, done == 0xFFu)) break;
        evals += __popc(~done & 0xFFu);
        const float4 ga = s_a[j];
        const float4 gb = s_b[j];
        const float cb = s_c[j];
        float dy, b2dy, c2dy2;
        row_terms(ga.y, py, ga.w, gb.x, dy, b2dy, c2dy2);
        const int pos1 = pos_base + j;
        float wsum = 0.f;
        int bcount = 0;
#pragma unroll
        for (int k = 0; k < WPX; ++k) {
          const float dx = __fsub_rn(ga.x, pxf[k]);
          const float p2 = power2_of(dx, ga.z, b2dy, c2dy2);
          const float G = ex2_approx(p2);
          const float alpha = alpha_of(gb.y, G, alpha_max);
          const float Tn = transmit(T[k], alpha);
          const bool valid = !((done >> k) & 1u) && !(p2 > 0.f) && !(alpha < alpha_min);
          const bool stop = valid && (Tn < T_min);
          const bool blend = valid && !stop;
          const float w = __fmul_rn(alpha, T[k]);
          if (blend) {
            C0[k] = __fmaf_rn(gb.z, w, C0[k]);
            C1[k] = __fmaf_rn(gb.w, w, C1[k]);
            C2[k] = __fmaf_rn(cb, w, C2[k]);
            T[k] = Tn;
            last[k] = pos1;
          }
          if (stop) done |= 1u << k;
          if (IMP) {
            wsum += blend ? w : 0.f;
            bcount += blend ? 1 : 0;
          }
        }
        if (IMP) {
          if (__any_sync(kFull, bcount > 0)) {
            float s = wsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            const int c = __reduce_add_sync(kFull, bcount);
            if (lane == 0) {
              atomicAdd(out.imp_w + s_id[j], s);
              atomicAdd(out.imp_cnt + s_id[j], (uint32_t)c);
            }
          }
        }
      }
      __syncwarp();
    }
    pairs += evals;
    const int64_t HW = (int64_t)cam.W * cam.H;
    float* rgb = out.rgb + 3 * cam.pix_base;
#pragma unroll
    for (int k = 0; k < WPX; ++k) {
      if ((px0 + k) < cam.W && py_i < cam.H) {
        const int64_t pix = (int64_t)py_i * cam.W + px0 + k;
        rgb[pix] = __fmaf_rn(T[k], a.rp.bg[0], C0[k]);
        rgb[HW + pix] = __fmaf_rn(T[k], a.rp.bg[1], C1[k]);
        rgb[2 * HW + pix] = __fmaf_rn(T[k], a.rp.bg[2], C2[k]);
        if (out.T) out.T[cam.pix_base + pix] = T[k];
        out.ncontrib[cam.pix_base + pix] = last[k];
        if (out.ncontrib_user) out.ncontrib_user[cam.pix_base + pix] = last[k];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
  if (lane == 0 && pairs) {
    atomicAdd(a.pair_counter, pairs);
    if (a.pair_total) atomicAdd(a.pair_total, pairs);
  }
}

// ------------------------------------------------------------------ 16 -> 4 transpose reduction
// On entry every lane holds v[0..15]; on exit lanes with (lane & 7) == 0 hold
// the warp totals of slots 4q .. 4q+3 in v[0..3], q = lane >> 3.
__device__ __forceinline__ void warp_reduce16_to4(float (&v)[16], int lane) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool up = lane & 16;
    const float send = up ? v[k] : v[k + 8];
    const float keep = up ? v[k + 8] : v[k];
    v[k] = keep + __shfl_xor_sync(kFull, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = lane & 8;
    const float send = up ? v[k] : v[k + 4];
    const float keep = up ? v[k + 4] : v[k];
    v[k] = keep + __shfl_xor_sync(kFull, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 4;
    const float send = up ? v[k] : v[k + 2];
    const float keep = up ? v[k + 2] : v[k];
    v[k] = keep + __shfl_xor_sync(kFull, send, 4);
  }
  // lanes now hold slots 2m, 2m+1 (m = (lane >> 2) & 7) summed over lane bits 2..4
  v[0] += __shfl_xor_sync(kFull, v[0], 1);
  v[1] += __shfl_xor_sync(kFull, v[1], 1);
  v[0] += __shfl_xor_sync(kFull, v[0], 2);
  v[1] += __shfl_xor_sync(kFull, v[1], 2);
  v[2] = __shfl_xor_sync(kFull, v[0], 4);
  v[3] = __shfl_xor_sync(kFull, v[1], 4);
}

// ------------------------------------------------------------------ backward
// Per (tile, Gaussian) sums, scaled at the end:
//   0: sum dL/dpow (2 a2 dx + b2 dy)  x ln2   -> dL/dmx
//   1: sum dL/dpow (2 c2 dy + b2 dx)  x ln2   -> dL/dmy
//   2: sum dL/dpow dx^2               x -1/2  -> dL/dA
//   3: sum dL/dpow dx dy              x -1    -> dL/dB
//   4: sum dL/dpow dy^2               x -1/2  -> dL/dC
//   5: dL/do, 6-8: dL/d(r, g, b), 9: blend weight
template <bool L1, bool IMP>
__global__ void __launch_bounds__(32) k_blend_bwd_warp(BlendArgs a, BwdIn in) {
  __shared__ float4 s_a[WBATCH];
  __shared__ float4 s_b[WBATCH];
  __shared__ float s_c[WBATCH];
  __shared__ uint32_t s_id[WBATCH];
  __shared__ int64_t s_tile_base[AIRGS_MAX_VIEWS_DEV];

  const int lane = threadIdx.x;
  for (int v = lane; v < a.n_views; v += 32) s_tile_base[v] = a.cams[v].tile_base;
  __syncwarp();
  const float alpha_max = a.rp.alpha_max, alpha_min = a.rp.alpha_min;
  unsigned long long pairs = 0;
  float loss_acc = 0.f;

  while (true) {
    const int item = warp_fetch(a.work_counter);
    if (item >= a.n_tiles) break;
    const int v = view_of_tile(s_tile_base, a.n_views, item);
    const CamDev& cam = a.cams[v];
    const int lt = (int)(item - s_tile_base[v]);
    const int tx = lt % cam.TW, ty = lt / cam.TW;
    const int py_i = ty * kTile + (lane >> 1);
    const int px0 = tx * kTile + (lane & 1) * WPX;
    const float py = (float)py_i + 0.5f;
    const int64_t HW = (int64_t)cam.W * cam.H;
    const int64_t base3 = 3 * cam.pix_base;

    float pxf[WPX], T[WPX], gP[WPX], gC[WPX], g0[WPX], g1[WPX], g2[WPX];
    int nc[WPX];
    int my_max = 0;
#pragma unroll
    for (int k = 0; k < WPX; ++k) {
      pxf[k] = (float)(px0 + k) + 0.5f;
      T[k] = 1.f;
      gP[k] = 0.f;
      g0[k] = g1[k] = g2[k] = 0.f;
      gC[k] = 0.f;
      nc[k] = 0;
      if ((px0 + k) < cam.W && py_i < cam.H) {
        const int64_t pix = (int64_t)py_i * cam.W + px0 + k;
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
        my_max = max(my_max, nc[k]);
      }
    }
    const int maxnc = (int)__reduce_max_sync(kFull, (unsigned)my_max);
    const uint2 range = a.ranges[item];
    const uint32_t end = range.x + (uint32_t)maxnc;
    const ProjRec* projv = a.proj + (size_t)v * a.n;
    GradRec* gradv = in.grad + (size_t)v * a.n;
    uint32_t evals = 0;
#pragma unroll
    for (int k = 0; k < WPX; ++k) evals += (uint32_t)nc[k];

    for (uint32_t b0 = range.x; b0 < end; b0 += WBATCH) {
      const int nb = (int)min((uint32_t)WBATCH, end - b0);
      for (int j = lane; j < nb; j += 32) {
        const uint32_t id = __ldg(a.ids + b0 + j);
        const ProjRec* r = projv + id;
        s_a[j] = __ldg(&r->a);
        s_b[j] = __ldg(&r->b);
        s_c[j] = __ldg(&r->c.x);
        s_id[j] = id;
      }
      __syncwarp();
      const int pos0 = (int)(b0 - range.x);
      for (int j = 0; j < nb; ++j) {
        const int pos = pos0 + j;
        const float4 ga = s_a[j];
        const float4 gb = s_b[j];
        const float cb = s_c[j];
        float dy, b2dy, c2dy2;
        row_terms(ga.y, py, ga.w, gb.x, dy, b2dy, c2dy2);
        const float dy2 = dy * dy;
        const float twoa2 = 2.f * ga.z;
        const float twoc2dy = 2.f * gb.x * dy;
        float acc[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = 0.f;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < WPX; ++k) {
          const float dx = __fsub_rn(ga.x, pxf[k]);
          const float p2 = power2_of(dx, ga.z, b2dy, c2dy2);
          const float G = ex2_approx(p2);
          const float oG = __fmul_rn(gb.y, G);
          const float alpha = alpha_of(gb.y, G, alpha_max);
          const bool valid = (pos < nc[k]) && !(p2 > 0.f) && !(alpha < alpha_min);
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
          acc[4] = fmaf(dL_dpow, dy2, acc[4]);
          acc[0] = fmaf(dL_dpow, fmaf(twoa2, dx, b2dy), acc[0]);
          acc[1] = fmaf(dL_dpow, fmaf(ga.w, dx, twoc2dy), acc[1]);
          if (IMP) acc[9] += w;
          cnt += valid ? 1 : 0;
        }
        if (__any_sync(kFull, cnt > 0)) {
          float vals[16];
#pragma unroll
          for (int q = 0; q < 10; ++q) vals[q] = acc[q];
#pragma unroll
          for (int q = 10; q < 16; ++q) vals[q] = 0.f;
          warp_reduce16_to4(vals, lane);
          const uint32_t id = s_id[j];
          float* gr = reinterpret_cast<float*>(gradv + id);
          if (lane == 0) red_add_v4(gr, vals[0] * kLn2, vals[1] * kLn2, -0.5f * vals[2], -vals[3]);
          if (lane == 8) red_add_v4(gr + 4, -0.5f * vals[0], vals[1], vals[2], vals[3]);
          if (lane == 16) {
            red_add_v4(gr + 8, vals[0], 0.f, 0.f, 0.f);
            if (IMP && vals[1] != 0.f) atomicAdd(in.imp_w + id, vals[1]);
          }
          if (IMP) {
            const int c = __reduce_add_sync(kFull, cnt);
            if (lane == 0 && c) atomicAdd(in.imp_cnt + id, (uint32_t)c);
          }
        }
      }
      __syncwarp();
    }
    pairs += evals;
  }
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
  if (lane == 0 && pairs) {
    atomicAdd(a.pair_counter, pairs);
    if (a.pair_total) atomicAdd(a.pair_total, pairs);
  }
  if (L1 && in.loss) {
    for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(kFull, loss_acc, o);
    if (lane == 0) atomicAdd(in.loss, loss_acc * in.inv_norm);
  }
}

// ------------------------------------------------------------------ launchers
template <class K>
static int persistent_grid(K kernel, int num_sms, int64_t n_tiles, cudaError_t& e) {
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 32, 0);
  int64_t g = (int64_t)(occ > 0 ? occ : 1) * num_sms;
  return (int)(n_tiles < g ? n_tiles : g);
}

cudaError_t launch_blend_fwd_warp(cudaStream_t st, int num_sms, const BlendArgs& a, const FwdOut& o) {
  cudaError_t e = cudaSuccess;
  if (o.imp_w) {
    int grid = persistent_grid(k_blend_fwd_warp<true>, num_sms, a.n_tiles, e);
    if (e != cudaSuccess) return e;
    if (grid > 0) k_blend_fwd_warp<true><<<grid, 32, 0, st>>>(a, o);
  } else {
    int grid = persistent_grid(k_blend_fwd_warp<false>, num_sms, a.n_tiles, e);
    if (e != cudaSuccess) return e;
    if (grid > 0) k_blend_fwd_warp<false><<<grid, 32, 0, st>>>(a, o);
  }
  count_launches(1);
  return cudaGetLastError();
}

template <bool L1, bool IMP>
static cudaError_t bwd_warp(cudaStream_t st, int num_sms, const BlendArgs& a, const BwdIn& in) {
  cudaError_t e = cudaSuccess;
  int grid = persistent_grid(k_blend_bwd_warp<L1, IMP>, num_sms, a.n_tiles, e);
  if (e != cudaSuccess) return e;
  if (grid > 0) k_blend_bwd_warp<L1, IMP><<<grid, 32, 0, st>>>(a, in);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_blend_bwd_warp(cudaStream_t st, int num_sms, const BlendArgs& a, const BwdIn& in) {
  const bool l1 = in.target != nullptr, imp = in.imp_w != nullptr;
  if (l1) return imp ? bwd_warp<true, true>(st, num_sms, a, in) : bwd_warp<true, false>(st, num_sms, a, in);
  return imp ? bwd_warp<false, true>(st, num_sms, a, in) : bwd_warp<false, false>(st, num_sms, a, in);
}

}  // namespace airgs
