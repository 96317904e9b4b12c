// Front-to-back blending of tile lists, forward and adjoint (sm_103a).
//
// Both kernels are persistent: a grid of (SMs x resident CTAs) CTAs pulls
// (view, tile) work items from an atomic counter, so one launch covers every
// view of a batch, whatever the views' resolutions.  A CTA owns one 16x16 tile
// at a time; each thread owns PX horizontally adjacent pixels of one row (the
// row terms of the conic are then shared by the thread's pixels).  The tile's
// Gaussians are staged through shared memory in batches of 256 records
// gathered by id; the CTA leaves the list as soon as every pixel has stopped
// (__syncthreads_count).
//
// Per pixel (sampled at (x + 0.5, y + 0.5)) and list entry i in order:
//   power = -1/2 (A dx^2 + C dy^2) - B dx dy       skip if power > 0
//   alpha = min(alpha_max, o_i exp(power))          skip if alpha < alpha_min
//   stop (i not blended) if T (1 - alpha) < T_min
//   C += c_i alpha T;  T *= 1 - alpha
// with the conic pre-scaled by log2(e) so exp is one ex2.approx.
//
// The adjoint replays the same list front to back (no per-pixel lists are
// stored): with P_i the colour accumulated through i and C the final colour
// (background term included),
//   dC/dc_i = alpha_i T_i,   dC/dalpha_i = c_i T_i - (C - P_i) / (1 - alpha_i).
// The forward and the replay share the exact-rounding helpers, so P_i is
// bit-identical to the forward's running sum.  Per-Gaussian gradients are
// reduced over the warp with a 16-slot transpose butterfly (16 shuffles for
// all ten values), over the CTA in shared memory, and leave the CTA with
// three vector reductions (red.global.add.v4.f32) per (tile, Gaussian).
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

constexpr int BATCH = 256;

__device__ __forceinline__ int fetch_item(int* counter, int* s_item) {
  if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
  __syncthreads();
  int it = *s_item;
  __syncthreads();
  return it;
}

// ------------------------------------------------------------------ forward
template <int PX, bool IMP>
__global__ void __launch_bounds__(kTilePixels / PX) k_blend_fwd(BlendArgs a, FwdOut out) {
  constexpr int NT = kTilePixels / PX;  // threads per CTA
  constexpr int COLS = kTile / PX;      // threads per pixel row
  __shared__ float4 s_a[BATCH];
  __shared__ float4 s_b[BATCH];
  __shared__ float s_c[BATCH];
  __shared__ int s_item;
  __shared__ int64_t s_tile_base[AIRGS_MAX_VIEWS_DEV];

  const int tid = threadIdx.x;
  for (int v = tid; v < a.n_views; v += NT) s_tile_base[v] = a.cams[v].tile_base;
  const float alpha_max = a.rp.alpha_max, alpha_min = a.rp.alpha_min, T_min = a.rp.T_min;
  unsigned long long pairs = 0;

  while (true) {
    int item = fetch_item(a.work_counter, &s_item);
    if (item >= a.n_tiles) break;
    const int v = view_of_tile(s_tile_base, a.n_views, item);
    const CamDev& cam = a.cams[v];
    const int lt = (int)(item - s_tile_base[v]);
    const int tx = lt % cam.TW, ty = lt / cam.TW;
    const int py_i = ty * kTile + tid / COLS;
    const int px0 = tx * kTile + (tid % COLS) * PX;
    const float py = (float)py_i + 0.5f;
    float pxf[PX];
    bool inside[PX];
    float T[PX], C[PX][3];
    int last[PX];
    bool done[PX];
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      pxf[k] = (float)(px0 + k) + 0.5f;
      inside[k] = (px0 + k) < cam.W && py_i < cam.H;
      done[k] = !inside[k];
      T[k] = 1.f;
      C[k][0] = C[k][1] = C[k][2] = 0.f;
      last[k] = 0;
    }
    const uint2 range = a.ranges[item];
    const ProjRec* projv = a.proj + (size_t)v * a.n;

    for (uint32_t b0 = range.x; b0 < range.y; b0 += BATCH) {
      bool active = false;
#pragma unroll
      for (int k = 0; k < PX; ++k) active |= !done[k];
      if (__syncthreads_count(active) == 0) break;
      const int nb = (int)min((uint32_t)BATCH, range.y - b0);
      for (int j = tid; j < nb; j += NT) {
        uint32_t id = __ldg(a.ids + b0 + j);
        const ProjRec* r = projv + id;
        s_a[j] = __ldg(&r->a);
        s_b[j] = __ldg(&r->b);
        s_c[j] = __ldg(&r->c.x);
      }
      __syncthreads();
      // the loop is warp-uniform (a warp leaves when all its pixels stopped), so
      // the importance reduction below can use full-warp shuffles
      for (int j = 0; j < nb; ++j) {
        bool any = false;
#pragma unroll
        for (int k = 0; k < PX; ++k) any |= !done[k];
        if (!__any_sync(0xffffffffu, any)) break;
        const float4 ga = s_a[j];
        const float4 gb = s_b[j];
        float dy, b2dy, c2dy2;
        row_terms(ga.y, py, ga.w, gb.x, dy, b2dy, c2dy2);
        float wsum = 0.f;
        int bcount = 0;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
          if (done[k]) continue;
          ++pairs;
          const float dx = __fsub_rn(ga.x, pxf[k]);
          const float p2 = power2_of(dx, ga.z, b2dy, c2dy2);
          if (p2 > 0.f) continue;
          const float G = ex2_approx(p2);
          const float alpha = alpha_of(gb.y, G, alpha_max);
          if (alpha < alpha_min) continue;
          const float Tn = transmit(T[k], alpha);
          if (Tn < T_min) {
            done[k] = true;
            continue;
          }
          const float w = __fmul_rn(alpha, T[k]);
          C[k][0] = __fmaf_rn(gb.z, w, C[k][0]);
          C[k][1] = __fmaf_rn(gb.w, w, C[k][1]);
          C[k][2] = __fmaf_rn(s_c[j], w, C[k][2]);
          T[k] = Tn;
          last[k] = (int)(b0 - range.x) + j + 1;
          if (IMP) {
            wsum += w;
            ++bcount;
          }
        }
        if (IMP) {
          // warp-reduce the blend weight of Gaussian j; one atomic per warp
          if (__any_sync(0xffffffffu, bcount > 0)) {
            float s = wsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const int c = __reduce_add_sync(0xffffffffu, bcount);
            if ((tid & 31) == 0) {
              const uint32_t id = __ldg(a.ids + b0 + j);
              atomicAdd(out.imp_w + id, s);
              atomicAdd(out.imp_cnt + id, (uint32_t)c);
            }
          }
        }
      }
      __syncthreads();
    }
    // outputs
    const int64_t HW = (int64_t)cam.W * cam.H;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      if (!inside[k]) continue;
      const int64_t pix = (int64_t)py_i * cam.W + px0 + k;
      float* rgb = out.rgb + 3 * cam.pix_base;
      rgb[pix] = __fmaf_rn(T[k], a.rp.bg[0], C[k][0]);
      rgb[HW + pix] = __fmaf_rn(T[k], a.rp.bg[1], C[k][1]);
      rgb[2 * HW + pix] = __fmaf_rn(T[k], a.rp.bg[2], C[k][2]);
      if (out.T) out.T[cam.pix_base + pix] = T[k];
      out.ncontrib[cam.pix_base + pix] = last[k];
      if (out.ncontrib_user) out.ncontrib_user[cam.pix_base + pix] = last[k];
    }
  }
  // evaluated-pair statistics
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
  if ((tid & 31) == 0 && pairs) {
    atomicAdd(a.pair_counter, pairs);
    if (a.pair_total) atomicAdd(a.pair_total, pairs);
  }
}

// ------------------------------------------------------------------ 16-slot warp transpose reduction
// On entry every lane holds v[0..15]; on exit lane l holds in v[0] the warp
// total of slot (l >> 1) & 15.
__device__ __forceinline__ void warp_transpose_reduce16(float (&v)[16], int lane) {
  const unsigned FULL = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool up = lane & 16;
    float send = up ? v[k] : v[k + 8];
    float keep = up ? v[k + 8] : v[k];
    v[k] = keep + __shfl_xor_sync(FULL, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = lane & 8;
    float send = up ? v[k] : v[k + 4];
    float keep = up ? v[k + 4] : v[k];
    v[k] = keep + __shfl_xor_sync(FULL, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 4;
    float send = up ? v[k] : v[k + 2];
    float keep = up ? v[k + 2] : v[k];
    v[k] = keep + __shfl_xor_sync(FULL, send, 4);
  }
  {
    const bool up = lane & 2;
    float send = up ? v[0] : v[1];
    float keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(FULL, send, 2);
  }
  v[0] += __shfl_xor_sync(FULL, v[0], 1);
}

// ------------------------------------------------------------------ backward
// Gradient slots: 0 mx, 1 my, 2 A, 3 B, 4 C, 5 opacity, 6 r, 7 g, 8 b, 9 blend weight.
constexpr int NSLOT = 10;

template <int PX, bool L1, bool IMP>
__global__ void __launch_bounds__(kTilePixels / PX) k_blend_bwd(BlendArgs a, BwdIn in) {
  constexpr int NT = kTilePixels / PX;
  constexpr int COLS = kTile / PX;
  constexpr int NW = NT / 32;
  __shared__ float4 s_a[BATCH];
  __shared__ float4 s_b[BATCH];
  __shared__ float s_c[BATCH];
  __shared__ float s_g[BATCH][NSLOT + 1];
  __shared__ uint32_t s_cnt[BATCH];
  __shared__ int s_item;
  __shared__ int s_maxnc;
  __shared__ float s_loss[NW];
  __shared__ int64_t s_tile_base[AIRGS_MAX_VIEWS_DEV];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int v = tid; v < a.n_views; v += NT) s_tile_base[v] = a.cams[v].tile_base;
  const float alpha_max = a.rp.alpha_max, alpha_min = a.rp.alpha_min;
  unsigned long long pairs = 0;
  float loss_acc = 0.f;

  while (true) {
    if (tid == 0) s_maxnc = 0;
    int item = fetch_item(a.work_counter, &s_item);
    if (item >= a.n_tiles) break;
    const int v = view_of_tile(s_tile_base, a.n_views, item);
    const CamDev& cam = a.cams[v];
    const int lt = (int)(item - s_tile_base[v]);
    const int tx = lt % cam.TW, ty = lt / cam.TW;
    const int py_i = ty * kTile + tid / COLS;
    const int px0 = tx * kTile + (tid % COLS) * PX;
    const float py = (float)py_i + 0.5f;
    const int64_t HW = (int64_t)cam.W * cam.H;

    float pxf[PX], T[PX], P[PX][3], g[PX][3], gC[PX];
    int nc[PX];
    int my_max = 0;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      pxf[k] = (float)(px0 + k) + 0.5f;
      const bool inside = (px0 + k) < cam.W && py_i < cam.H;
      T[k] = 1.f;
      P[k][0] = P[k][1] = P[k][2] = 0.f;
      nc[k] = 0;
      g[k][0] = g[k][1] = g[k][2] = 0.f;
      gC[k] = 0.f;
      if (inside) {
        const int64_t pix = (int64_t)py_i * cam.W + px0 + k;
        const int64_t base = 3 * cam.pix_base;
        float cf[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          cf[ch] = in.rgb[base + ch * HW + pix];
          if (L1) {
            const float d = cf[ch] - in.target[base + ch * HW + pix];
            g[k][ch] = d > 0.f ? in.inv_norm : (d < 0.f ? -in.inv_norm : 0.f);
            loss_acc += fabsf(d);
          } else {
            g[k][ch] = in.dL[base + ch * HW + pix];
          }
        }
        gC[k] = g[k][0] * cf[0] + g[k][1] * cf[1] + g[k][2] * cf[2];
        nc[k] = in.ncontrib[cam.pix_base + pix];
        my_max = max(my_max, nc[k]);
      }
    }
    atomicMax(&s_maxnc, my_max);
    __syncthreads();
    const uint2 range = a.ranges[item];
    const uint32_t end = range.x + (uint32_t)s_maxnc;
    __syncthreads();  // s_maxnc is reset by thread 0 at the next item
    const ProjRec* projv = a.proj + (size_t)v * a.n;
    GradRec* gradv = in.grad + (size_t)v * a.n;

    for (uint32_t b0 = range.x; b0 < end; b0 += BATCH) {
      const int nb = (int)min((uint32_t)BATCH, end - b0);
      for (int j = tid; j < nb; j += NT) {
        uint32_t id = __ldg(a.ids + b0 + j);
        const ProjRec* r = projv + id;
        s_a[j] = __ldg(&r->a);
        s_b[j] = __ldg(&r->b);
        s_c[j] = __ldg(&r->c.x);
#pragma unroll
        for (int q = 0; q < NSLOT; ++q) s_g[j][q] = 0.f;
        s_cnt[j] = 0;
      }
      __syncthreads();
      const int pos0 = (int)(b0 - range.x);
      for (int j = 0; j < nb; ++j) {
        const int pos = pos0 + j;
        const float4 ga = s_a[j];
        const float4 gb = s_b[j];
        const float cb = s_c[j];
        float dy, b2dy, c2dy2;
        row_terms(ga.y, py, ga.w, gb.x, dy, b2dy, c2dy2);
        float acc[NSLOT];
#pragma unroll
        for (int q = 0; q < NSLOT; ++q) acc[q] = 0.f;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
          if (pos >= nc[k]) continue;
          ++pairs;
          const float dx = __fsub_rn(ga.x, pxf[k]);
          const float p2 = power2_of(dx, ga.z, b2dy, c2dy2);
          if (p2 > 0.f) continue;
          const float G = ex2_approx(p2);
          const float oG = __fmul_rn(gb.y, G);
          const float alpha = alpha_of(gb.y, G, alpha_max);
          if (alpha < alpha_min) continue;
          const float w = __fmul_rn(alpha, T[k]);
          // colour adjoint and the running colour P_i (bit-identical to the forward)
          const float gc = g[k][0] * gb.z + g[k][1] * gb.w + g[k][2] * cb;
          acc[6] += w * g[k][0];
          acc[7] += w * g[k][1];
          acc[8] += w * g[k][2];
          P[k][0] = __fmaf_rn(gb.z, w, P[k][0]);
          P[k][1] = __fmaf_rn(gb.w, w, P[k][1]);
          P[k][2] = __fmaf_rn(cb, w, P[k][2]);
          const float gPn = g[k][0] * P[k][0] + g[k][1] * P[k][1] + g[k][2] * P[k][2];
          const float om = __fsub_rn(1.0f, alpha);
          const float dL_dalpha = T[k] * gc - __fdividef(gC[k] - gPn, om);
          T[k] = transmit(T[k], alpha);
          if (IMP) {
            acc[9] += w;
            ++cnt;
          }
          if (oG <= alpha_max) {
            // alpha = o G, G = exp(power)
            const float dL_dpow = dL_dalpha * alpha;
            acc[5] += dL_dalpha * G;
            acc[2] += dL_dpow * (-0.5f * dx * dx);
            acc[3] += dL_dpow * (-dx * dy);
            acc[4] += dL_dpow * (-0.5f * dy * dy);
            // dpower/dmx = ln2 (2 a2 dx + b2 dy), dpower/dmy = ln2 (2 c2 dy + b2 dx)
            acc[0] += dL_dpow * kLn2 * (2.f * ga.z * dx + ga.w * dy);
            acc[1] += dL_dpow * kLn2 * (2.f * gb.x * dy + ga.w * dx);
          }
        }
        const bool contributed = cnt > 0 || acc[6] != 0.f || acc[7] != 0.f || acc[8] != 0.f || acc[5] != 0.f;
        if (__ballot_sync(0xffffffffu, contributed)) {
          float vals[16];
#pragma unroll
          for (int q = 0; q < NSLOT; ++q) vals[q] = acc[q];
#pragma unroll
          for (int q = NSLOT; q < 16; ++q) vals[q] = 0.f;
          warp_transpose_reduce16(vals, lane);
          const int slot = (lane >> 1) & 15;
          if ((lane & 1) == 0 && slot < NSLOT) atomicAdd(&s_g[j][slot], vals[0]);
          if (IMP) {
            const int c = __reduce_add_sync(0xffffffffu, cnt);
            if (lane == 0 && c) atomicAdd(&s_cnt[j], (uint32_t)c);
          }
        }
      }
      __syncthreads();
      // one vector reduction per (tile, Gaussian) and record word
      for (int j = tid; j < nb; j += NT) {
        const float* q = s_g[j];
        bool nz = false;
#pragma unroll
        for (int t = 0; t < NSLOT; ++t) nz |= q[t] != 0.f;
        if (!nz && s_cnt[j] == 0) continue;
        const uint32_t id = __ldg(a.ids + b0 + j);
        float* gr = reinterpret_cast<float*>(gradv + id);
        red_add_v4(gr, q[0], q[1], q[2], q[3]);
        red_add_v4(gr + 4, q[4], q[5], q[6], q[7]);
        red_add_v4(gr + 8, q[8], 0.f, 0.f, 0.f);
        if (IMP) {
          if (q[9] != 0.f) atomicAdd(in.imp_w + id, q[9]);
          if (s_cnt[j]) atomicAdd(in.imp_cnt + id, s_cnt[j]);
        }
      }
      __syncthreads();
    }
  }
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
  if (lane == 0 && pairs) {
    atomicAdd(a.pair_counter, pairs);
    if (a.pair_total) atomicAdd(a.pair_total, pairs);
  }
  if (L1 && in.loss) {
    for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
    if (lane == 0) s_loss[warp] = loss_acc;
    __syncthreads();
    if (tid == 0) {
      float s = 0.f;
      for (int w = 0; w < NW; ++w) s += s_loss[w];
      atomicAdd(in.loss, s * in.inv_norm);
    }
  }
}

// ------------------------------------------------------------------ variants and launchers
// Variants 0-2: a 16x16 tile per CTA with 1, 2 or 4 pixels per thread;
// variant 3: a tile per warp with 8 pixels per lane (blend_warp.cu);
// variant 4: a tile per warp in eight 8x4 blocks with exact block culling;
// variant 5: the same with a half tile (four blocks) per warp (blend_cull.cu);
// variant 6: variant 5 with compacted staging and deferred backward reductions.
static const char* kVariantName[] = {"px1_256t", "px2_128t", "px4_64t", "warp_px8", "warp_cull8x4",
                                     "halfwarp_cull8x4", "halfwarp_cull8x4_compact"};
constexpr int kNumVariants = 7;

int blend_variant_count() { return kNumVariants; }
const char* blend_variant_name(int v) { return (v >= 0 && v < kNumVariants) ? kVariantName[v] : ""; }

template <int PX, bool IMP>
static cudaError_t fwd_launch(cudaStream_t st, int grid_per_sm, int num_sms, const BlendArgs& a, const FwdOut& o) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_fwd<PX, IMP>, kTilePixels / PX, 0);
  if (e != cudaSuccess) return e;
  int grid = max(1, occ) * num_sms;
  if (grid_per_sm > 0) grid = min(grid, grid_per_sm * num_sms);
  grid = (int)(a.n_tiles < (int64_t)grid ? a.n_tiles : (int64_t)grid);
  if (grid <= 0) return cudaSuccess;
  k_blend_fwd<PX, IMP><<<grid, kTilePixels / PX, 0, st>>>(a, o);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_blend_fwd(cudaStream_t st, int variant, int num_sms, const BlendArgs& a, const FwdOut& o) {
  bool imp = o.imp_w != nullptr;
  switch (variant) {
    case 3:
      return launch_blend_fwd_warp(st, num_sms, a, o);
    case 4:
      return launch_blend_fwd_cull(st, num_sms, 8, false, a, o);
    case 5:
      return launch_blend_fwd_cull(st, num_sms, 4, false, a, o);
    case 6:
      return launch_blend_fwd_cull(st, num_sms, 4, true, a, o);
    case 1:
      return imp ? fwd_launch<2, true>(st, 0, num_sms, a, o) : fwd_launch<2, false>(st, 0, num_sms, a, o);
    case 2:
      return imp ? fwd_launch<4, true>(st, 0, num_sms, a, o) : fwd_launch<4, false>(st, 0, num_sms, a, o);
    default:
      return imp ? fwd_launch<1, true>(st, 0, num_sms, a, o) : fwd_launch<1, false>(st, 0, num_sms, a, o);
  }
}

template <int PX, bool L1, bool IMP>
static cudaError_t bwd_launch(cudaStream_t st, int num_sms, const BlendArgs& a, const BwdIn& in) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_bwd<PX, L1, IMP>, kTilePixels / PX, 0);
  if (e != cudaSuccess) return e;
  int64_t g64 = (int64_t)max(1, occ) * num_sms;
  int grid = (int)(a.n_tiles < g64 ? a.n_tiles : g64);
  if (grid <= 0) return cudaSuccess;
  k_blend_bwd<PX, L1, IMP><<<grid, kTilePixels / PX, 0, st>>>(a, in);
  count_launches(1);
  return cudaGetLastError();
}

template <int PX>
static cudaError_t bwd_dispatch(cudaStream_t st, int num_sms, const BlendArgs& a, const BwdIn& in) {
  bool l1 = in.target != nullptr, imp = in.imp_w != nullptr;
  if (l1) return imp ? bwd_launch<PX, true, true>(st, num_sms, a, in) : bwd_launch<PX, true, false>(st, num_sms, a, in);
  return imp ? bwd_launch<PX, false, true>(st, num_sms, a, in) : bwd_launch<PX, false, false>(st, num_sms, a, in);
}

cudaError_t launch_blend_bwd(cudaStream_t st, int variant, int num_sms, const BlendArgs& a, const BwdIn& in) {
  switch (variant) {
    case 3:
      return launch_blend_bwd_warp(st, num_sms, a, in);
    case 4:
      return launch_blend_bwd_cull(st, num_sms, 8, false, a, in);
    case 5:
      return launch_blend_bwd_cull(st, num_sms, 4, false, a, in);
    case 6:
      return launch_blend_bwd_cull(st, num_sms, 4, true, a, in);
    case 1:
      return bwd_dispatch<2>(st, num_sms, a, in);
    case 2:
      return bwd_dispatch<4>(st, num_sms, a, in);
    default:
      return bwd_dispatch<1>(st, num_sms, a, in);
  }
}

}  // namespace airgs
