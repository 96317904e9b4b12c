// Blend backward (sm_103a): the adjoint of the blend forward by a per-tile
// front-to-back replay, persistent over an atomic queue of all (view, item)
// work items of a batch.  No per-pixel list is stored: each pixel replays its
// list up to n_contrib with the forward's exact arithmetic, recomputing the
// transmittance T_i.  With R_i the colour still ahead after entry i
// (C_final - P_i, background included):
//     dC/dalpha_i = c_i T_i - R_i / (1 - alpha_i),   dC/dc_i = alpha_i T_i,
// chained through alpha = o G, G = exp(power) to the opacity, the 2D mean and
// the conic; a clamped alpha (o G > alpha_max) passes no gradient to o or G.
//
// One warp replays a 16x8 half tile (four 8x4 blocks, a lane's four pixels),
// walking the half's compacted list with the forward's exact block masks
// stored in its entries, restricted to the blocks whose largest n_contrib lies
// beyond the entry's position.  Each entry's ten per-lane sums, in five pairs
//   (S_x = sum t dx, S_y = sum t dy), (sum t dx^2, sum t dy^2),
//   (sum t, blend weight), (colour r, g), (colour b, sum t dx dy)
// (t = dL/dalpha G on unclamped pairs) are deferred into a per-warp
// shared-memory table of three entries with one 8-byte store per pair, reduced
// by two lanes per pair (a transpose through shared memory), each adding its
// half of the pair with one 8-byte vector reduction into the Gaussian's
// gradient record (the projection adjoint applies the 2D coefficients); the entry's blended-pair
// count is a warp reduction of the lanes' counts.  With L1 the image gradient
// sign(C - target)/(3 sum H W) and the loss are computed from the forward's
// image and the target in the kernel; with IMP the blend weights and counts of
// the replay, the Gaussians' usage frequency, go to the record's weight and
// count slots, which the projection adjoint adds to the caller's accumulators.
#include "blend_common.cuh"

#include <cstddef>
#include <type_traits>

namespace airgs {

namespace {

// Row 5 f + p of the table holds, per lane, sum pair p of the f-th deferred
// Gaussian: lanes 0-15 at float2 slots 0-15, lanes 16-31 at slots 18-33 (rows
// of 36 float2 = 72 words, 8 banks apart; the 16-byte gap before the upper
// half puts the two halves 4 banks apart, so each 8-lane phase of the flush's
// 16-byte loads touches 32 different banks).  In the flush lanes 2i and 2i+1
// sum row i over lanes 0-15 and 16-31 (eight 16-byte loads each) and each adds
// its part of pair p to the record's floats 2p, 2p + 1 with one 8-byte vector
// reduction (trading components by shuffle for one scalar reduction per sum
// cost 2 % more time); with IMP pair 2 holds the blend weight in the record's
// weight slot, and the even lane of that pair also adds the entry's
// blended-pair count to the count slot.
constexpr int kDeferG = 3;
constexpr int kPairRows = kDeferG * 5;
constexpr int kPairStride = 36;  // float2 slots per row

__device__ __forceinline__ int table_slot(int lane) { return lane + ((lane >> 4) << 1); }

template <bool IMP>
__device__ __forceinline__ void flush_deferred(float2 (*s_tab)[kPairStride], const uint2* s_fmeta, int nf,
                                               GradRec* gradv, int lane) {
  __syncwarp();
  const int row = lane < 2 * kPairRows ? lane >> 1 : kPairRows - 1, h = lane & 1;
  const float4* rp = reinterpret_cast<const float4*>(&s_tab[row][18 * h]);
  float4 u = rp[0];
  float2 s0 = make_float2(u.x, u.y), s1 = make_float2(u.z, u.w);
#pragma unroll
  for (int i = 1; i < 8; ++i) {  // the half row's 16 pairs as packed FP32x2 additions
    u = rp[i];
    s0 = __fadd2_rn(s0, make_float2(u.x, u.y));
    s1 = __fadd2_rn(s1, make_float2(u.z, u.w));
  }
  const float2 ps = __fadd2_rn(s0, s1);  // this half row's part of sum pair p, both components
  const int f = row / 5, p = row - 5 * f;
  static_assert(kGradWeightSlot == 5, "pair 2 of an entry holds its blend weight");
  if (lane < 10 * nf) {
    const uint2 fm = s_fmeta[f];  // (Gaussian id, blended pairs)
    float* rec = reinterpret_cast<float*>(gradv + fm.x);
    atomicAdd(reinterpret_cast<float2*>(rec) + p, ps);  // one 8-byte reduction per half row
    if (IMP && p == 2 && h == 0)
      asm volatile("red.global.add.u32 [%0], %1;" ::"l"(rec + kGradCountSlot), "r"(fm.y) : "memory");
  }
  __syncwarp();  // the table is refilled after this
}

// Defers one replayed entry into slot ns of the table.
__device__ __forceinline__ void defer_entry(float2 (*s_tab)[kPairStride], uint2* s_fmeta, int ns, int slot,
                                            const float2 (&acc)[5], uint32_t id, int cnt) {
#pragma unroll
  for (int p = 0; p < 5; ++p) s_tab[5 * ns + p][slot] = acc[p];
  // every lane stores the same value (one shared-memory word pair, no branch)
  s_fmeta[ns] = make_uint2(id, (uint32_t)cnt);
}

// Replays one staged entry over the blocks of its mask m (non-zero; block k =
// 2 by + bx, the lane's pixel of block k at (pxb[bx], pyb[by])) with the
// forward's arithmetic: updates each pixel's T and colour still ahead (gC,
// dotted with the image gradient g), returns the lane's ten sums in five pairs
// (acc) and, with IMP, the warp's blended-pair count in cnt (warp-uniform).
template <bool IMP>
__device__ __forceinline__ void replay_entry(const float4 ga, const float4 gb, float cb, int pos1, unsigned m,
                                             const float (&pxb)[2], const float (&pyb)[2], float alpha_max,
                                             float alpha_min, float (&T)[kBlocks], float (&gC)[kBlocks],
                                             const float (&g0)[kBlocks], const float (&g1)[kBlocks],
                                             const float (&g2)[kBlocks], const int (&nc)[kBlocks],
                                             float2 (&acc)[5], int& cnt) {
  const float dxb[2] = {__fsub_rn(ga.x, pxb[0]), __fsub_rn(ga.x, pxb[1])};
  float2 a01, a24, a59, a67, a83;  // assigned by the entry's first block
  int lcnt;
  // one block: the lane's pixel of block k (column bx) against the entry; INIT:
  // the entry's first block, which assigns the sums instead of adding to them
  auto block = [&](auto init, int k, int bx, float dy, float b2dy, float c2dy2) {
    constexpr bool INIT = decltype(init)::value;
    const float dx = dxb[bx];
    const float p2 = power2_of(dx, ga.z, b2dy, c2dy2);
    const float G = ex2_approx(p2);
    const float oG = __fmul_rn(gb.y, G);
    const float alpha = alpha_of(gb.y, G, alpha_max);
    // pair (pixel, entry) replayed iff pos1 <= n_contrib and the forward blended it
    const bool valid = (pos1 <= nc[k]) && !(alpha < alpha_min);
    const float ae = valid ? alpha : 0.f;
    const float w = blend_weight(ae, T[k]);
    const float gc = g0[k] * gb.z + g1[k] * gb.w + g2[k] * cb;
    // independent sums in pairs: one packed FP32x2 operation each
    if (INIT) {
      a67 = __fmul2_rn(make_float2(w, w), make_float2(g0[k], g1[k]));
      a83.x = w * g2[k];
    } else {
      a67 = __ffma2_rn(make_float2(w, w), make_float2(g0[k], g1[k]), a67);
      a83.x = fmaf(w, g2[k], a83.x);
    }
    // gC[k] holds the colour still ahead of the replay, R = gC - gP
    gC[k] = fmaf(-gc, w, gC[k]);
    const float dL_dalpha = fmaf(-gC[k], rcp_approx_ftz(__fsub_rn(1.0f, ae)), T[k] * gc);
    T[k] = transmit(T[k], w);
    // t = dL/dalpha G on unclamped replayed pairs, whose ae equals o G
    // exactly (a clamped pair has ae = alpha_max < o G, a skipped one 0)
    const float tt = dL_dalpha * (ae == oG ? G : 0.f);
    const float2 d2 = make_float2(dx, dy);
    const float2 td = __fmul2_rn(make_float2(tt, tt), d2);  // (t dx, t dy)
    if (INIT) {
      a01 = td;
      a24 = __fmul2_rn(td, d2);
      a83.y = td.x * dy;
    } else {
      a01 = __fadd2_rn(a01, td);
      a24 = __ffma2_rn(td, d2, a24);
      a83.y = fmaf(td.x, dy, a83.y);
    }
    if (IMP) {
      if (INIT) {
        a59 = make_float2(tt, w);
        lcnt = valid ? 1 : 0;
      } else {
        a59 = __fadd2_rn(a59, make_float2(tt, w));
        if (valid) ++lcnt;
      }
    } else {
      if (INIT) {
        a59 = make_float2(tt, 0.f);
        lcnt = 0;
      } else {
        a59.x += tt;
      }
    }
  };
  using First = std::integral_constant<bool, true>;
  using Next = std::integral_constant<bool, false>;
  // the row's live blocks (warp-uniform): both, or one of them; m != 0
  auto row = [&](auto first, int by, unsigned rm) {
    float dy, b2dy, c2dy2;  // shared by the row's two blocks
    row_terms(ga.y, pyb[by], ga.w, gb.x, dy, b2dy, c2dy2);
    if (rm == 3u) {
      block(first, 2 * by, 0, dy, b2dy, c2dy2);
      block(Next{}, 2 * by + 1, 1, dy, b2dy, c2dy2);
    } else if (rm == 1u) {
      block(first, 2 * by, 0, dy, b2dy, c2dy2);
    } else {
      block(first, 2 * by + 1, 1, dy, b2dy, c2dy2);
    }
  };
  const unsigned r0 = m & 3u, r1 = (m >> 2) & 3u;
  if (r0) {
    row(First{}, 0, r0);
    if (r1) row(Next{}, 1, r1);
  } else {
    row(First{}, 1, r1);
  }
  acc[0] = a01;
  acc[1] = a24;
  acc[2] = a59;
  acc[3] = a67;
  acc[4] = a83;
  cnt = IMP ? (int)__reduce_add_sync(kAll, (unsigned)lcnt) : 0;
}

// Per-pixel state of a replay at the start of an item: T = 1, the image
// gradient g (from the L1 target or the given dL/dC), gC = g . C_final and
// n_contrib (0 outside the image); adds the pixel's list length to `pairs` and
// |C - target| to the loss.
template <bool L1>
__device__ __forceinline__ void load_pixel(const BwdIn& in, const CamDev& cam, int x, int y, float& T, float& gC,
                                           float& g0, float& g1, float& g2, int& nc, unsigned long long& pairs,
                                           float& loss_acc) {
  T = 1.f;
  g0 = g1 = g2 = gC = 0.f;
  nc = 0;
  if (x < cam.W && y < cam.H) {
    const int64_t HW = (int64_t)cam.W * cam.H;
    const int64_t base3 = 3 * cam.pix_base;
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
    g0 = gg[0];
    g1 = gg[1];
    g2 = gg[2];
    gC = gg[0] * cf[0] + gg[1] * cf[1] + gg[2] * cf[2];
    nc = in.ncontrib[cam.pix_base + pix];
    pairs += (unsigned long long)nc;
  }
}

// The warp's running statistics, kept in shared memory so that no register
// holds them through the replay: replayed pairs and, with L1, the loss.
struct WarpTotals {
  unsigned long long pairs;
  float loss;
};

// Adds an item's replayed pairs and loss to the warp's totals (at the item's
// start).
template <bool L1>
__device__ __forceinline__ void item_counters(WarpTotals& t, unsigned long long pairs, float loss_acc, int lane) {
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kAll, pairs, o);
  if (L1)
    for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(kAll, loss_acc, o);
  if (lane == 0) {
    t.pairs += pairs;
    if (L1) t.loss += loss_acc;
  }
}

// Adds the warp's totals and issued block evaluations (32 lane evaluations
// each) to the launch counters.
template <bool L1>
__device__ __forceinline__ void finish_counters(const BlendArgs& a, const BwdIn& in, const WarpTotals& t,
                                                uint32_t groups, int lane) {
  unsigned long long executed = groups;
  for (int o = 16; o > 0; o >>= 1) executed += __shfl_xor_sync(kAll, executed, o);
  if (lane == 0) {
    if (a.exec_total && executed) atomicAdd(a.exec_total, 32ull * executed);
    if (t.pairs) {
      atomicAdd(a.pair_counter, t.pairs);
      if (a.pair_total) atomicAdd(a.pair_total, t.pairs);
    }
    if (L1 && in.loss) atomicAdd(in.loss, t.loss * in.inv_norm);
  }
}

}  // namespace

template <bool L1, bool IMP, int CB, int MINB>
__global__ void __launch_bounds__(32, MINB) k_blend_bwd(BlendArgs a, BwdIn in) {
  // the warp's shared memory as one block, the table first (measured 1.4 %
  // faster than separate arrays); the flush reads the table with 16-byte loads
  struct __align__(16) WarpSmem {
    alignas(16) float2 tab[kPairRows][kPairStride];
    float4 a[CB];
    float4 b[CB];
    StageMeta meta[CB];
    uint2 fmeta[kDeferG];  // (Gaussian id, blended pairs) of the deferred entries
    int gmax[kBlocks];     // largest n_contrib of each block
    WarpTotals tot;
  };
  static_assert(offsetof(WarpSmem, tab) % 16 == 0 && (kPairStride * sizeof(float2)) % 16 == 0 &&
                    offsetof(WarpSmem, a) % 16 == 0 && offsetof(WarpSmem, b) % 16 == 0 &&
                    offsetof(WarpSmem, meta) % 16 == 0,
                "16-byte shared loads need 16-byte aligned rows and records");
  __shared__ WarpSmem sw;
  auto& s_tab = sw.tab;
  uint2* s_fmeta = sw.fmeta;
  float4* s_a = sw.a;
  float4* s_b = sw.b;
  StageMeta* s_meta = sw.meta;
  int* s_gmax = sw.gmax;
  WarpTotals& s_tot = sw.tot;

  const int lane = threadIdx.x;
  const int slot = table_slot(lane);
  const float alpha_max = a.rp.alpha_max, alpha_min = a.rp.alpha_min;
  const float log2_amin = log2f(alpha_min);
  const int lx = lane & 7, ly = lane >> 3;
  uint32_t exec_groups = 0;
  if (lane == 0) s_tot = WarpTotals{0ull, 0.f};

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

    float T[kBlocks], gC[kBlocks], g0[kBlocks], g1[kBlocks], g2[kBlocks];
    int nc[kBlocks];
    int maxnc = 0;
    {
      unsigned long long pairs = 0;
      float loss_acc = 0.f;
#pragma unroll
      for (int k = 0; k < kBlocks; ++k) {
        load_pixel<L1>(in, cam, X0 + 8 * (k & 1) + lx, Y0 + 4 * (k >> 1) + ly, T[k], gC[k], g0[k], g1[k], g2[k],
                       nc[k], pairs, loss_acc);
        const int gm = (int)__reduce_max_sync(kAll, (unsigned)nc[k]);  // warp-uniform
        if (lane == k) s_gmax[k] = gm;
        maxnc = max(maxnc, gm);
      }
      item_counters<L1>(s_tot, pairs, loss_acc, lane);
    }
    __syncwarp();
    const uint2 range = a.ranges[item];
    const bool use_hl = a.hl != nullptr;  // this half's compacted list
    uint2 er = make_uint2(range.x, range.x + (uint32_t)maxnc);
    if (use_hl) er = a.hranges[(int64_t)part * a.n_tiles + item];
    const ProjRec* projv = a.proj + (size_t)v * a.n;
    GradRec* gradv = in.grad + (size_t)v * a.n;
    bool past_end = false;
    int ns = 0;  // deferred Gaussians in the table

    for (uint32_t b0 = er.x; b0 < er.y && !past_end; b0 += CB) {
      const int nb = stage_compact<true>(a, use_hl, b0, (int)min((uint32_t)CB, er.y - b0), range.x, projv, log2_amin,
                                         (float)X0, (float)Y0, s_gmax, maxnc, (1u << kBlocks) - 1u, s_a, s_b, s_meta,
                                         past_end, exec_groups);
      for (int j = 0; j < nb; ++j) {
        const StageMeta me = s_meta[j];
        const float4 ga = s_a[j];
        const float4 gb = s_b[j];
        float2 acc[5];
        int cnt;
        replay_entry<IMP>(ga, gb, me.c, (int)me.pos1, me.mask, pxb, pyb, alpha_max, alpha_min, T, gC, g0, g1, g2, nc,
                          acc, cnt);
        // every compacted entry has a live block: defer without a vote
        defer_entry(s_tab, s_fmeta, ns, slot, acc, me.id, cnt);
        if (++ns == kDeferG) {
          flush_deferred<IMP>(s_tab, s_fmeta, ns, gradv, lane);
          ns = 0;
        }
      }
      __syncwarp();
    }
    if (ns > 0) flush_deferred<IMP>(s_tab, s_fmeta, ns, gradv, lane);
  }
  __syncwarp();
  finish_counters<L1>(a, in, s_tot, exec_groups, lane);
}

namespace {

template <class K>
cudaError_t launch_persistent(K kernel, int64_t items, cudaStream_t st, int num_sms, const BlendArgs& a,
                              const BwdIn& in) {
  cudaError_t e = prefer_shared(kernel);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid(kernel, num_sms, items, e);
  if (e != cudaSuccess) return e;
  if (grid > 0) kernel<<<grid, 32, 0, st>>>(a, in);
  count_launches(1);
  return cudaGetLastError();
}

template <bool L1, bool IMP, int CB, int MINB>
cudaError_t bwd_launch(cudaStream_t st, int num_sms, const BlendArgs& a, const BwdIn& in) {
  return launch_persistent(k_blend_bwd<L1, IMP, CB, MINB>, a.n_tiles * 2, st, num_sms, a, in);
}

template <int CB, int MINB>
cudaError_t bwd_dispatch(cudaStream_t st, int num_sms, const BlendArgs& a, const BwdIn& in) {
  const bool l1 = in.target != nullptr, imp = in.imp_w != nullptr;
  if (l1)
    return imp ? bwd_launch<true, true, CB, MINB>(st, num_sms, a, in)
               : bwd_launch<true, false, CB, MINB>(st, num_sms, a, in);
  return imp ? bwd_launch<false, true, CB, MINB>(st, num_sms, a, in)
             : bwd_launch<false, false, CB, MINB>(st, num_sms, a, in);
}

}  // namespace

// The compiled backward shapes (kBwdShapes in kernels.h): staged entries per
// batch and warps per SM (the register bound).
cudaError_t launch_blend_bwd(cudaStream_t st, int shape, int num_sms, const BlendArgs& a, const BwdIn& in) {
  switch (shape) {
    case 1: return bwd_dispatch<16, 32>(st, num_sms, a, in);
    case 2: return bwd_dispatch<64, 32>(st, num_sms, a, in);
    case 3: return bwd_dispatch<32, 28>(st, num_sms, a, in);
    case 4: return bwd_dispatch<32, 24>(st, num_sms, a, in);
    default: return bwd_dispatch<32, 32>(st, num_sms, a, in);
  }
}

}  // namespace airgs
