// Blend backward (sm_103a): the adjoint of the blend forward by a per-tile
// front-to-back replay, one warp per 16x8 half tile, persistent over an atomic
// queue of all (view, half tile) items of a batch.  No per-pixel list is
// stored: each pixel replays its list up to n_contrib with the forward's exact
// arithmetic, recomputing the transmittance T_i.  With R_i the colour still
// ahead after entry i (C_final - P_i, background included):
//     dC/dalpha_i = c_i T_i - R_i / (1 - alpha_i),   dC/dc_i = alpha_i T_i,
// chained through alpha = o G, G = exp(power) to the opacity, the 2D mean and
// the conic; a clamped alpha (o G > alpha_max) passes no gradient to o or G.
//
// Staging uses the forward's exact block masks (stored in the half-list
// entries) restricted to the blocks whose largest n_contrib lies beyond the
// entry's position.  Each entry's ten per-lane sums
//   0 S_x = sum t dx, 1 S_y = sum t dy, 2 sum t dx^2, 3 sum t dx dy,
//   4 sum t dy^2, 5 sum t, 6-8 colour, 9 blend weight
// (t = dL/dalpha G on unclamped pairs) plus its blended-pair count are
// deferred into a per-warp shared-memory table of three entries, reduced by one
// row sum per lane (a transpose through shared memory) and flushed with one
// scalar red.global.add per sum; with power2 = a2 dx^2 + b2 dx dy + c2 dy^2
// and dL/dpower = o t the mean gradient is o ln2 (2 a2 S_x + b2 S_y,
// b2 S_x + 2 c2 S_y).  With L1 the image gradient sign(C - target)/(3 sum H W)
// and the loss are computed from the forward's image and the target in the
// kernel; with IMP the blend weights and counts of the replay are the
// Gaussians' usage frequency.
#include "blend_common.cuh"

namespace airgs {

namespace {

// Table rows 10 f + q hold, per lane (column), sum q of the f-th deferred
// Gaussian; row 30 holds the lanes' blended-pair counts of the three Gaussians
// packed in 8-bit fields (at most 4 pixels per lane and 128 per half tile, so
// the packed sums are integers below 2^24 and exact in single precision).
// Lane s sums row s with eight 16-byte loads (rows padded to 36 floats: each
// 8-lane phase of a 16-byte load touches 32 different banks) and sends it with
// one scalar reduction.
constexpr int kDeferG = 3;
constexpr int kRedStride = 36;

template <bool IMP>
__device__ __forceinline__ void flush_deferred(float (*s_red)[kRedStride], const uint32_t* s_fid, const float4* s_fcon,
                                               int nf, uint32_t cpack, GradRec* gradv, const BwdIn& in, int lane) {
  if (IMP) s_red[30][lane] = (float)cpack;
  __syncwarp();
  const int row = lane < 31 ? lane : 30;
  const float4* rp = reinterpret_cast<const float4*>(&s_red[row][0]);
  float4 s = rp[0];
  float2 s01 = make_float2(s.x, s.y), s23 = make_float2(s.z, s.w);
#pragma unroll
  for (int i = 1; i < 8; ++i) {  // row sums as packed FP32x2 additions
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

}  // namespace

template <bool L1, bool IMP, int CB, int MINB>
__global__ void __launch_bounds__(32, MINB) k_blend_bwd(BlendArgs a, BwdIn in) {
  __shared__ __align__(16) float s_red[kDeferG * 10 + 1][kRedStride];
  __shared__ uint32_t s_fid[kDeferG];
  __shared__ float4 s_fcon[kDeferG];  // (a2, b2, c2, o) of the deferred Gaussians
  __shared__ float4 s_a[CB];
  __shared__ float4 s_b[CB];
  __shared__ StageMeta s_meta[CB];

  const int lane = threadIdx.x;
  const float alpha_max = a.rp.alpha_max, alpha_min = a.rp.alpha_min;
  const float log2_amin = log2f(alpha_min);
  const int lx = lane & 7, ly = lane >> 3;
  unsigned long long pairs = 0, executed = 0;
  float loss_acc = 0.f;

  while (true) {
    const int work = cull_fetch(a.work_counter);
    if (work >= a.n_tiles * 2) break;
    const int item = work >> 1, part = work & 1;
    const int v = view_of_tile_cams(a.cams, a.n_views, item);
    const CamDev& cam = a.cams[v];
    const int lt = item - (int)__ldg(&a.cams[v].tile_base);
    const int X0 = (lt % cam.TW) * kTile, Y0 = (lt / cam.TW) * kTile + part * (kTile / 2);
    const float pxb[2] = {(float)(X0 + lx) + 0.5f, (float)(X0 + 8 + lx) + 0.5f};
    const float pyb[2] = {(float)(Y0 + ly) + 0.5f, (float)(Y0 + 4 + ly) + 0.5f};  // the two block rows
    const int64_t HW = (int64_t)cam.W * cam.H;
    const int64_t base3 = 3 * cam.pix_base;

    float T[kBlocks], gC[kBlocks], g0[kBlocks], g1[kBlocks], g2[kBlocks];
    int nc[kBlocks], gmax[kBlocks];
#pragma unroll
    for (int k = 0; k < kBlocks; ++k) {
      const int x = X0 + 8 * (k & 1) + lx, y = Y0 + 4 * (k >> 1) + ly;
      T[k] = 1.f;
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
    for (int k = 0; k < kBlocks; ++k) maxnc = max(maxnc, gmax[k]);
    const uint2 range = a.ranges[item];
    const bool use_hl = a.hl != nullptr;  // this half's compacted list
    uint2 er = make_uint2(range.x, range.x + (uint32_t)maxnc);
    if (use_hl) er = a.hranges[(int64_t)part * a.n_tiles + item];
    const ProjRec* projv = a.proj + (size_t)v * a.n;
    GradRec* gradv = in.grad + (size_t)v * a.n;
    uint32_t exec_groups = 0;
    bool past_end = false;
    int ns = 0;          // deferred Gaussians in the table
    uint32_t cpack = 0;  // this lane's packed pair counts of those

    for (uint32_t b0 = er.x; b0 < er.y && !past_end; b0 += CB) {
      const int nb = stage_compact<true>(a, use_hl, b0, (int)min((uint32_t)CB, er.y - b0), range.x, projv, log2_amin,
                                         (float)X0, (float)Y0, gmax, maxnc, (1u << kBlocks) - 1u, s_a, s_b, s_meta,
                                         past_end, exec_groups);
      for (int j = 0; j < nb; ++j) {
        const StageMeta me = s_meta[j];
        const int pos1 = (int)me.pos1;  // pair (pixel, entry) replayed iff pos1 <= n_contrib
        const unsigned m = me.mask;
        const float4 ga = s_a[j];
        const float4 gb = s_b[j];
        const float cb = me.c;
        const float dxb[2] = {__fsub_rn(ga.x, pxb[0]), __fsub_rn(ga.x, pxb[1])};
        float acc[10];
        int cnt = 0;
        float2 a01 = make_float2(0.f, 0.f), a24 = a01, a67 = a01;
        acc[3] = acc[5] = acc[8] = acc[9] = 0.f;
#pragma unroll
        for (int by = 0; by < 2; ++by) {
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
        // every compacted entry has a live block: defer without a vote
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
      __syncwarp();
    }
    if (ns > 0) flush_deferred<IMP>(s_red, s_fid, s_fcon, ns, cpack, gradv, in, lane);
    executed += exec_groups;
  }
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kAll, pairs, o);
  for (int o = 16; o > 0; o >>= 1) executed += __shfl_xor_sync(kAll, executed, o);
  executed *= 32ull;  // 32 lane evaluations per block
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

namespace {

template <bool L1, bool IMP, int CB, int MINB>
cudaError_t bwd_launch(cudaStream_t st, int num_sms, const BlendArgs& a, const BwdIn& in) {
  cudaError_t e = prefer_shared(k_blend_bwd<L1, IMP, CB, MINB>);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid(k_blend_bwd<L1, IMP, CB, MINB>, num_sms, a.n_tiles * 2, e);
  if (e != cudaSuccess) return e;
  if (grid > 0) k_blend_bwd<L1, IMP, CB, MINB><<<grid, 32, 0, st>>>(a, in);
  count_launches(1);
  return cudaGetLastError();
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
    case 1: return bwd_dispatch<16, 28>(st, num_sms, a, in);
    case 2: return bwd_dispatch<64, 28>(st, num_sms, a, in);
    case 3: return bwd_dispatch<32, 24>(st, num_sms, a, in);
    case 4: return bwd_dispatch<32, 32>(st, num_sms, a, in);
    default: return bwd_dispatch<32, 28>(st, num_sms, a, in);
  }
}

}  // namespace airgs
