// The clone / split / discard step of keyframe reconstruction (Sec. III-B:
// Gaussians in high-gradient regions are cloned or split, Gaussians of low
// opacity are discarded), with the clone and split rules of the adaptive
// density control of 3D Gaussian Splatting (sm_103a):
//   selected, small (every log scale <= log size_threshold): kept, plus an identical copy
//   selected, large: two children mean + R(q/|q|) diag(exp(log_scale)) z_j,
//                    log_scale - log(split_factor), quaternion, opacity and SH copied
//   logit < logit(min_opacity): discarded with its copy or children.
// Outputs: the kept originals [0, K), the copies [K, K + C), the children
// [K + C, K + C + 2 S) (child 0, child 1 of each split Gaussian), each region in
// index order, with the input index of every output in `parent`.
//
//   k_densify_classify  per Gaussian its class bits, per CTA tile the three counts
//   k_densify_offsets   one CTA: exclusive scan of the tile counts, region sizes, output count
//   k_densify_scatter   per tile: index-ordered offsets inside the tile (blocked scan),
//                       then each Gaussian's parameters read once (coalesced order) and
//                       written to each of its outputs
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

namespace {

#ifndef AIRGS_DS_ITEMS
#define AIRGS_DS_ITEMS 2  // measured best of 1, 2, 4 (0.062, 0.057, 0.059 ms at 300k SH3)
#endif
#ifndef AIRGS_DS_SCATTER_MINB
#define AIRGS_DS_SCATTER_MINB 1  // unbounded (100 registers); bounds for 3 or 4 CTAs per SM spill: 0.064, 0.074 against 0.056 ms
#endif
constexpr int DS_THREADS = 256;
constexpr int DS_ITEMS = AIRGS_DS_ITEMS;  // Gaussians per thread
constexpr int DS_TILE = DS_THREADS * DS_ITEMS;  // Gaussians per CTA
constexpr int DS_SCAN_THREADS = 1024;
constexpr uint32_t kDsKeep = 1u, kDsClone = 2u, kDsSplit = 4u;
constexpr uint32_t kNoPos = 0xFFFFFFFFu;

struct DensifyIn {
  const float* means;
  const float* log_scales;
  const float4* quats;
  const float* opacity_logit;
  const float* sh;
};

struct DensifyOutDev {
  float* means;
  float* log_scales;
  float4* quats;
  float* opacity_logit;
  float* sh;
  uint32_t* parent;  // nullable
};

// Inclusive scan of a (keep, clone, split) triple over the CTA; returns the
// inclusive value of this thread and leaves the CTA total in *total.
template <int THREADS>
__device__ __forceinline__ uint3 cta_scan3(uint3 v, uint3* s_w, uint3* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, v.x, o), b = __shfl_up_sync(0xffffffffu, v.y, o),
                   c = __shfl_up_sync(0xffffffffu, v.z, o);
    if (lane >= o) {
      v.x += a;
      v.y += b;
      v.z += c;
    }
  }
  if (lane == 31) s_w[warp] = v;
  __syncthreads();
  uint3 pre = make_uint3(0u, 0u, 0u), tot = make_uint3(0u, 0u, 0u);
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) {
    const uint3 u = s_w[w];
    if (w < warp) {
      pre.x += u.x;
      pre.y += u.y;
      pre.z += u.z;
    }
    tot.x += u.x;
    tot.y += u.y;
    tot.z += u.z;
  }
  __syncthreads();  // s_w is reused by the caller
  *total = tot;
  return make_uint3(v.x + pre.x, v.y + pre.y, v.z + pre.z);
}

__global__ void __launch_bounds__(DS_THREADS) k_densify_classify(int64_t n, const float* __restrict__ log_scales,
                                                                 const float* __restrict__ logit,
                                                                 const uint8_t* __restrict__ select, float ls_thr,
                                                                 float lo_thr, uint8_t* __restrict__ cls,
                                                                 uint3* __restrict__ tile_counts) {
  __shared__ uint3 s_w[DS_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * DS_TILE;
  uint3 c = make_uint3(0u, 0u, 0u);
#pragma unroll
  for (int j = 0; j < DS_ITEMS; ++j) {
    const int64_t i = base + j * DS_THREADS + threadIdx.x;
    if (i < n) {
      const float l0 = log_scales[3 * i], l1 = log_scales[3 * i + 1], l2 = log_scales[3 * i + 2];
      const bool large = (l0 > ls_thr) || (l1 > ls_thr) || (l2 > ls_thr);
      const bool alive = !(logit[i] < lo_thr);
      const bool sel = select[i] != 0;
      const uint32_t k = (alive && !(sel && large)) ? kDsKeep : 0u;
      const uint32_t cl = (alive && sel && !large) ? kDsClone : 0u;
      const uint32_t sp = (alive && sel && large) ? kDsSplit : 0u;
      cls[i] = (uint8_t)(k | cl | sp);
      c.x += k ? 1u : 0u;
      c.y += cl ? 1u : 0u;
      c.z += sp ? 1u : 0u;
    }
  }
  uint3 tot;
  cta_scan3<DS_THREADS>(c, s_w, &tot);
  if (threadIdx.x == 0) tile_counts[blockIdx.x] = tot;
}

// tile_counts -> exclusive offsets (in place); totals = (K, C, S, K + C + 2 S).
__global__ void __launch_bounds__(DS_SCAN_THREADS) k_densify_offsets(int64_t n_tiles, uint3* __restrict__ tile_counts,
                                                                     uint32_t* __restrict__ totals,
                                                                     int64_t* __restrict__ n_out) {
  __shared__ uint3 s_w[DS_SCAN_THREADS / 32];
  uint3 carry = make_uint3(0u, 0u, 0u);
  for (int64_t c0 = 0; c0 < n_tiles; c0 += DS_SCAN_THREADS) {
    const int64_t t = c0 + threadIdx.x;
    const uint3 v = t < n_tiles ? tile_counts[t] : make_uint3(0u, 0u, 0u);
    uint3 tot;
    const uint3 inc = cta_scan3<DS_SCAN_THREADS>(v, s_w, &tot);
    if (t < n_tiles) tile_counts[t] = make_uint3(carry.x + inc.x - v.x, carry.y + inc.y - v.y, carry.z + inc.z - v.z);
    carry.x += tot.x;
    carry.y += tot.y;
    carry.z += tot.z;
  }
  if (threadIdx.x == 0) {
    totals[0] = carry.x;
    totals[1] = carry.y;
    totals[2] = carry.z;
    totals[3] = carry.x + carry.y + 2u * carry.z;
    *n_out = (int64_t)carry.x + carry.y + 2 * (int64_t)carry.z;
  }
}

// One output Gaussian at row p.
template <int SH3>
__device__ __forceinline__ void write_gaussian(const DensifyOutDev& o, uint32_t p, float mx, float my, float mz,
                                               float l0, float l1, float l2, float4 q, float op,
                                               const float (&shv)[SH3], bool sh_vec, uint32_t parent) {
  o.means[3 * (size_t)p] = mx;
  o.means[3 * (size_t)p + 1] = my;
  o.means[3 * (size_t)p + 2] = mz;
  o.log_scales[3 * (size_t)p] = l0;
  o.log_scales[3 * (size_t)p + 1] = l1;
  o.log_scales[3 * (size_t)p + 2] = l2;
  o.quats[p] = q;
  o.opacity_logit[p] = op;
  float* dst = o.sh + (size_t)p * SH3;
  if constexpr (SH3 % 4 == 0) {
    if (sh_vec) {
#pragma unroll
      for (int k = 0; k < SH3 / 4; ++k)
        reinterpret_cast<float4*>(dst)[k] = make_float4(shv[4 * k], shv[4 * k + 1], shv[4 * k + 2], shv[4 * k + 3]);
    } else {
#pragma unroll
      for (int k = 0; k < SH3; ++k) dst[k] = shv[k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < SH3; ++k) dst[k] = shv[k];
  }
  if (o.parent) o.parent[p] = parent;
}

template <int SH3>
__global__ void __launch_bounds__(DS_THREADS, AIRGS_DS_SCATTER_MINB) k_densify_scatter(int64_t n, DensifyIn in, const uint8_t* __restrict__ cls,
                                                                const uint3* __restrict__ tile_off,
                                                                const uint32_t* __restrict__ totals,
                                                                const float* __restrict__ z, float ls_div, bool sh_vec,
                                                                DensifyOutDev out) {
  __shared__ uint3 s_w[DS_THREADS / 32];
  __shared__ uint32_t s_pos[3][DS_TILE];  // per Gaussian of the tile: kept row, copy row, first child row
  const int64_t base = (int64_t)blockIdx.x * DS_TILE;
  // blocked scan: thread t owns Gaussians base + DS_ITEMS t .., so that the
  // offsets follow the index order
  uint32_t c4[DS_ITEMS];
  uint3 mine = make_uint3(0u, 0u, 0u);
#pragma unroll
  for (int j = 0; j < DS_ITEMS; ++j) {
    const int64_t i = base + DS_ITEMS * threadIdx.x + j;
    c4[j] = i < n ? cls[i] : 0u;
    mine.x += (c4[j] & kDsKeep) ? 1u : 0u;
    mine.y += (c4[j] & kDsClone) ? 1u : 0u;
    mine.z += (c4[j] & kDsSplit) ? 1u : 0u;
  }
  uint3 tot;
  const uint3 inc = cta_scan3<DS_THREADS>(mine, s_w, &tot);
  const uint3 to = tile_off[blockIdx.x];
  const uint32_t K = totals[0], C = totals[1];
  uint32_t pk = to.x + inc.x - mine.x, pc = K + to.y + inc.y - mine.y, ps = K + C + 2u * (to.z + inc.z - mine.z);
#pragma unroll
  for (int j = 0; j < DS_ITEMS; ++j) {
    const int l = DS_ITEMS * threadIdx.x + j;
    s_pos[0][l] = (c4[j] & kDsKeep) ? pk++ : kNoPos;
    s_pos[1][l] = (c4[j] & kDsClone) ? pc++ : kNoPos;
    s_pos[2][l] = (c4[j] & kDsSplit) ? (ps += 2u) - 2u : kNoPos;
  }
  __syncthreads();
  // each Gaussian of the tile in coalesced order: parameters read once, written
  // to each of its rows
#pragma unroll 1
  for (int j = 0; j < DS_ITEMS; ++j) {
    const int l = j * DS_THREADS + threadIdx.x;
    const int64_t i = base + l;
    if (i >= n) break;
    const uint32_t p0 = s_pos[0][l], p1 = s_pos[1][l], p2 = s_pos[2][l];
    if (p0 == kNoPos && p1 == kNoPos && p2 == kNoPos) continue;  // discarded
    const float mx = in.means[3 * i], my = in.means[3 * i + 1], mz = in.means[3 * i + 2];
    const float l0 = in.log_scales[3 * i], l1 = in.log_scales[3 * i + 1], l2 = in.log_scales[3 * i + 2];
    const float4 q = in.quats[i];
    const float op = in.opacity_logit[i];
    float shv[SH3];
    const float* src = in.sh + (size_t)i * SH3;
    if constexpr (SH3 % 4 == 0) {
      if (sh_vec) {
#pragma unroll
        for (int k = 0; k < SH3 / 4; ++k) {
          const float4 v = reinterpret_cast<const float4*>(src)[k];
          shv[4 * k] = v.x;
          shv[4 * k + 1] = v.y;
          shv[4 * k + 2] = v.z;
          shv[4 * k + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < SH3; ++k) shv[k] = src[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < SH3; ++k) shv[k] = src[k];
    }
    if (p0 != kNoPos) write_gaussian<SH3>(out, p0, mx, my, mz, l0, l1, l2, q, op, shv, sh_vec, (uint32_t)i);
    if (p1 != kNoPos) write_gaussian<SH3>(out, p1, mx, my, mz, l0, l1, l2, q, op, shv, sh_vec, (uint32_t)i);
    if (p2 != kNoPos) {
      // children sample the Gaussian: mean + R(q/|q|) (s * z_j), s = exp(log_scale)
      const float qi = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
      const float w = q.x * qi, x = q.y * qi, y = q.z * qi, zq = q.w * qi;
      const float R[9] = {1.f - 2.f * (y * y + zq * zq), 2.f * (x * y - w * zq),       2.f * (x * zq + w * y),
                          2.f * (x * y + w * zq),       1.f - 2.f * (x * x + zq * zq), 2.f * (y * zq - w * x),
                          2.f * (x * zq - w * y),       2.f * (y * zq + w * x),       1.f - 2.f * (x * x + y * y)};
      const float s0 = expf(l0), s1 = expf(l1), s2 = expf(l2);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float* zc = z + (size_t)i * 6 + 3 * c;
        const float u0 = s0 * zc[0], u1 = s1 * zc[1], u2 = s2 * zc[2];
        const float cx = mx + (R[0] * u0 + R[1] * u1 + R[2] * u2);
        const float cy = my + (R[3] * u0 + R[4] * u1 + R[5] * u2);
        const float cz = mz + (R[6] * u0 + R[7] * u1 + R[8] * u2);
        write_gaussian<SH3>(out, p2 + c, cx, cy, cz, l0 - ls_div, l1 - ls_div, l2 - ls_div, q, op, shv, sh_vec,
                            (uint32_t)i);
      }
    }
  }
}

}  // namespace

int64_t densify_tiles(int64_t n) { return (n + DS_TILE - 1) / DS_TILE; }

cudaError_t launch_densify_apply(cudaStream_t st, int64_t n, int sh_degree, const float* means,
                                 const float* log_scales, const float* quats, const float* opacity_logit,
                                 const float* sh, const uint8_t* select, const float* z, float ls_thr, float ls_div,
                                 float lo_thr, uint8_t* cls, uint3* tile_counts, uint32_t* totals, float* o_means,
                                 float* o_log_scales, float* o_quats, float* o_opacity_logit, float* o_sh,
                                 uint32_t* o_parent, int64_t* n_out) {
  if (n == 0) return cudaMemsetAsync(n_out, 0, sizeof(int64_t), st);
  const int64_t tiles = densify_tiles(n);
  k_densify_classify<<<(unsigned)tiles, DS_THREADS, 0, st>>>(n, log_scales, opacity_logit, select, ls_thr, lo_thr, cls,
                                                             tile_counts);
  k_densify_offsets<<<1, DS_SCAN_THREADS, 0, st>>>(tiles, tile_counts, totals, n_out);
  const DensifyIn in{means, log_scales, reinterpret_cast<const float4*>(quats), opacity_logit, sh};
  const DensifyOutDev out{o_means, o_log_scales, reinterpret_cast<float4*>(o_quats), o_opacity_logit, o_sh, o_parent};
  const bool sh_vec = ((reinterpret_cast<uintptr_t>(sh) | reinterpret_cast<uintptr_t>(o_sh)) & 15u) == 0;
  switch (sh_degree) {
    case 0:
      k_densify_scatter<3><<<(unsigned)tiles, DS_THREADS, 0, st>>>(n, in, cls, tile_counts, totals, z, ls_div, sh_vec,
                                                                   out);
      break;
    case 1:
      k_densify_scatter<12><<<(unsigned)tiles, DS_THREADS, 0, st>>>(n, in, cls, tile_counts, totals, z, ls_div, sh_vec,
                                                                    out);
      break;
    case 2:
      k_densify_scatter<27><<<(unsigned)tiles, DS_THREADS, 0, st>>>(n, in, cls, tile_counts, totals, z, ls_div, sh_vec,
                                                                    out);
      break;
    default:
      k_densify_scatter<48><<<(unsigned)tiles, DS_THREADS, 0, st>>>(n, in, cls, tile_counts, totals, z, ls_div, sh_vec,
                                                                    out);
      break;
  }
  count_launches(3);
  return cudaGetLastError();
}

}  // namespace airgs
