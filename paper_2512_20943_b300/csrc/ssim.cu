// The 3DGS training loss of Eq. 1, L = (1 - lambda) L1 + lambda (1 - SSIM),
// and its gradient with respect to the rendered image (sm_103a).
//
// SSIM per (view, channel) plane with an 11x11 Gaussian window (sigma 1.5,
// weights normalised, zero padding, output the size of the image),
// C1 = 0.01^2, C2 = 0.03^2, averaged over views, pixels and channels; L1 is the
// mean absolute difference.  With local moments mu_x = G*x, m_xx = G*x^2,
// m_xy = G*(x y) (and mu_y, m_yy of the target),
//   A = 2 mu_x mu_y + C1, B = 2 (m_xy - mu_x mu_y) + C2,
//   C = mu_x^2 + mu_y^2 + C1, D = (m_xx - mu_x^2) + (m_yy - mu_y^2) + C2,
//   S = A B / (C D),
// and the gradient is a correlation of the per-pixel partials with the window:
//   dS/dx(q) = (G * P1)(q) + 2 x(q) (G * P2)(q) + y(q) (G * P3)(q),
//   P1 = dS/dmu_x = 2 mu_y (B - A)/(C D) - 2 mu_x S / C + 2 mu_x S / D,
//   P2 = dS/dm_xx = -S / D,   P3 = dS/dm_xy = 2 A / (C D),
// the partials being zero outside the image (zero padding of the second
// correlation).
//
// One CTA per 32x32 output tile of a plane does all four separable passes in
// shared memory: x and y with a halo of 2 radii (52x52), horizontal moments
// (52 rows x 42 columns), vertical moments, SSIM and partials on the 42x42
// region the second correlation needs, horizontal partials (42 x 32), then the
// vertical partials and the combination on the tile.  Each thread walks a strip
// of 4 to 8 outputs along the pass direction, so that a loaded value serves the
// strip's outputs from registers.  Moments and partials are FP32x2 pairs
// ((mu_x, mu_y), (m_xx, m_yy), (P1, P2)), so that a tap is two packed FMAs and
// one scalar, and one reciprocal of C D per point gives 1/C and 1/D.  Global
// memory sees x and y once (plus the halo, from L2) and the gradient written
// once.
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

namespace {

constexpr int SSIM_R = 5;                  // window radius (11 taps)
constexpr int SSIM_TAPS = 2 * SSIM_R + 1;
constexpr int ST = 32;                     // output tile edge
constexpr int MID = ST + 2 * SSIM_R;       // 42: moments / partials region
constexpr int IN = ST + 4 * SSIM_R;        // 52: x, y with their halo
constexpr int IN_S = IN + 1;               // row strides: odd, so that lanes on consecutive rows
constexpr int MID_S = MID + 1;             // of one column hit different banks
constexpr int ST_S = ST + 1;
constexpr int SSIM_THREADS = 320;  // the horizontal moments' 312 strips in one round (256: 0.801 ms, 320: 0.782, 384: 1.004)
constexpr int A_STRIP = 7, A_STRIPS = MID / A_STRIP;  // horizontal moments: 6 strips of 7 columns
constexpr int B_STRIP = 7, B_STRIPS = MID / B_STRIP;  // vertical moments: 6 strips of 7 rows
constexpr int C_STRIP = 8, C_STRIPS = ST / C_STRIP;   // horizontal partials: 4 strips of 8 columns
constexpr int D_STRIP = 4, D_STRIPS = ST / D_STRIP;   // vertical partials: 8 strips of 4 rows
static_assert(MID % A_STRIP == 0 && MID % B_STRIP == 0 && ST % C_STRIP == 0 && ST % D_STRIP == 0, "strips");

// shared layout (floats): region 0 holds x, y as pairs (IN x IN_S float2),
// later the partials P1, P2 as pairs and P3 (MID x MID_S each); region 1 the
// horizontal moments (mu_x, mu_y) and (m_xx, m_yy) as pairs and m_xy
// (IN x MID_S each), later the horizontal partials (MID x ST_S each)
constexpr int REGION0 = 2 * IN * IN_S;
constexpr int REGION1 = 5 * IN * MID_S;
static_assert(3 * MID * MID_S <= REGION0 && 3 * MID * ST_S <= REGION1, "region reuse");
static_assert(REGION0 % 2 == 0 && (2 * MID * MID_S) % 2 == 0 && (4 * IN * MID_S) % 2 == 0, "float2 alignment");
constexpr size_t SSIM_SMEM = (size_t)(REGION0 + REGION1) * sizeof(float);

__constant__ float c_ssim_w[SSIM_TAPS];

struct Planes {
  const int64_t* off;        // [n_planes + 1] first value of each plane
  const int* width;          // [n_planes]
  const int* height;         // [n_planes]
  const int64_t* tile_base;  // [n_planes + 1] first output tile of each plane
  int n_planes;
};

}  // namespace

namespace {

// Plane of output tile b (binary search over the tile bases).
__device__ __forceinline__ int plane_of_tile(const Planes& p, int64_t b) {
  int lo = 0, hi = p.n_planes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.tile_base[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Sums over the CTA (double), added to *dst by one thread.
__device__ __forceinline__ void cta_add(double v, double* s_red, double* dst) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < SSIM_THREADS / 32; ++w) t += s_red[w];
    atomicAdd(dst, t);
  }
}

__global__ void __launch_bounds__(SSIM_THREADS, 2) k_ssim_tile(Planes P, const float* __restrict__ x,
                                                               const float* __restrict__ y, float s_scale,
                                                               float l1_scale, float* __restrict__ grad,
                                                               double* __restrict__ sums) {
  extern __shared__ float sm[];
  __shared__ double s_red[SSIM_THREADS / 32];
  float2* s_xy = reinterpret_cast<float2*>(sm);                       // [IN][IN_S]
  float2* s_p12 = reinterpret_cast<float2*>(sm);                      // [MID][MID_S], after the moments
  float* s_p3 = sm + 2 * MID * MID_S;                                 // [MID][MID_S]
  float2* s_m01 = reinterpret_cast<float2*>(sm + REGION0);            // [IN][MID_S]
  float2* s_m23 = reinterpret_cast<float2*>(sm + REGION0 + 2 * IN * MID_S);
  float* s_m4 = sm + REGION0 + 4 * IN * MID_S;                        // [IN][MID_S]
  float2* s_h12 = reinterpret_cast<float2*>(sm + REGION0);            // [MID][ST_S], after the partials
  float* s_h3 = sm + REGION0 + 2 * MID * ST_S;                        // [MID][ST_S]
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  const int pl = plane_of_tile(P, b);
  const int W = P.width[pl], H = P.height[pl];
  const int64_t o = P.off[pl];
  const int tw = (W + ST - 1) / ST;
  const int lt = (int)(b - P.tile_base[pl]);
  const int X0 = (lt % tw) * ST, Y0 = (lt / tw) * ST;
  float w[SSIM_TAPS];
#pragma unroll
  for (int j = 0; j < SSIM_TAPS; ++j) w[j] = c_ssim_w[j];

  // x and y over image rows Y0 - 2R .. and columns X0 - 2R .., zero outside the
  // image (a fixed trip count, so that every load is issued before the first wait)
  constexpr int LOAD_ITERS = (IN * IN + SSIM_THREADS - 1) / SSIM_THREADS;
#pragma unroll
  for (int li = 0; li < LOAD_ITERS; ++li) {
    const int i = tid + li * SSIM_THREADS;
    if (i >= IN * IN) break;
    const int r = i / IN, c = i - r * IN;
    const int gy = Y0 - 2 * SSIM_R + r, gx = X0 - 2 * SSIM_R + c;
    float2 v = make_float2(0.f, 0.f);
    if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
      const int64_t k = o + (int64_t)gy * W + gx;
      v = make_float2(__ldg(x + k), __ldg(y + k));
    }
    s_xy[r * IN_S + c] = v;
  }
  __syncthreads();

  // horizontal moments: row r, moment column c (image column X0 - R + c) from
  // input columns c .. c + 2R; (mu_x, mu_y) and (m_xx, m_yy) as packed pairs
  for (int it = tid; it < A_STRIPS * IN; it += SSIM_THREADS) {
    const int s = it / IN, r = it - s * IN, c0 = s * A_STRIP;
    float2 a01[A_STRIP], a23[A_STRIP];
    float a4[A_STRIP];
#pragma unroll
    for (int k = 0; k < A_STRIP; ++k) {
      a01[k] = a23[k] = make_float2(0.f, 0.f);
      a4[k] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < A_STRIP + 2 * SSIM_R; ++t) {
      const float2 v = s_xy[r * IN_S + c0 + t];
      const float2 sq = __fmul2_rn(v, v);
      const float xy = v.x * v.y;
#pragma unroll
      for (int k = 0; k < A_STRIP; ++k)
        if (t - k >= 0 && t - k < SSIM_TAPS) {
          const float g = w[t - k];
          a01[k] = __ffma2_rn(make_float2(g, g), v, a01[k]);
          a23[k] = __ffma2_rn(make_float2(g, g), sq, a23[k]);
          a4[k] = fmaf(g, xy, a4[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < A_STRIP; ++k) {
      s_m01[r * MID_S + c0 + k] = a01[k];
      s_m23[r * MID_S + c0 + k] = a23[k];
      s_m4[r * MID_S + c0 + k] = a4[k];
    }
  }
  __syncthreads();

  // vertical moments at region point (rr, c) (image (Y0 - R + rr, X0 - R + c)),
  // SSIM and its partials scaled by dL/dS (zero outside the image); one
  // reciprocal of C D per point gives 1/C = D/(C D) and 1/D = C/(C D)
  float ssim_acc = 0.f;
  for (int it = tid; it < B_STRIPS * MID; it += SSIM_THREADS) {
    const int s = it / MID, c = it - s * MID, r0 = s * B_STRIP;
    float2 m01[B_STRIP], m23[B_STRIP];
    float m4[B_STRIP];
#pragma unroll
    for (int k = 0; k < B_STRIP; ++k) {
      m01[k] = m23[k] = make_float2(0.f, 0.f);
      m4[k] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < B_STRIP + 2 * SSIM_R; ++t) {
      const float2 u01 = s_m01[(r0 + t) * MID_S + c], u23 = s_m23[(r0 + t) * MID_S + c];
      const float u4 = s_m4[(r0 + t) * MID_S + c];
#pragma unroll
      for (int k = 0; k < B_STRIP; ++k)
        if (t - k >= 0 && t - k < SSIM_TAPS) {
          const float g = w[t - k];
          m01[k] = __ffma2_rn(make_float2(g, g), u01, m01[k]);
          m23[k] = __ffma2_rn(make_float2(g, g), u23, m23[k]);
          m4[k] = fmaf(g, u4, m4[k]);
        }
    }
    const int gx = X0 - SSIM_R + c;
    const bool col_in = gx >= 0 && gx < W, col_centre = c >= SSIM_R && c < SSIM_R + ST;
#pragma unroll
    for (int k = 0; k < B_STRIP; ++k) {
      const int rr = r0 + k, gy = Y0 - SSIM_R + rr;
      float p1 = 0.f, p2 = 0.f, p3 = 0.f;
      if (col_in && gy >= 0 && gy < H) {
        const float C1 = 1e-4f, C2 = 9e-4f;
        const float mx = m01[k].x, my = m01[k].y;
        const float A = 2.f * mx * my + C1;
        const float B = 2.f * (m4[k] - mx * my) + C2;
        const float C = mx * mx + my * my + C1;
        const float D = (m23[k].x - mx * mx) + (m23[k].y - my * my) + C2;
        const float inv = 1.f / (C * D);
        const float S = A * B * inv;
        const float inv_c = D * inv, inv_d = C * inv;
        if (col_centre && rr >= SSIM_R && rr < SSIM_R + ST) ssim_acc += S;
        p1 = s_scale * (2.f * my * (B - A) * inv - 2.f * mx * S * inv_c + 2.f * mx * S * inv_d);
        p2 = s_scale * (-S * inv_d);
        p3 = s_scale * (2.f * A * inv);
      }
      s_p12[rr * MID_S + c] = make_float2(p1, p2);
      s_p3[rr * MID_S + c] = p3;
    }
  }
  __syncthreads();

  // horizontal partials: region row rr, tile column c (image column X0 + c) from
  // region columns c .. c + 2R
  for (int it = tid; it < C_STRIPS * MID; it += SSIM_THREADS) {
    const int s = it / MID, rr = it - s * MID, c0 = s * C_STRIP;
    float2 a12[C_STRIP];
    float a3[C_STRIP];
#pragma unroll
    for (int k = 0; k < C_STRIP; ++k) {
      a12[k] = make_float2(0.f, 0.f);
      a3[k] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < C_STRIP + 2 * SSIM_R; ++t) {
      const float2 q12 = s_p12[rr * MID_S + c0 + t];
      const float q3 = s_p3[rr * MID_S + c0 + t];
#pragma unroll
      for (int k = 0; k < C_STRIP; ++k)
        if (t - k >= 0 && t - k < SSIM_TAPS) {
          const float g = w[t - k];
          a12[k] = __ffma2_rn(make_float2(g, g), q12, a12[k]);
          a3[k] = fmaf(g, q3, a3[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < C_STRIP; ++k) {
      s_h12[rr * ST_S + c0 + k] = a12[k];
      s_h3[rr * ST_S + c0 + k] = a3[k];
    }
  }
  __syncthreads();

  // vertical partials at tile pixel (r, c) from region rows r .. r + 2R, combined
  // with x, y and the L1 term into the gradient
  float l1_acc = 0.f;
  for (int it = tid; it < D_STRIPS * ST; it += SSIM_THREADS) {
    const int s = it / ST, c = it - s * ST, r0 = s * D_STRIP;
    const int gx = X0 + c;
    // the strip's x and y, fetched before the correlation so that their latency overlaps it
    float xv[D_STRIP], yv[D_STRIP];
#pragma unroll
    for (int k = 0; k < D_STRIP; ++k) {
      const int gy = Y0 + r0 + k;
      xv[k] = yv[k] = 0.f;
      if (gx < W && gy < H) {
        const int64_t kk = o + (int64_t)gy * W + gx;
        xv[k] = __ldg(x + kk);
        yv[k] = __ldg(y + kk);
      }
    }
    float2 a12[D_STRIP];
    float a3[D_STRIP];
#pragma unroll
    for (int k = 0; k < D_STRIP; ++k) {
      a12[k] = make_float2(0.f, 0.f);
      a3[k] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < D_STRIP + 2 * SSIM_R; ++t) {
      const float2 q12 = s_h12[(r0 + t) * ST_S + c];
      const float q3 = s_h3[(r0 + t) * ST_S + c];
#pragma unroll
      for (int k = 0; k < D_STRIP; ++k)
        if (t - k >= 0 && t - k < SSIM_TAPS) {
          const float g = w[t - k];
          a12[k] = __ffma2_rn(make_float2(g, g), q12, a12[k]);
          a3[k] = fmaf(g, q3, a3[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < D_STRIP; ++k) {
      const int gy = Y0 + r0 + k;
      if (gx < W && gy < H) {
        const int64_t kk = o + (int64_t)gy * W + gx;
        const float d = xv[k] - yv[k];
        l1_acc += fabsf(d);
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        grad[kk] = a12[k].x + 2.f * xv[k] * a12[k].y + yv[k] * a3[k] + l1_scale * sgn;
      }
    }
  }
  cta_add((double)ssim_acc, s_red, sums);
  __syncthreads();  // s_red is reused
  cta_add((double)l1_acc, s_red, sums + 1);
}

__global__ void k_ssim_finalize(const double* __restrict__ sums, int64_t total, float lambda, double* out) {
  const double ssim = sums[0] / (double)total, l1 = sums[1] / (double)total;
  out[0] = (1.0 - lambda) * l1 + lambda * (1.0 - ssim);
  out[1] = l1;
  out[2] = ssim;
}

}  // namespace

cudaError_t launch_ssim_loss(cudaStream_t st, const int64_t* d_off, const int* d_w, const int* d_h,
                             const int64_t* d_tile_base, int n_planes, int64_t total, int64_t n_tiles, const float* x,
                             const float* y, float lambda, double* sums, float* grad) {
  if (total == 0) return cudaSuccess;
  static bool attr_set[kMaxDevicesAttr] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= kMaxDevicesAttr || !attr_set[dev]) {
    e = cudaFuncSetAttribute(k_ssim_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SSIM_SMEM);
    if (e != cudaSuccess) return e;
    if (dev < kMaxDevicesAttr) attr_set[dev] = true;
  }
  float w[SSIM_TAPS];
  double s = 0.0;
  for (int j = -SSIM_R; j <= SSIM_R; ++j) s += exp(-(double)(j * j) / (2.0 * 1.5 * 1.5));
  for (int j = -SSIM_R; j <= SSIM_R; ++j) w[j + SSIM_R] = (float)(exp(-(double)(j * j) / (2.0 * 1.5 * 1.5)) / s);
  e = cudaMemcpyToSymbolAsync(c_ssim_w, w, sizeof(w), 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const Planes P{d_off, d_w, d_h, d_tile_base, n_planes};
  const double inv = 1.0 / (double)total;
  k_ssim_tile<<<(unsigned)n_tiles, SSIM_THREADS, SSIM_SMEM, st>>>(P, x, y, (float)(-lambda * inv),
                                                                 (float)((1.0 - lambda) * inv), grad, sums);
  k_ssim_finalize<<<1, 1, 0, st>>>(sums, total, lambda, sums + 2);
  count_launches(2);
  return cudaGetLastError();
}

// Output tiles of a w x h plane.
int64_t ssim_tiles(int w, int h) { return (int64_t)((w + ST - 1) / ST) * ((h + ST - 1) / ST); }

}  // namespace airgs
