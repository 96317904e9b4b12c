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
//   P2 = dS/dm_xx = -S / D,   P3 = dS/dm_xy = 2 A / (C D).
// Four separable passes: horizontal moments, vertical moments + SSIM map +
// partials, horizontal partials, vertical partials + combination with the L1
// gradient.
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

constexpr int SSIM_R = 5;  // window radius (11 taps)
__constant__ float c_ssim_w[2 * SSIM_R + 1];

struct Planes {
  const int64_t* off;  // [n_planes + 1] first value of each plane
  const int* width;    // [n_planes]
  const int* height;   // [n_planes]
  int n_planes;
};

__device__ __forceinline__ int plane_of(const Planes& p, int64_t k) {
  int lo = 0, hi = p.n_planes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.off[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Pass 1: horizontal blur of x, y, x^2, y^2, x y (five planes of scratch).
__global__ void k_ssim_h1(Planes P, int64_t total, const float* __restrict__ x, const float* __restrict__ y,
                          float* __restrict__ h) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  const int pl = plane_of(P, k);
  const int64_t o = P.off[pl];
  const int W = P.width[pl];
  const int64_t r = (k - o) / W, c = (k - o) - r * W;
  float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int j = -SSIM_R; j <= SSIM_R; ++j) {
    const int64_t cc = c + j;
    if (cc < 0 || cc >= W) continue;
    const float g = c_ssim_w[j + SSIM_R];
    const float a = x[o + r * W + cc], b = y[o + r * W + cc];
    s[0] += g * a;
    s[1] += g * b;
    s[2] += g * a * a;
    s[3] += g * b * b;
    s[4] += g * a * b;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) h[q * total + k] = s[q];
}

// Pass 2: vertical blur, SSIM map and its partials (scaled by dL/dS).
__global__ void __launch_bounds__(256) k_ssim_v1(Planes P, int64_t total, const float* __restrict__ h, float scale,
                                                 float* __restrict__ part, double* __restrict__ ssim_sum) {
  __shared__ double s_w[8];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double local = 0.0;
  if (k < total) {
    const int pl = plane_of(P, k);
    const int64_t o = P.off[pl];
    const int W = P.width[pl], H = P.height[pl];
    const int64_t r = (k - o) / W, c = (k - o) - r * W;
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = -SSIM_R; i <= SSIM_R; ++i) {
      const int64_t rr = r + i;
      if (rr < 0 || rr >= H) continue;
      const float g = c_ssim_w[i + SSIM_R];
#pragma unroll
      for (int q = 0; q < 5; ++q) m[q] += g * h[q * total + o + rr * W + c];
    }
    const float C1 = 1e-4f, C2 = 9e-4f;
    const float mx = m[0], my = m[1];
    const float A = 2.f * mx * my + C1;
    const float B = 2.f * (m[4] - mx * my) + C2;
    const float C = mx * mx + my * my + C1;
    const float D = (m[2] - mx * mx) + (m[3] - my * my) + C2;
    const float S = A * B / (C * D);
    local = S;
    const float P1 = 2.f * my * (B - A) / (C * D) - 2.f * mx * S / C + 2.f * mx * S / D;
    const float P2 = -S / D;
    const float P3 = 2.f * A / (C * D);
    part[k] = scale * P1;
    part[total + k] = scale * P2;
    part[2 * total + k] = scale * P3;
  }
  for (int s = 16; s > 0; s >>= 1) local += __shfl_xor_sync(0xffffffffu, local, s);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    atomicAdd(ssim_sum, t);
  }
}

// Pass 3: horizontal blur of the three partial planes.
__global__ void k_ssim_h2(Planes P, int64_t total, const float* __restrict__ part, float* __restrict__ h) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  const int pl = plane_of(P, k);
  const int64_t o = P.off[pl];
  const int W = P.width[pl];
  const int64_t r = (k - o) / W, c = (k - o) - r * W;
  float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int j = -SSIM_R; j <= SSIM_R; ++j) {
    const int64_t cc = c + j;
    if (cc < 0 || cc >= W) continue;
    const float g = c_ssim_w[j + SSIM_R];
#pragma unroll
    for (int q = 0; q < 3; ++q) s[q] += g * part[q * total + o + r * W + cc];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) h[q * total + k] = s[q];
}

// Pass 4: vertical blur, combination with x and y, plus the L1 gradient.
__global__ void __launch_bounds__(256) k_ssim_v2(Planes P, int64_t total, const float* __restrict__ h,
                                                 const float* __restrict__ x, const float* __restrict__ y,
                                                 float l1_scale, float* __restrict__ grad,
                                                 double* __restrict__ l1_sum) {
  __shared__ double s_w[8];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double local = 0.0;
  if (k < total) {
    const int pl = plane_of(P, k);
    const int64_t o = P.off[pl];
    const int W = P.width[pl], H = P.height[pl];
    const int64_t r = (k - o) / W, c = (k - o) - r * W;
    float g3[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = -SSIM_R; i <= SSIM_R; ++i) {
      const int64_t rr = r + i;
      if (rr < 0 || rr >= H) continue;
      const float g = c_ssim_w[i + SSIM_R];
#pragma unroll
      for (int q = 0; q < 3; ++q) g3[q] += g * h[q * total + o + rr * W + c];
    }
    const float xv = x[k], yv = y[k];
    const float d = xv - yv;
    local = fabs((double)d);
    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    grad[k] = g3[0] + 2.f * xv * g3[1] + yv * g3[2] + l1_scale * sgn;
  }
  for (int s = 16; s > 0; s >>= 1) local += __shfl_xor_sync(0xffffffffu, local, s);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    atomicAdd(l1_sum, t);
  }
}

__global__ void k_ssim_finalize(const double* __restrict__ sums, int64_t total, float lambda, double* out) {
  const double ssim = sums[0] / (double)total, l1 = sums[1] / (double)total;
  out[0] = (1.0 - lambda) * l1 + lambda * (1.0 - ssim);
  out[1] = l1;
  out[2] = ssim;
}

cudaError_t launch_ssim_loss(cudaStream_t st, const int64_t* d_off, const int* d_w, const int* d_h, int n_planes,
                             int64_t total, const float* x, const float* y, float lambda, float* scratch,
                             double* sums, float* grad) {
  if (total == 0) return cudaSuccess;
  float w[2 * SSIM_R + 1];
  double s = 0.0;
  for (int j = -SSIM_R; j <= SSIM_R; ++j) s += exp(-(double)(j * j) / (2.0 * 1.5 * 1.5));
  for (int j = -SSIM_R; j <= SSIM_R; ++j) w[j + SSIM_R] = (float)(exp(-(double)(j * j) / (2.0 * 1.5 * 1.5)) / s);
  cudaError_t e = cudaMemcpyToSymbolAsync(c_ssim_w, w, sizeof(w), 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  Planes P{d_off, d_w, d_h, n_planes};
  const unsigned blocks = (unsigned)((total + 255) / 256);
  float* h = scratch;               // 5 planes
  float* part = scratch + 5 * total;  // 3 planes
  const float inv = (float)(1.0 / (double)total);
  k_ssim_h1<<<blocks, 256, 0, st>>>(P, total, x, y, h);
  k_ssim_v1<<<blocks, 256, 0, st>>>(P, total, h, -lambda * inv, part, sums);
  k_ssim_h2<<<blocks, 256, 0, st>>>(P, total, part, h);
  k_ssim_v2<<<blocks, 256, 0, st>>>(P, total, h, x, y, (1.f - lambda) * inv, grad, sums + 1);
  k_ssim_finalize<<<1, 1, 0, st>>>(sums, total, lambda, sums + 2);
  count_launches(5);
  return cudaGetLastError();
}

}  // namespace airgs
