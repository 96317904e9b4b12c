// Usage-frequency pruning of streamed deltas (Sec. III-C) and helpers for the
// pruning-level space of Algorithm 1 (sm_103a).
//
//   k_importance_keys  sort keys of the per-Gaussian blend weights (float bits;
//                      weights are non-negative, negative / NaN rank lowest)
//   k_prune_mark       keep[i] = 0 for the n_prune Gaussians of lowest usage
//                      frequency (equal weights: lower index pruned first)
//   k_prune_delta      d'_t = p(D_t - D'_{t-1}) and D'_t = D'_{t-1} + d'_t
//   k_apply_delta      apply float deltas [7][n] to the previous frame or anchor
//   k_sq_err           per-view sum of squared differences of two images
//   k_densify_select   Gaussians whose mean screen-space gradient norm exceeds a threshold
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

__global__ void k_importance_keys(int64_t n, const float* __restrict__ w, uint32_t* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = w[i];
  keys[i] = (x > 0.f) ? __float_as_uint(x) : 0u;  // +0, negatives and NaN rank lowest
}

__global__ void k_prune_mark(int64_t n, int64_t n_prune, const uint32_t* __restrict__ order,
                             uint8_t* __restrict__ keep) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  keep[order[p]] = p >= n_prune ? 1 : 0;
}

__global__ void k_prune_delta(int64_t n, int channels, const float* __restrict__ D_t, float* __restrict__ D_sent,
                              const uint8_t* __restrict__ keep, float* __restrict__ d_out,
                              unsigned long long* __restrict__ nonzero) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool any = false;
  if (i < n) {
    const bool k = keep[i] != 0;
    for (int c = 0; c < channels; ++c) {
      const int64_t o = (int64_t)c * n + i;
      const float d = k ? D_t[o] - D_sent[o] : 0.f;
      d_out[o] = d;
      D_sent[o] += d;
      any |= d != 0.f;
    }
  }
  if (nonzero) {
    const unsigned c = __popc(__ballot_sync(0xffffffffu, any));
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(nonzero, (unsigned long long)c);
  }
}

__global__ void k_apply_delta(int64_t n, const float* __restrict__ delta, int quat_add,
                              const float* __restrict__ base_means, const float* __restrict__ base_quats,
                              float* out_means, float* out_quats) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) v[c] = delta[(int64_t)c * n + i];
  const float m0 = base_means[3 * i], m1 = base_means[3 * i + 1], m2 = base_means[3 * i + 2];
  const float4 q = reinterpret_cast<const float4*>(base_quats)[i];
  out_means[3 * i] = m0 + v[0];
  out_means[3 * i + 1] = m1 + v[1];
  out_means[3 * i + 2] = m2 + v[2];
  float4 r;
  if (quat_add) {
    r = make_float4(q.x + v[3], q.y + v[4], q.z + v[5], q.w + v[6]);
  } else {
    const float dw = v[3], dx = v[4], dy = v[5], dz = v[6];
    r.x = dw * q.x - dx * q.y - dy * q.z - dz * q.w;
    r.y = dw * q.y + dx * q.x + dy * q.w - dz * q.z;
    r.z = dw * q.z - dx * q.w + dy * q.x + dz * q.y;
    r.w = dw * q.w + dx * q.z - dy * q.y + dz * q.x;
    const float inv = rsqrtf(r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w);
    r.x *= inv;
    r.y *= inv;
    r.z *= inv;
    r.w *= inv;
  }
  reinterpret_cast<float4*>(out_quats)[i] = r;
}

// One block row of views: grid.y = view, partial sums in double.
// Sum of squared differences in double-single arithmetic: each thread keeps a
// (hi, lo) float pair, fed by error-free transformations (Knuth's TwoSum for
// a - b and for the running sum, the FMA residual for the square), and the
// threads' pairs are reduced in double.  The work stays on the FP32 pipe (the
// FP64 pipe of this part is a small fraction of it) with a relative error far
// below single precision.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__global__ void __launch_bounds__(256) k_sq_err(const float* __restrict__ a, const float* __restrict__ b,
                                                const int64_t* __restrict__ view_off, double* __restrict__ out) {
  __shared__ double s[8];
  const int v = blockIdx.y;
  const int64_t o0 = view_off[v], o1 = view_off[v + 1];
  float hi = 0.f, lo = 0.f;
  for (int64_t k = o0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < o1; k += (int64_t)gridDim.x * blockDim.x) {
    float dh, dl;
    two_sum(__ldg(a + k), -__ldg(b + k), dh, dl);  // a - b = dh + dl exactly
    const float p = __fmul_rn(dh, dh);
    const float pe = __fmaf_rn(dh, dh, -p);        // dh^2 = p + pe exactly
    const float small = __fmaf_rn(2.f * dh, dl, __fmaf_rn(dl, dl, pe));
    float sh, se;
    two_sum(hi, p, sh, se);
    hi = sh;
    lo = __fadd_rn(lo, __fadd_rn(se, small));
  }
  double acc = (double)hi + (double)lo;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s[w];
    atomicAdd(out + v, t);
  }
}

__global__ void k_densify_select(int64_t n, const float* __restrict__ g, const uint32_t* __restrict__ views,
                                 float threshold, uint8_t* __restrict__ mask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t c = views[i];
  mask[i] = (c > 0 && g[i] > threshold * (float)c) ? 1 : 0;
}

cudaError_t launch_densify_select(cudaStream_t st, int64_t n, const float* g, const uint32_t* views, float threshold,
                                  uint8_t* mask) {
  if (n == 0) return cudaSuccess;
  k_densify_select<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, g, views, threshold, mask);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_prune_mask(cudaStream_t st, int num_sms, int64_t n, int64_t n_prune, const float* w,
                              uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b,
                              uint32_t* scratch, uint8_t* keep) {
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  k_importance_keys<<<blocks, 256, 0, st>>>(n, w, keys_a);
  bool in_b = false;
  cudaError_t e = radix_sort_pairs(st, num_sms, keys_a, vals_a, keys_b, vals_b, n, 1, 32, true, scratch, &in_b);
  if (e != cudaSuccess) return e;
  k_prune_mark<<<blocks, 256, 0, st>>>(n, n_prune, in_b ? vals_b : vals_a, keep);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_prune_delta(cudaStream_t st, int64_t n, int channels, const float* D_t, float* D_sent,
                               const uint8_t* keep, float* d_out, unsigned long long* nonzero) {
  if (n == 0) return cudaSuccess;
  k_prune_delta<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, channels, D_t, D_sent, keep, d_out, nonzero);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_apply_delta(cudaStream_t st, int64_t n, const float* delta, int quat_add, const float* base_means,
                               const float* base_quats, float* out_means, float* out_quats) {
  if (n == 0) return cudaSuccess;
  k_apply_delta<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, delta, quat_add, base_means, base_quats, out_means,
                                                             out_quats);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sq_err(cudaStream_t st, const float* a, const float* b, const int64_t* view_off, int n_views,
                          double* out) {
  if (n_views == 0) return cudaSuccess;
  dim3 grid(256, (unsigned)n_views);  // one view alone still fills the SMs
  k_sq_err<<<grid, 256, 0, st>>>(a, b, view_off, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace airgs
