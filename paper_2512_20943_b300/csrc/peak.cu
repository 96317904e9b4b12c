// FP32 throughput probe (sm_103a): the denominator the blend kernels' roofline
// is read against, measured rather than derived.  Each thread runs 16
// independent FMA chains for `iters` rounds (2 flops per FMA); the grid is 8
// CTAs of 256 threads per SM.  The chains' results are written out so that
// nothing is optimised away.
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

constexpr int PK_CHAINS = 16;
constexpr int PK_THREADS = 256;
constexpr int PK_CTAS_PER_SM = 8;

__global__ void __launch_bounds__(PK_THREADS) k_fp32_probe(float* out, float a, float b, int iters) {
  float s[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s[c] = fmaf(s[c], a, b);
  }
  float t = 0.f;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) t += s[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

cudaError_t measure_fp32_peak(cudaStream_t st, int num_sms, float* scratch, double* tflops) {
  const int blocks = num_sms * PK_CTAS_PER_SM, iters = 4096;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up; keep the fastest
    cudaEventRecord(e0, st);
    k_fp32_probe<<<blocks, PK_THREADS, 0, st>>>(scratch, 0.999f, 1e-3f, iters);
    count_launches(1);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * PK_CHAINS * (double)iters * blocks * PK_THREADS;
  *tflops = flops / (best * 1e-3) / 1e12;
  return cudaSuccess;
}

size_t fp32_probe_words(int num_sms) { return (size_t)num_sms * PK_CTAS_PER_SM * PK_THREADS; }

}  // namespace airgs
