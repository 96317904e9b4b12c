// Throughput probes (sm_103a): the denominators the blend kernels' roofline is
// read against, measured rather than derived.
//
// FP32: each thread runs 16 independent FMA chains for `iters` rounds (2 flops
// per FMA); the grid is 8 CTAs of 256 threads per SM.  The chains' results are
// written out so that nothing is optimised away.
//
// Shared memory: each thread issues 16-byte shared loads of consecutive words,
// 512 bytes per warp instruction and no bank conflict, 4 per round for `iters`
// rounds, summing them; 4 CTAs of 256 threads per SM, each over its own 16 KB
// table.  The loads are ld.volatile: the same addresses repeat every round, and
// plain loads could be merged or hoisted out of the loop.
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

constexpr int LP_THREADS = 256;
constexpr int LP_CTAS_PER_SM = 4;
constexpr int LP_WORDS = 1024;  // 16-byte words per CTA table (16 KB)
constexpr int LP_LOADS = 4;     // loads per round: words tid + j * LP_THREADS, j < LP_LOADS (< LP_WORDS)

__global__ void __launch_bounds__(LP_THREADS) k_smem_probe(float* out, int iters) {
  __shared__ float4 s_t[LP_WORDS];
  for (int k = threadIdx.x; k < LP_WORDS; k += LP_THREADS)
    s_t[k] = make_float4((float)k, (float)(k + 1), (float)(k + 2), (float)(k + 3));
  __syncthreads();
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(&s_t[0]);
  float2 a0 = make_float2(0.f, 0.f), a1 = a0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < LP_LOADS; ++j) {
      const uint32_t addr = base + 16u * (threadIdx.x + (uint32_t)j * LP_THREADS);
      float4 v;
      asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                   : "r"(addr));
      a0 = __fadd2_rn(a0, make_float2(v.x, v.y));
      a1 = __fadd2_rn(a1, make_float2(v.z, v.w));
    }
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = a0.x + a0.y + a1.x + a1.y;
}

cudaError_t measure_smem_peak(cudaStream_t st, int num_sms, float* scratch, double* tbs) {
  static_assert((LP_LOADS - 1) * LP_THREADS + LP_THREADS <= LP_WORDS, "probe loads stay inside the table");
  const int blocks = num_sms * LP_CTAS_PER_SM, iters = 4096;
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
    k_smem_probe<<<blocks, LP_THREADS, 0, st>>>(scratch, iters);
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
  const double bytes = 16.0 * LP_LOADS * (double)iters * blocks * LP_THREADS;
  *tbs = bytes / (best * 1e-3) / 1e12;
  return cudaSuccess;
}

size_t smem_probe_words(int num_sms) { return (size_t)num_sms * LP_CTAS_PER_SM * LP_THREADS; }

}  // namespace airgs
