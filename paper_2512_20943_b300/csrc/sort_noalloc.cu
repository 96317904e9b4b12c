// Allocation-free entry point: the stable radix sort of airgs_sort_pairs with
// its scratch in a fixed device array instead of memory allocated per call.
//
// Some callers cannot allocate device memory while they run: a cudaMalloc or
// cudaFree can synchronise the whole device and stall every other stream, a
// real-time render or streaming loop may not tolerate that, and hosts such as
// engine plug-ins often run under a device-memory budget owned by the host
// application.  This entry point needs no context and allocates nothing; its
// scratch (one ping-pong half of keys + values and the digit counts) lives in
// g_sort_scratch below, which every GPU that loads the library holds until the
// process exits.
#include <cuda_runtime.h>

#include "airgs.h"
#include "airgs_internal.cuh"
#include "kernels.h"

namespace {

constexpr int64_t kMaxPairs = AIRGS_NOALLOC_SORT_MAX_PAIRS;
constexpr size_t kCountWords = 256 * 1024;  // digit counts: 256 digits x up to 1024 CTAs
constexpr size_t kScratchWords = 2 * kMaxPairs + kCountWords;

}  // namespace

// Shared by every call on a device; holds the previous call's contents.
static __device__ __align__(256) uint32_t g_sort_scratch[kScratchWords];

extern "C" int airgs_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                        uint32_t* vals_out, int64_t n, int key_bits, void* stream) {
  if (n < 0 || key_bits < 1 || key_bits > 32) return AIRGS_E_ARG;
  if (n > kMaxPairs) return AIRGS_E_CAPACITY;
  if (n == 0) return AIRGS_OK;
  if (!keys_in || !vals_in || !keys_out || !vals_out) return AIRGS_E_ARG;
  // The array's name is only a host-side stand-in: its device address is
  // looked up on every call, with the caller's device current.  The lookup is a
  // host-side table read that allocates nothing, and doing it per call keeps
  // the address right under whatever context is current (a cached address
  // would dangle after cudaDeviceReset, which loads the module again).  The
  // first call in a context may load the library's device code: make it before
  // any stream capture.
  int dev = 0;
  void* p = nullptr;
  int sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || p == nullptr ||
      sms <= 0) {
    cudaGetLastError();
    return AIRGS_E_CUDA;
  }
  if (airgs::radix_scratch_bytes(n, 1, sms) > kCountWords * sizeof(uint32_t)) return AIRGS_E_CAPACITY;
  uint32_t* sk = static_cast<uint32_t*>(p);  // scratch keys  [kMaxPairs]
  uint32_t* sv = sk + kMaxPairs;             // scratch values [kMaxPairs]
  uint32_t* counts = sk + 2 * kMaxPairs;     // digit counts, fully rewritten by every pass
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // Ping-pong so that the last pass writes the caller's outputs and the inputs
  // are only read: odd pass counts start in -> out, even ones in -> scratch.
  const int passes = (key_bits + 7) / 8;
  const uint32_t* ki = keys_in;
  const uint32_t* vi = vals_in;
  bool to_out = (passes % 2) == 1;
  for (int pass = 0; pass < passes; ++pass) {
    uint32_t* ko = to_out ? keys_out : sk;
    uint32_t* vo = to_out ? vals_out : sv;
    cudaError_t e = airgs::radix_sort_pass(st, sms, ki, vi, ko, vo, n, 8 * pass, key_bits, counts);
    if (e != cudaSuccess) return AIRGS_E_CUDA;
    ki = ko;
    vi = vo;
    to_out = !to_out;
  }
  return AIRGS_OK;
}
