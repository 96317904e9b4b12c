// Per-tile ordering of (tile, Gaussian) instances (sm_103a).
//
// The blend needs every tile's Gaussians in (depth, index) order.  Instead of
// sorting all instances globally, this path builds each tile's list in place:
//   1. k_project counts the instances of every tile (atomics);
//   2. k_tile_chunk_sums + scan + k_tile_offsets turn the counts into the tile
//      ranges [start, end) (and a cursor per tile, the longest list and the
//      tiles too long for one 256-thread CTA);
//   3. k_scatter writes each instance (depth bits, Gaussian id), one 8-byte
//      pair, to its tile's segment through the tile's atomic cursor (arbitrary
//      order);
//   4. k_sort_tiles sorts each segment by the 64-bit key (depth bits, id) in
//      shared memory with a bitonic network and writes the ids back in order.
// Ids are distinct within a view, so (depth, id) is a total order: the result
// is exactly the stable (depth, index) order of the definition.  Tiles longer
// than kTileSortBig entries are handled by the two-stage radix path instead
// (the host picks the path after reading the longest list).
#include "airgs_internal.cuh"
#include "kernels.h"

namespace airgs {

constexpr int OF_THREADS = 1024;
constexpr int OF_CHUNK = 4096;

size_t tile_offsets_chunks(int64_t n_tiles) { return (size_t)((n_tiles + OF_CHUNK - 1) / OF_CHUNK); }

__global__ void __launch_bounds__(OF_THREADS) k_tile_chunk_sums(const uint32_t* __restrict__ counts,
                                                               int64_t n_tiles, uint64_t* __restrict__ sums) {
  __shared__ uint64_t s_w[OF_THREADS / 32];
  const int64_t c0 = (int64_t)blockIdx.x * OF_CHUNK;
  uint64_t s = 0;
  for (int k = threadIdx.x; k < OF_CHUNK; k += OF_THREADS)
    if (c0 + k < n_tiles) s += counts[c0 + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < OF_THREADS / 32; ++w) t += s_w[w];
    sums[blockIdx.x] = t;
  }
}

// info[0] = longest list, info[1] = number of tiles longer than kTileSortSmall.
__global__ void __launch_bounds__(OF_THREADS) k_tile_offsets(const uint32_t* __restrict__ counts, int64_t n_tiles,
                                                            const uint64_t* __restrict__ chunk_offsets,
                                                            uint2* __restrict__ ranges, uint32_t* __restrict__ cursor,
                                                            uint32_t* __restrict__ big_list,
                                                            uint32_t* __restrict__ info) {
  constexpr int PER = OF_CHUNK / OF_THREADS;  // consecutive tiles per thread
  __shared__ uint32_t s_w[OF_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t t0 = (int64_t)blockIdx.x * OF_CHUNK + (int64_t)tid * PER;
  uint32_t c[PER], local = 0, mx = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    c[k] = (t0 + k < n_tiles) ? counts[t0 + k] : 0u;
    local += c[k];
    mx = max(mx, c[k]);
  }
  uint32_t x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t ws = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += y;
    }
    s_w[lane] = ws;
  }
  __syncthreads();
  uint64_t start = chunk_offsets[blockIdx.x] + (warp ? s_w[warp - 1] : 0) + (x - local);
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    if (t0 + k < n_tiles) {
      ranges[t0 + k] = make_uint2((uint32_t)start, (uint32_t)(start + c[k]));
      cursor[t0 + k] = (uint32_t)start;
      if (c[k] > (uint32_t)kTileSortSmall) big_list[atomicAdd(info + 1, 1u)] = (uint32_t)(t0 + k);
    }
    start += c[k];
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0 && mx) atomicMax(info, mx);
}

// One thread per (view, Gaussian): every instance goes to its tile's segment.
__global__ void __launch_bounds__(256) k_scatter(int64_t total, int64_t n, const ProjRec* __restrict__ proj,
                                                const CamDev* __restrict__ cams,
                                                const uint32_t* __restrict__ depth_keys, uint32_t* cursor,
                                                uint2* __restrict__ pairs) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= total) return;
  const int v = (int)(o / n);
  const uint32_t gid = (uint32_t)(o - (int64_t)v * n);
  const ProjRec rec = proj[o];
  const int radius = __float_as_int(rec.c.z);
  if (!(__float_as_int(rec.c.w) & kFlagVisible)) return;
  const CamDev& cam = cams[v];
  int x0, y0, x1, y1;
  tile_rect(rec.a.x, rec.a.y, radius, cam.TW, cam.TH, x0, y0, x1, y1);
  const uint32_t dk = depth_keys[o];
  uint32_t* cur = cursor + cam.tile_base;
  for (int ty = y0; ty < y1; ++ty)
    for (int tx = x0; tx < x1; ++tx) {
      const uint32_t slot = atomicAdd(cur + ty * cam.TW + tx, 1u);
      pairs[slot] = make_uint2(dk, gid);
    }
}

// Bitonic sort of one tile's (depth bits, id) pairs in shared memory.
template <int THREADS>
__device__ __forceinline__ void sort_segment(unsigned long long* s, uint32_t n, uint32_t start,
                                             const uint2* __restrict__ pairs, uint32_t* __restrict__ vals) {
  uint32_t P = 1;
  while (P < n) P <<= 1;
  for (uint32_t i = threadIdx.x; i < P; i += THREADS) {
    if (i < n) {
      const uint2 kv = pairs[start + i];
      s[i] = ((unsigned long long)kv.x << 32) | kv.y;
    } else {
      s[i] = ~0ull;
    }
  }
  __syncthreads();
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const uint32_t lj = __ffs(j) - 1;  // j = 2^lj
      for (uint32_t p = threadIdx.x; p < (P >> 1); p += THREADS) {
        const uint32_t i = ((p >> lj) << (lj + 1)) | (p & (j - 1));  // bit j of i is clear
        const uint32_t l = i + j;
        const unsigned long long a = s[i], b = s[l];
        const bool up = (i & k) == 0;
        if ((a > b) == up) {
          s[i] = b;
          s[l] = a;
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += THREADS) vals[start + i] = (uint32_t)s[i];
}

__global__ void __launch_bounds__(256) k_sort_tiles_small(int64_t n_tiles, const uint2* __restrict__ ranges,
                                                         const uint2* __restrict__ pairs,
                                                         uint32_t* __restrict__ vals) {
  __shared__ unsigned long long s[kTileSortSmall];
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint2 r = ranges[t];
    const uint32_t n = r.y - r.x;
    if (n == 1) {
      if (threadIdx.x == 0) vals[r.x] = pairs[r.x].y;
      continue;
    }
    if (n < 2 || n > (uint32_t)kTileSortSmall) continue;  // uniform over the CTA
    sort_segment<256>(s, n, r.x, pairs, vals);
    __syncthreads();
  }
}

// One CTA per long list; with n_big_dev (the count on the device, the grid an
// upper bound) the CTAs beyond the count return at once.
__global__ void __launch_bounds__(1024) k_sort_tiles_big(const uint32_t* __restrict__ big_list,
                                                        const uint2* __restrict__ ranges,
                                                        const uint2* __restrict__ pairs,
                                                        uint32_t* __restrict__ vals,
                                                        const uint32_t* __restrict__ n_big_dev) {
  extern __shared__ unsigned long long s_big[];
  if (n_big_dev && blockIdx.x >= *n_big_dev) return;
  const uint2 r = ranges[big_list[blockIdx.x]];
  sort_segment<1024>(s_big, r.y - r.x, r.x, pairs, vals);
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_tile_offsets(cudaStream_t st, const uint32_t* counts, int64_t n_tiles, uint64_t* chunk_sums,
                                uint2* ranges, uint32_t* cursor, uint32_t* big_list, uint32_t* info) {
  const int64_t chunks = (int64_t)tile_offsets_chunks(n_tiles);
  if (chunks == 0) return cudaSuccess;
  k_tile_chunk_sums<<<(unsigned)chunks, OF_THREADS, 0, st>>>(counts, n_tiles, chunk_sums);
  cudaError_t e = launch_scan_spans(st, chunk_sums, chunks, chunk_sums + chunks);
  if (e != cudaSuccess) return e;
  k_tile_offsets<<<(unsigned)chunks, OF_THREADS, 0, st>>>(counts, n_tiles, chunk_sums, ranges, cursor, big_list,
                                                          info);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_scatter(cudaStream_t st, int64_t total, int64_t n, const ProjRec* proj, const CamDev* cams,
                           const uint32_t* depth_keys, uint32_t* cursor, uint2* pairs) {
  if (total == 0) return cudaSuccess;
  k_scatter<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(total, n, proj, cams, depth_keys, cursor, pairs);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sort_tiles(cudaStream_t st, int64_t n_tiles, const uint2* ranges, const uint32_t* big_list,
                              int64_t n_big, const uint2* pairs, uint32_t* vals, const uint32_t* n_big_dev) {
  if (n_tiles == 0) return cudaSuccess;
  const int grid = (int)(n_tiles < 65535 * 8 ? n_tiles : 65535 * 8);
  k_sort_tiles_small<<<grid, 256, 0, st>>>(n_tiles, ranges, pairs, vals);
  count_launches(1);
  if (n_big > 0) {
    const size_t smem = (size_t)kTileSortBig * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(k_sort_tiles_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sort_tiles_big<<<(unsigned)n_big, 1024, smem, st>>>(big_list, ranges, pairs, vals, n_big_dev);
    count_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace airgs
