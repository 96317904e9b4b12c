// Shared-memory staging of a block's SH coefficients (sm_103a).
//
// The coefficients of consecutive Gaussians are one contiguous run of
// 3 (DEG + 1)^2 floats each; a thread per Gaussian reading its own run from
// global memory makes every warp load touch 32 lines.  Instead a block copies
// its run into shared memory with coalesced accesses, one row per Gaussian, and
// each thread reads (or writes) its own row there.
#pragma once

namespace airgs {

// Row stride (floats) of the tile: the 3 (DEG + 1)^2 coefficients padded to an
// odd count, so that the 32 lanes of a warp, each at its own row, hit 32
// different banks.
template <int DEG>
__host__ __device__ constexpr int sh_tile_stride() {
  return (3 * (DEG + 1) * (DEG + 1)) % 2 ? 3 * (DEG + 1) * (DEG + 1) : 3 * (DEG + 1) * (DEG + 1) + 1;
}

// Copy the coefficients of Gaussians [g0, g0 + nloc) into the tile (all threads of the block take part).
template <int DEG, int THREADS>
__device__ __forceinline__ void sh_tile_load(float* tile, const float* __restrict__ sh, int64_t g0, int nloc) {
  constexpr int W = 3 * (DEG + 1) * (DEG + 1), S = sh_tile_stride<DEG>();
  const float* src = sh + g0 * W;
  for (int e = threadIdx.x; e < nloc * W; e += THREADS) tile[(e / W) * S + e % W] = __ldg(src + e);
}

// Write the tile's rows of Gaussians [g0, g0 + nloc) back to global memory.
template <int DEG, int THREADS>
__device__ __forceinline__ void sh_tile_store(const float* tile, float* __restrict__ dst_all, int64_t g0, int nloc) {
  constexpr int W = 3 * (DEG + 1) * (DEG + 1), S = sh_tile_stride<DEG>();
  float* dst = dst_all + g0 * W;
  for (int e = threadIdx.x; e < nloc * W; e += THREADS) dst[e] = tile[(e / W) * S + e % W];
}

}  // namespace airgs
