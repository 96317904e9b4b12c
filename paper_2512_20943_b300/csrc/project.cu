// Decode/apply of streamed updates and the fused multi-view EWA projection +
// SH colour kernel (sm_103a).
//
//   k_decode_apply  one frame's 7-channel 16-bit map -> new means / quats
//                   (Sec. II Eq. 3: one Gaussian per pixel, one attribute per
//                   channel; Sec. III-B Eq. 5 / Sec. III-C: applied to the
//                   previous frame (d_t) or to the anchor (D_t)).
//   k_project       every Gaussian read once, projected for all views:
//                   Sigma = R S S^T R^T (Sec. II), EWA 2D covariance, conic,
//                   radius, tile rectangle, depth key, SH colour.
#include "airgs_internal.cuh"
#include "kernels.h"
#include "launch.cuh"

namespace airgs {

// ------------------------------------------------------------------ decode / apply
struct DecodeParams {
  float lo[7];
  float scale[7];  // (hi - lo) / 65535, rounded once on the host
};

__global__ void __launch_bounds__(256) k_decode_apply(int64_t n, const uint16_t* __restrict__ map, int64_t plane,
                                                      DecodeParams dp, int quat_add,
                                                      const float* __restrict__ base_means,
                                                      const float* __restrict__ base_quats, float* out_means,
                                                      float* out_quats) {
  wait_prior_grid();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) v[c] = fmaf((float)__ldg(map + c * plane + i), dp.scale[c], dp.lo[c]);
  float m0 = base_means[3 * i], m1 = base_means[3 * i + 1], m2 = base_means[3 * i + 2];
  float4 q = reinterpret_cast<const float4*>(base_quats)[i];
  out_means[3 * i] = m0 + v[0];
  out_means[3 * i + 1] = m1 + v[1];
  out_means[3 * i + 2] = m2 + v[2];
  float4 r;
  if (quat_add) {
    r = make_float4(q.x + v[3], q.y + v[4], q.z + v[5], q.w + v[6]);
  } else {
    // Hamilton product dq (x) q with dq = (v3, v4, v5, v6) = (w, x, y, z)
    float dw = v[3], dx = v[4], dy = v[5], dz = v[6];
    r.x = dw * q.x - dx * q.y - dy * q.z - dz * q.w;
    r.y = dw * q.y + dx * q.x + dy * q.w - dz * q.z;
    r.z = dw * q.z - dx * q.w + dy * q.x + dz * q.y;
    r.w = dw * q.w + dx * q.z - dy * q.y + dz * q.x;
    float inv = rsqrtf(r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w);
    r.x *= inv;
    r.y *= inv;
    r.z *= inv;
    r.w *= inv;
  }
  reinterpret_cast<float4*>(out_quats)[i] = r;
}

// ------------------------------------------------------------------ SH basis
// Real spherical harmonics up to degree 3 at a unit direction (x, y, z), in
// the 3DGS sign convention (Condon-Shortley phase kept).  Constants:
//   k00 = 1/(2 sqrt(pi)), k1 = sqrt(3/(4 pi)),
//   k2a = sqrt(15/pi)/2, k2b = sqrt(5/pi)/4, k2c = sqrt(15/pi)/4,
//   k3a = sqrt(35/(2 pi))/4, k3b = sqrt(105/pi)/2, k3c = sqrt(21/(2 pi))/4,
//   k3d = sqrt(7/pi)/4, k3e = sqrt(105/pi)/4.
constexpr float k00 = 0.28209479177387814f;
constexpr float k1 = 0.48860251190291992f;
constexpr float k2a = 1.0925484305920792f;
constexpr float k2b = 0.31539156525252005f;
constexpr float k2c = 0.54627421529603959f;
constexpr float k3a = 0.59004358992664352f;
constexpr float k3b = 2.8906114426405538f;
constexpr float k3c = 0.45704579946446572f;
constexpr float k3d = 0.3731763325901154f;
constexpr float k3e = 1.4453057213202769f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = k00;
  if (DEG >= 1) {
    Y[1] = -k1 * y;
    Y[2] = k1 * z;
    Y[3] = -k1 * x;
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = k2a * x * y;
    Y[5] = -k2a * y * z;
    Y[6] = k2b * (2.f * zz - xx - yy);
    Y[7] = -k2a * x * z;
    Y[8] = k2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -k3a * y * (3.f * xx - yy);
      Y[10] = k3b * x * y * z;
      Y[11] = -k3c * y * (4.f * zz - xx - yy);
      Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -k3c * x * (4.f * zz - xx - yy);
      Y[14] = k3e * z * (xx - yy);
      Y[15] = -k3a * x * (xx - 3.f * yy);
    }
  }
}

// ------------------------------------------------------------------ projection
#ifndef AIRGS_PROJ_MINB
#define AIRGS_PROJ_MINB 1  // unbounded (117 registers); 5 and 6 measured no faster
#endif
template <int DEG>
__global__ void __launch_bounds__(128, AIRGS_PROJ_MINB) k_project(int64_t n, const float* __restrict__ means,
                                                 const float* __restrict__ log_scales,
                                                 const float* __restrict__ quats,
                                                 const float* __restrict__ opacity_logit,
                                                 const float* __restrict__ sh, const CamDev* __restrict__ cams,
                                                 int n_views, RasterParams rp, ProjRec* __restrict__ proj,
                                                 uint32_t* __restrict__ depth_keys,
                                                 uint32_t* __restrict__ tiles_touched,
                                                 uint32_t* __restrict__ tile_counts, int cull, float log2_amin) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;

  float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
  float s[3] = {expf(log_scales[3 * i]), expf(log_scales[3 * i + 1]), expf(log_scales[3 * i + 2])};
  float4 q4 = reinterpret_cast<const float4*>(quats)[i];
  float qi = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
  float w = q4.x * qi, x = q4.y * qi, y = q4.z * qi, z = q4.w * qi;
  float Rq[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z),       2.f * (x * z + w * y),
                 2.f * (x * y + w * z),       1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                 2.f * (x * z - w * y),       2.f * (y * z + w * x),       1.f - 2.f * (x * x + y * y)};
  float opacity = 1.f / (1.f + expf(-opacity_logit[i]));
  float coef[K * 3];
  const float* shi = sh + (size_t)i * K * 3;
  if ((K * 3) % 4 == 0 && (reinterpret_cast<uintptr_t>(sh) & 15u) == 0) {  // 16-byte loads when aligned
#pragma unroll
    for (int q = 0; q < (K * 3) / 4; ++q) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(shi) + q);
      coef[4 * q] = v.x;
      coef[4 * q + 1] = v.y;
      coef[4 * q + 2] = v.z;
      coef[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < K * 3; ++k) coef[k] = __ldg(shi + k);
  }

  for (int v = 0; v < n_views; ++v) {
    const CamDev& cam = cams[v];
    size_t o = (size_t)v * n + i;
    float tx = fmaf(cam.R[0], mu[0], fmaf(cam.R[1], mu[1], fmaf(cam.R[2], mu[2], cam.t[0])));
    float ty = fmaf(cam.R[3], mu[0], fmaf(cam.R[4], mu[1], fmaf(cam.R[5], mu[2], cam.t[1])));
    float tz = fmaf(cam.R[6], mu[0], fmaf(cam.R[7], mu[1], fmaf(cam.R[8], mu[2], cam.t[2])));

    // colour from SH in the direction camera -> mean
    float dx = mu[0] - cam.campos[0], dy = mu[1] - cam.campos[1], dz = mu[2] - cam.campos[2];
    float dinv = rsqrtf(dx * dx + dy * dy + dz * dz);
    float Y[K];
    sh_basis<DEG>(dx * dinv, dy * dinv, dz * dinv, Y);
    float rgb[3];
    int flags = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float c = 0.5f;
#pragma unroll
      for (int k = 0; k < K; ++k) c = fmaf(coef[3 * k + ch], Y[k], c);
      if (c < 0.f) {
        flags |= 1 << (kFlagClampShift + ch);
        c = 0.f;
      }
      rgb[ch] = c;
    }

    ProjRec rec;
    uint32_t dkey = 0xFFFFFFFFu, ntiles = 0;
    int radius = 0;
    float mx = 0.f, my = 0.f, a2 = 0.f, b2 = 0.f, c2 = 0.f;
    if (tz > cam.znear) {
      float iz = 1.f / tz;
      float rx = tx * iz, ry = ty * iz;
      if (rx < -cam.limx || rx > cam.limx) flags |= kFlagGuardX;
      if (ry < -cam.limy || ry > cam.limy) flags |= kFlagGuardY;
      float ux = fminf(fmaxf(rx, -cam.limx), cam.limx), uy = fminf(fmaxf(ry, -cam.limy), cam.limy);
      // J = [[fx/z, 0, -fx ux/z], [0, fy/z, -fy uy/z]];  T = J R_cam
      float j00 = cam.fx * iz, j02 = -cam.fx * ux * iz, j11 = cam.fy * iz, j12 = -cam.fy * uy * iz;
      float T0[3], T1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T0[k] = fmaf(j00, cam.R[k], j02 * cam.R[6 + k]);
        T1[k] = fmaf(j11, cam.R[3 + k], j12 * cam.R[6 + k]);
      }
      // M = T Rq S; Sigma' = M M^T + dilation I
      float M0[3], M1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        M0[k] = (T0[0] * Rq[k] + T0[1] * Rq[3 + k] + T0[2] * Rq[6 + k]) * s[k];
        M1[k] = (T1[0] * Rq[k] + T1[1] * Rq[3 + k] + T1[2] * Rq[6 + k]) * s[k];
      }
      float ca = M0[0] * M0[0] + M0[1] * M0[1] + M0[2] * M0[2] + rp.dilation;
      float cb = M0[0] * M1[0] + M0[1] * M1[1] + M0[2] * M1[2];
      float cc = M1[0] * M1[0] + M1[1] * M1[1] + M1[2] * M1[2] + rp.dilation;
      float det = fmaf(ca, cc, -cb * cb);
      if (det > 0.f) {
        float idet = 1.f / det;
        float A = cc * idet, B = -cb * idet, C = ca * idet;
        float mid = 0.5f * (ca + cc);
        float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
        float r = ceilf(3.f * sqrtf(lam));
        radius = (int)fminf(r, 1048576.f);
        mx = fmaf(cam.fx, tx * iz, cam.cx);
        my = fmaf(cam.fy, ty * iz, cam.cy);
        int x0, y0, x1, y1;
        tile_rect(mx, my, radius, cam.TW, cam.TH, x0, y0, x1, y1);
        if (x0 < x1 && y0 < y1) {
          ntiles = (uint32_t)((x1 - x0) * (y1 - y0));

          if (tile_counts) {  // per-tile list lengths for the per-tile ordering
            uint32_t* tc = tile_counts + cam.tile_base;
            for (int ty = y0; ty < y1; ++ty)
              for (int tx = x0; tx < x1; ++tx) atomicAdd(tc + ty * cam.TW + tx, 1u);
          }
          dkey = __float_as_uint(tz);
          flags |= kFlagVisible;
          a2 = -0.5f * kLog2e * A;
          b2 = -kLog2e * B;
          c2 = -0.5f * kLog2e * C;
          if (cull == kCullBox) {  // the rectangle clipped to the alpha_min box, from the record's values
            clip_rect_to_alpha_box(mx, my, a2, b2, c2, opacity, log2_amin, x0, y0, x1, y1);
            ntiles = (uint32_t)((x1 - x0) * (y1 - y0));
          } else if (cull == kCullBands) {  // only the tiles in which the Gaussian can reach alpha_min, from
                                            // the values the record stores, as the emission will read them
            const EllipseBands e = ellipse_bands(mx, my, a2, b2, c2, opacity, log2_amin);
            uint32_t live = 0;
            for (int ty = y0; ty < y1; ++ty) {
              const LiveRow r = live_row(e, ty, x0, x1);
              live += (uint32_t)(r.hi - r.lo);
            }
            ntiles = live;
          }
        }
      }
    }
    if (!(flags & kFlagVisible)) radius = 0;
    rec.a = make_float4(mx, my, a2, b2);
    rec.b = make_float4(c2, opacity, rgb[0], rgb[1]);
    rec.c = make_float4(rgb[2], tz, __int_as_float(radius), __int_as_float(flags));
    proj[o] = rec;
    depth_keys[o] = dkey;
    tiles_touched[o] = ntiles;
  }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_decode_apply(cudaStream_t st, int64_t n, const uint16_t* map, int64_t plane, const float* lo,
                                const float* hi, int quat_add, const float* base_means, const float* base_quats,
                                float* out_means, float* out_quats) {
  if (n == 0) return cudaSuccess;
  DecodeParams dp;
  for (int c = 0; c < 7; ++c) {
    dp.lo[c] = lo[c];
    dp.scale[c] = (float)(((double)hi[c] - (double)lo[c]) / 65535.0);
  }
  int blocks = (int)((n + 255) / 256);
  cudaError_t e = launch_serialised(k_decode_apply, dim3(blocks), dim3(256), 0, st, n, map, plane, dp, quat_add,
                                    base_means, base_quats, out_means, out_quats);
  count_launches(1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_project(cudaStream_t st, int64_t n, int sh_degree, const float* means, const float* log_scales,
                           const float* quats, const float* opacity_logit, const float* sh, const CamDev* cams,
                           int n_views, const RasterParams& rp, ProjRec* proj, uint32_t* depth_keys,
                           uint32_t* tiles_touched, uint32_t* tile_counts, int cull) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 127) / 128);
  switch (sh_degree) {
    case 0:
      k_project<0><<<blocks, 128, 0, st>>>(n, means, log_scales, quats, opacity_logit, sh, cams, n_views, rp, proj,
                                           depth_keys, tiles_touched, tile_counts, cull, log2f(rp.alpha_min));
      break;
    case 1:
      k_project<1><<<blocks, 128, 0, st>>>(n, means, log_scales, quats, opacity_logit, sh, cams, n_views, rp, proj,
                                           depth_keys, tiles_touched, tile_counts, cull, log2f(rp.alpha_min));
      break;
    case 2:
      k_project<2><<<blocks, 128, 0, st>>>(n, means, log_scales, quats, opacity_logit, sh, cams, n_views, rp, proj,
                                           depth_keys, tiles_touched, tile_counts, cull, log2f(rp.alpha_min));
      break;
    default:
      k_project<3><<<blocks, 128, 0, st>>>(n, means, log_scales, quats, opacity_logit, sh, cams, n_views, rp, proj,
                                           depth_keys, tiles_touched, tile_counts, cull, log2f(rp.alpha_min));
      break;
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace airgs
