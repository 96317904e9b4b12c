// Adjoint of the projection + SH colour (sm_103a).
//
// One thread per Gaussian reads its parameters once (the SH coefficients
// through a shared-memory tile, see k_project_bwd), loops over the views,
// reads the per-(view, Gaussian) gradient record the blend backward
// accumulated (dL/d mean2d, conic (A, B, C), opacity, colour) and chains it to
// the raw parameters, summing over views:
//   mean2d = (fx x/z + cx, fy y/z + cy),  t = R_cam mu + t_cam
//   K = Sigma'^-1:  dL/dSigma' = -K G_K K  (G_K the symmetric gradient of K)
//   Sigma' = M M^T + dilation I,  M = J R_cam Rq S
//   J = [[fx/z, 0, -fx ux/z], [0, fy/z, -fy uy/z]],  ux = clamp(x/z) (frustum guard)
//   Rq = R(q/|q|),  S = diag(exp(log_s)),  opacity = sigmoid(logit)
//   colour = max(0, sum_k sh_k Y_k(dir) + 0.5),  dir = (mu - campos)/|mu - campos|
// Every gradient buffer is written once (overwrite), coalesced.
#include "airgs_internal.cuh"
#include "kernels.h"
#include "launch.cuh"
#include "sh_tile.cuh"

namespace airgs {

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

// SH basis (same convention as the forward) and its gradient with respect to
// the direction as a point of R^3 (projected onto the sphere by the caller).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float* Y, float* Gx, float* Gy, float* Gz) {
  Y[0] = k00;
  Gx[0] = Gy[0] = Gz[0] = 0.f;
  if (DEG >= 1) {
    Y[1] = -k1 * y; Gx[1] = 0.f;  Gy[1] = -k1; Gz[1] = 0.f;
    Y[2] = k1 * z;  Gx[2] = 0.f;  Gy[2] = 0.f; Gz[2] = k1;
    Y[3] = -k1 * x; Gx[3] = -k1;  Gy[3] = 0.f; Gz[3] = 0.f;
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = k2a * x * y;  Gx[4] = k2a * y;  Gy[4] = k2a * x;  Gz[4] = 0.f;
    Y[5] = -k2a * y * z; Gx[5] = 0.f;      Gy[5] = -k2a * z; Gz[5] = -k2a * y;
    Y[6] = k2b * (2.f * zz - xx - yy);
    Gx[6] = -2.f * k2b * x; Gy[6] = -2.f * k2b * y; Gz[6] = 4.f * k2b * z;
    Y[7] = -k2a * x * z; Gx[7] = -k2a * z; Gy[7] = 0.f;      Gz[7] = -k2a * x;
    Y[8] = k2c * (xx - yy); Gx[8] = 2.f * k2c * x; Gy[8] = -2.f * k2c * y; Gz[8] = 0.f;
    if (DEG >= 3) {
      const float c9 = -k3a, c11 = -k3c, c13 = -k3c, c15 = -k3a;
      Y[9] = c9 * y * (3.f * xx - yy);
      Gx[9] = 6.f * c9 * x * y; Gy[9] = c9 * (3.f * xx - 3.f * yy); Gz[9] = 0.f;
      Y[10] = k3b * x * y * z;
      Gx[10] = k3b * y * z; Gy[10] = k3b * x * z; Gz[10] = k3b * x * y;
      Y[11] = c11 * y * (4.f * zz - xx - yy);
      Gx[11] = -2.f * c11 * x * y; Gy[11] = c11 * (4.f * zz - xx - 3.f * yy); Gz[11] = 8.f * c11 * y * z;
      Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Gx[12] = -6.f * k3d * x * z; Gy[12] = -6.f * k3d * y * z; Gz[12] = k3d * (6.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = c13 * x * (4.f * zz - xx - yy);
      Gx[13] = c13 * (4.f * zz - 3.f * xx - yy); Gy[13] = -2.f * c13 * x * y; Gz[13] = 8.f * c13 * x * z;
      Y[14] = k3e * z * (xx - yy);
      Gx[14] = 2.f * k3e * x * z; Gy[14] = -2.f * k3e * y * z; Gz[14] = k3e * (xx - yy);
      Y[15] = c15 * x * (xx - 3.f * yy);
      Gx[15] = c15 * (3.f * xx - 3.f * yy); Gy[15] = -6.f * c15 * x * y; Gz[15] = 0.f;
    }
  }
}

#ifndef AIRGS_PROJ_BWD_MINB
#define AIRGS_PROJ_BWD_MINB 4  // 128 registers, 16 warps per SM (measured best of 1, 3, 4, 5, 6)
#endif
constexpr int PB_THREADS = 128;

// The block's SH coefficients (one contiguous run of 128 x 3K floats) move
// between global and shared memory with coalesced accesses; each thread then
// reads and writes its own Gaussian's row of the tile.
template <int DEG>
__global__ void __launch_bounds__(PB_THREADS, AIRGS_PROJ_BWD_MINB) k_project_bwd(int64_t n, const float* __restrict__ means,
                                                     const float* __restrict__ log_scales,
                                                     const float* __restrict__ quats,
                                                     const float* __restrict__ opacity_logit,
                                                     const float* __restrict__ sh, const CamDev* __restrict__ cams,
                                                     int n_views, const ProjRec* __restrict__ proj,
                                                     const GradRec* __restrict__ grad, float* __restrict__ g_means,
                                                     float* __restrict__ g_log_scales, float* __restrict__ g_quats,
                                                     float* __restrict__ g_opacity, float* __restrict__ g_sh,
                                                     float* __restrict__ dens_grad, uint32_t* __restrict__ dens_views,
                                                     float* __restrict__ imp_w, uint32_t* __restrict__ imp_cnt) {
  wait_prior_grid();
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int S = sh_tile_stride<DEG>();
  __shared__ float s_sh[PB_THREADS * S];
  const int64_t g0 = (int64_t)blockIdx.x * PB_THREADS;
  const int nloc = (int)min((int64_t)PB_THREADS, n - g0);
  sh_tile_load<DEG, PB_THREADS>(s_sh, sh, g0, nloc);
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t i = g0 + t;
  float gsh[K * 3];
#pragma unroll
  for (int k = 0; k < K * 3; ++k) gsh[k] = 0.f;
  if (t < nloc) {
    float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float s[3] = {expf(log_scales[3 * i]), expf(log_scales[3 * i + 1]), expf(log_scales[3 * i + 2])};
    float4 q4 = reinterpret_cast<const float4*>(quats)[i];
    float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
    float qi = rsqrtf(qn2);
    float w = q4.x * qi, x = q4.y * qi, y = q4.z * qi, z = q4.w * qi;
    float Rq[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z),       2.f * (x * z + w * y),
                   2.f * (x * y + w * z),       1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                   2.f * (x * z - w * y),       2.f * (y * z + w * x),       1.f - 2.f * (x * x + y * y)};
    float opacity = 1.f / (1.f + expf(-opacity_logit[i]));
    const float* shi = s_sh + t * S;

    float gmu[3] = {0.f, 0.f, 0.f};
    float gs[3] = {0.f, 0.f, 0.f};  // dL/d s_j (scale, not log)
    float gR[9];
  #pragma unroll
    for (int k = 0; k < 9; ++k) gR[k] = 0.f;
    float gop = 0.f;
    float dgrad = 0.f;   // sum over views of |dL/d mean2d| (densification statistic)
    uint32_t dviews = 0; // views in which the Gaussian is visible
    float wimp = 0.f;    // usage frequency over the views: blend weight and blended pairs
    uint32_t cimp = 0;

    for (int v = 0; v < n_views; ++v) {
      const size_t o = (size_t)v * n + i;
      const ProjRec rec = proj[o];
      const int flags = __float_as_int(rec.c.w);
      if (!(flags & kFlagVisible)) continue;
      const GradRec gr = grad[o];
      static_assert(kGradWeightSlot == 5 && kGradCountSlot == 10, "record slots read below");
      wimp += gr.b.y;
      cimp += __float_as_uint(gr.c.z);
      // the blend backward's sums -> gradients of the 2D mean, the conic and the opacity
      const float op2 = rec.b.y, lo = kLn2 * op2;
      const float gmx = lo * fmaf(2.f * rec.a.z, gr.a.x, rec.a.w * gr.a.y);
      const float gmy = lo * fmaf(rec.a.w, gr.a.x, 2.f * rec.b.x * gr.a.y);
      const float gA = -0.5f * op2 * gr.a.z, gB = -op2 * gr.c.y, gC = -0.5f * op2 * gr.a.w, go = gr.b.x;
      ++dviews;
      dgrad += sqrtf(gmx * gmx + gmy * gmy);
      const float grgb[3] = {gr.b.z, gr.b.w, gr.c.x};
      if (gmx == 0.f && gmy == 0.f && gA == 0.f && gB == 0.f && gC == 0.f && go == 0.f && grgb[0] == 0.f &&
          grgb[1] == 0.f && grgb[2] == 0.f)
        continue;
      const CamDev& cam = cams[v];
      gop += go;

      // ---- colour
      {
        float dx = mu[0] - cam.campos[0], dy = mu[1] - cam.campos[1], dz = mu[2] - cam.campos[2];
        float dinv = rsqrtf(dx * dx + dy * dy + dz * dz);
        float ux = dx * dinv, uy = dy * dinv, uz = dz * dinv;
        float Y[K], Gx[K], Gy[K], Gz[K];
        sh_basis_grad<DEG>(ux, uy, uz, Y, Gx, Gy, Gz);
        float graw[3];
  #pragma unroll
        for (int ch = 0; ch < 3; ++ch) graw[ch] = (flags & (1 << (kFlagClampShift + ch))) ? 0.f : grgb[ch];
        float gdx = 0.f, gdy = 0.f, gdz = 0.f;
  #pragma unroll
        for (int k = 0; k < K; ++k) {
          float acc = 0.f;
  #pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            gsh[3 * k + ch] = fmaf(Y[k], graw[ch], gsh[3 * k + ch]);
            acc = fmaf(shi[3 * k + ch], graw[ch], acc);
          }
          gdx = fmaf(acc, Gx[k], gdx);
          gdy = fmaf(acc, Gy[k], gdy);
          gdz = fmaf(acc, Gz[k], gdz);
        }
        float dd = gdx * ux + gdy * uy + gdz * uz;
        gmu[0] += (gdx - ux * dd) * dinv;
        gmu[1] += (gdy - uy * dd) * dinv;
        gmu[2] += (gdz - uz * dd) * dinv;
      }

      // ---- geometry
      const float tx = fmaf(cam.R[0], mu[0], fmaf(cam.R[1], mu[1], fmaf(cam.R[2], mu[2], cam.t[0])));
      const float ty = fmaf(cam.R[3], mu[0], fmaf(cam.R[4], mu[1], fmaf(cam.R[5], mu[2], cam.t[1])));
      const float tz = fmaf(cam.R[6], mu[0], fmaf(cam.R[7], mu[1], fmaf(cam.R[8], mu[2], cam.t[2])));
      const float iz = 1.f / tz, iz2 = iz * iz;
      const float rx = tx * iz, ry = ty * iz;
      const float ux = fminf(fmaxf(rx, -cam.limx), cam.limx), uy = fminf(fmaxf(ry, -cam.limy), cam.limy);
      const float j00 = cam.fx * iz, j02 = -cam.fx * ux * iz, j11 = cam.fy * iz, j12 = -cam.fy * uy * iz;
      float T0[3], T1[3];
  #pragma unroll
      for (int k = 0; k < 3; ++k) {
        T0[k] = fmaf(j00, cam.R[k], j02 * cam.R[6 + k]);
        T1[k] = fmaf(j11, cam.R[3 + k], j12 * cam.R[6 + k]);
      }
      // W2 = T Rq (2x3), M = W2 S
      float W0[3], W1[3], M0[3], M1[3];
  #pragma unroll
      for (int k = 0; k < 3; ++k) {
        W0[k] = T0[0] * Rq[k] + T0[1] * Rq[3 + k] + T0[2] * Rq[6 + k];
        W1[k] = T1[0] * Rq[k] + T1[1] * Rq[3 + k] + T1[2] * Rq[6 + k];
        M0[k] = W0[k] * s[k];
        M1[k] = W1[k] * s[k];
      }
      // conic K from the stored (a2, b2, c2): A = -2 a2 ln2, B = -b2 ln2, C = -2 c2 ln2
      const float A = -2.f * kLn2 * rec.a.z, B = -kLn2 * rec.a.w, C = -2.f * kLn2 * rec.b.x;
      // G_K = [[gA, gB/2], [gB/2, gC]];  G_S = -K G_K K
      const float hB = 0.5f * gB;
      const float t00 = A * gA + B * hB, t01 = A * hB + B * gC;
      const float t10 = B * gA + C * hB, t11 = B * hB + C * gC;
      const float G00 = -(t00 * A + t01 * B), G01 = -(t00 * B + t01 * C);
      const float G11 = -(t10 * B + t11 * C);
      // dL/dM = 2 G_S M
      float gM0[3], gM1[3];
  #pragma unroll
      for (int k = 0; k < 3; ++k) {
        gM0[k] = 2.f * (G00 * M0[k] + G01 * M1[k]);
        gM1[k] = 2.f * (G01 * M0[k] + G11 * M1[k]);
      }
      // M = W2 S:  dL/ds_k += sum_a gM_ak W2_ak;  dL/dW2 = gM S
      float gW0[3], gW1[3];
  #pragma unroll
      for (int k = 0; k < 3; ++k) {
        gs[k] += gM0[k] * W0[k] + gM1[k] * W1[k];
        gW0[k] = gM0[k] * s[k];
        gW1[k] = gM1[k] * s[k];
      }
      // W2 = T Rq:  dL/dRq = T^T gW2,  dL/dT = gW2 Rq^T
      float gT0[3], gT1[3];
  #pragma unroll
      for (int r = 0; r < 3; ++r) {
  #pragma unroll
        for (int c = 0; c < 3; ++c) gR[3 * r + c] += T0[r] * gW0[c] + T1[r] * gW1[c];
        gT0[r] = gW0[0] * Rq[3 * r] + gW0[1] * Rq[3 * r + 1] + gW0[2] * Rq[3 * r + 2];
        gT1[r] = gW1[0] * Rq[3 * r] + gW1[1] * Rq[3 * r + 1] + gW1[2] * Rq[3 * r + 2];
      }
      // T = J R_cam:  dL/dJ = gT R_cam^T
      const float gJ00 = gT0[0] * cam.R[0] + gT0[1] * cam.R[1] + gT0[2] * cam.R[2];
      const float gJ02 = gT0[0] * cam.R[6] + gT0[1] * cam.R[7] + gT0[2] * cam.R[8];
      const float gJ11 = gT1[0] * cam.R[3] + gT1[1] * cam.R[4] + gT1[2] * cam.R[5];
      const float gJ12 = gT1[0] * cam.R[6] + gT1[1] * cam.R[7] + gT1[2] * cam.R[8];
      float gtx = gmx * cam.fx * iz;
      float gty = gmy * cam.fy * iz;
      float gtz = -(gmx * cam.fx * tx + gmy * cam.fy * ty) * iz2;
      gtz -= (gJ00 * cam.fx + gJ11 * cam.fy) * iz2;
      if (!(flags & kFlagGuardX)) {
        gtx -= gJ02 * cam.fx * iz2;
        gtz += gJ02 * 2.f * cam.fx * tx * iz2 * iz;
      } else {
        gtz += gJ02 * cam.fx * ux * iz2;
      }
      if (!(flags & kFlagGuardY)) {
        gty -= gJ12 * cam.fy * iz2;
        gtz += gJ12 * 2.f * cam.fy * ty * iz2 * iz;
      } else {
        gtz += gJ12 * cam.fy * uy * iz2;
      }
      gmu[0] += cam.R[0] * gtx + cam.R[3] * gty + cam.R[6] * gtz;
      gmu[1] += cam.R[1] * gtx + cam.R[4] * gty + cam.R[7] * gtz;
      gmu[2] += cam.R[2] * gtx + cam.R[5] * gty + cam.R[8] * gtz;
    }

    // Rq(q^) -> q^:  explicit partials of the rotation matrix
    const float G00 = gR[0], G01 = gR[1], G02 = gR[2], G10 = gR[3], G11 = gR[4], G12 = gR[5], G20 = gR[6],
                G21 = gR[7], G22 = gR[8];
    float gw = 2.f * (-z * G01 + y * G02 + z * G10 - x * G12 - y * G20 + x * G21);
    float gx = 2.f * (y * G01 + z * G02 + y * G10 - 2.f * x * G11 - w * G12 + z * G20 + w * G21 - 2.f * x * G22);
    float gy = 2.f * (-2.f * y * G00 + x * G01 + w * G02 + x * G10 + z * G12 - w * G20 + z * G21 - 2.f * y * G22);
    float gz = 2.f * (-2.f * z * G00 - w * G01 + x * G02 + w * G10 - 2.f * z * G11 + y * G12 + x * G20 + y * G21);
    // q^ = q / |q|
    float dot = gw * w + gx * x + gy * y + gz * z;
    float4 gq = make_float4((gw - w * dot) * qi, (gx - x * dot) * qi, (gy - y * dot) * qi, (gz - z * dot) * qi);

    g_means[3 * i] = gmu[0];
    g_means[3 * i + 1] = gmu[1];
    g_means[3 * i + 2] = gmu[2];
  #pragma unroll
    for (int k = 0; k < 3; ++k) g_log_scales[3 * i + k] = gs[k] * s[k];
    reinterpret_cast<float4*>(g_quats)[i] = gq;
    g_opacity[i] = gop * opacity * (1.f - opacity);
    if (dens_grad) {
      dens_grad[i] += dgrad;
      dens_views[i] += dviews;
    }
    if (imp_w) {  // one thread per Gaussian: plain read-modify-write
      imp_w[i] += wimp;
      imp_cnt[i] += cimp;
    }
  }
  __syncthreads();  // every thread has finished reading the coefficients
  if (t < nloc) {
#pragma unroll
    for (int k = 0; k < K * 3; ++k) s_sh[t * S + k] = gsh[k];
  }
  __syncthreads();
  sh_tile_store<DEG, PB_THREADS>(s_sh, g_sh, g0, nloc);
}

cudaError_t launch_project_bwd(cudaStream_t st, int64_t n, int sh_degree, const float* means,
                               const float* log_scales, const float* quats, const float* opacity_logit,
                               const float* sh, const CamDev* cams, int n_views, const ProjRec* proj,
                               const GradRec* grad, float* g_means, float* g_log_scales, float* g_quats,
                               float* g_opacity, float* g_sh, float* dens_grad, uint32_t* dens_views, float* imp_w,
                               uint32_t* imp_cnt) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + PB_THREADS - 1) / PB_THREADS);
  cudaError_t e;
#define AIRGS_PB(D)                                                                                                 \
  e = launch_serialised(k_project_bwd<D>, dim3(blocks), dim3(PB_THREADS), 0, st, n, means, log_scales, quats,       \
                        opacity_logit, sh, cams, n_views, proj, grad, g_means, g_log_scales, g_quats, g_opacity, g_sh, \
                        dens_grad, dens_views, imp_w, imp_cnt)
  switch (sh_degree) {
    case 0: AIRGS_PB(0); break;
    case 1: AIRGS_PB(1); break;
    case 2: AIRGS_PB(2); break;
    default: AIRGS_PB(3); break;
  }
#undef AIRGS_PB
  count_launches(1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace airgs
