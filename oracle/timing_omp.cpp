// Timing build of the FP64 oracle, for the CPU baseline of the benchmark only.
//
// It compiles the oracle's source unchanged (included below) and adds
// OpenMP versions of the render and of its adjoint that spread the same loops
// over the host's cores: the per-Gaussian projection, the per-pixel blending
// (dynamic schedule over rows of 16x16 tiles) and the per-Gaussian adjoint.
// Per-Gaussian sums that several pixels add to (usage frequency, the 2D
// gradients) use atomic additions, so the forward's images, transmittance,
// n_contrib and pair count are bit-identical to the oracle's and the adjoint
// differs from it only in the order of additions.  The parity tests use the
// single-threaded oracle (liboracle.so), never this build.
#include "airgs_oracle.cpp"

#include <omp.h>

namespace {

// forward_view with the projection loop in parallel (binning as the oracle).
void forward_view_omp(int64_t N, int degree, const double* means, const double* log_scales, const double* quats,
                      const double* opacity_logit, const double* sh, const double* camv, const Settings& st,
                      ViewForward& vf) {
  int K = (degree + 1) * (degree + 1);
  vf.cam = read_camera(camv);
  vf.proj.resize(N);
  vf.mean2d.assign(2 * N, 0);
  vf.conic.assign(3 * N, 0);
  vf.opacity.assign(N, 0);
  vf.rgb.assign(3 * N, 0);
  vf.depth.assign(N, 0);
  vf.visible.assign(N, 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    Gaussian g = read_gaussian(i, K, means, log_scales, quats, opacity_logit, sh);
    vf.proj[i] = project_one(g, K, degree, vf.cam, st);
    const Proj& p = vf.proj[i];
    vf.mean2d[2 * i] = p.mean2d[0];
    vf.mean2d[2 * i + 1] = p.mean2d[1];
    for (int k = 0; k < 3; ++k) {
      vf.conic[3 * i + k] = p.conic[k];
      vf.rgb[3 * i + k] = p.rgb[k];
    }
    vf.opacity[i] = p.opacity;
    vf.depth[i] = p.depth;
    vf.visible[i] = p.in_front && p.det > 0 && p.visible;
  }
  std::vector<const int*> rects(N);
  for (int64_t i = 0; i < N; ++i) rects[i] = vf.proj[i].rect;
  vf.tl = bin_and_order(N, rects, vf.depth, vf.visible, vf.cam.W, vf.cam.H);
}

}  // namespace

extern "C" {

int orc_omp_threads(void) { return omp_get_max_threads(); }

// orc_render without the ambiguity flags, the pixel loop over tile rows in parallel.
int orc_omp_render(int64_t N, int degree, const double* means, const double* log_scales, const double* quats,
                   const double* opacity_logit, const double* sh, int n_views, const double* cams,
                   const double* settings, double* rgb_out, double* T_out, int32_t* ncontrib_out, double* imp_w,
                   int64_t* imp_cnt, int64_t* pairs) {
  if (degree < 0 || degree > 3) return -1;
  Settings st = read_settings(settings);
  if (imp_w) std::fill(imp_w, imp_w + N, 0.0);
  if (imp_cnt) std::fill(imp_cnt, imp_cnt + N, (int64_t)0);
  int64_t total_pairs = 0;
  int64_t pix_off = 0;
  for (int vi = 0; vi < n_views; ++vi) {
    ViewForward vf;
    forward_view_omp(N, degree, means, log_scales, quats, opacity_logit, sh, cams + 23 * vi, st, vf);
    BlendView bv = blend_view_of(vf);
    const int W = vf.cam.W, H = vf.cam.H;
    const int64_t HW = (int64_t)W * H;
    const int tile_rows = (H + kTile - 1) / kTile;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total_pairs)
    for (int tr = 0; tr < tile_rows; ++tr)
      for (int v = tr * kTile; v < std::min(H, (tr + 1) * kTile); ++v)
        for (int u = 0; u < W; ++u) {
          PixelResult pr = blend_pixel(bv, vf.tl, u, v, st, [&](int, int32_t i, double alpha, double T, double) {
            if (imp_w) {
#pragma omp atomic
              imp_w[i] += alpha * T;
            }
            if (imp_cnt) {
#pragma omp atomic
              imp_cnt[i] += 1;
            }
          });
          const int64_t pix = (int64_t)v * W + u;
          for (int ch = 0; ch < 3; ++ch) rgb_out[3 * pix_off + ch * HW + pix] = pr.C[ch];
          if (T_out) T_out[pix_off + pix] = pr.T;
          if (ncontrib_out) ncontrib_out[pix_off + pix] = pr.n_contrib;
          total_pairs += pr.n_eval;
        }
    pix_off += HW;
  }
  if (pairs) *pairs = total_pairs;
  return 0;
}

// orc_render_backward (no windows, no densification statistics) with the pixel
// replay over tile rows and the per-Gaussian adjoint in parallel.
int orc_omp_render_backward(int64_t N, int degree, const double* means, const double* log_scales, const double* quats,
                            const double* opacity_logit, const double* sh, int n_views, const double* cams,
                            const double* settings, const double* dL_drgb, double* g_means, double* g_log_scales,
                            double* g_quats, double* g_opacity_logit, double* g_sh) {
  if (degree < 0 || degree > 3) return -1;
  const int K = (degree + 1) * (degree + 1);
  Settings st = read_settings(settings);
  std::fill(g_means, g_means + 3 * N, 0.0);
  std::fill(g_log_scales, g_log_scales + 3 * N, 0.0);
  std::fill(g_quats, g_quats + 4 * N, 0.0);
  std::fill(g_opacity_logit, g_opacity_logit + N, 0.0);
  std::fill(g_sh, g_sh + (size_t)N * K * 3, 0.0);
  int64_t pix_off = 0;
  for (int vi = 0; vi < n_views; ++vi) {
    ViewForward vf;
    forward_view_omp(N, degree, means, log_scales, quats, opacity_logit, sh, cams + 23 * vi, st, vf);
    BlendView bv = blend_view_of(vf);
    const int W = vf.cam.W, H = vf.cam.H;
    const int64_t HW = (int64_t)W * H;
    std::vector<double> g_m2(2 * N, 0), g_con(3 * N, 0), g_op(N, 0), g_rgb(3 * N, 0);
    const int tile_rows = (H + kTile - 1) / kTile;
#pragma omp parallel for schedule(dynamic, 1)
    for (int tr = 0; tr < tile_rows; ++tr)
      for (int v = tr * kTile; v < std::min(H, (tr + 1) * kTile); ++v)
        for (int u = 0; u < W; ++u) {
          const int64_t pix = (int64_t)v * W + u;
          PixelResult fin = blend_pixel(bv, vf.tl, u, v, st, [](int, int32_t, double, double, double) {});
          double gC[3];
          for (int ch = 0; ch < 3; ++ch) gC[ch] = dL_drgb[3 * pix_off + ch * HW + pix];
          const double px = u + 0.5, py = v + 0.5;
          double P[3] = {0, 0, 0};
          blend_pixel(bv, vf.tl, u, v, st, [&](int, int32_t i, double alpha, double T, double G) {
            const double w = alpha * T;
            double dL_dalpha = 0;
            for (int ch = 0; ch < 3; ++ch) {
              const double c = bv.rgb[3 * i + ch];
              P[ch] += c * w;
#pragma omp atomic
              g_rgb[3 * i + ch] += w * gC[ch];
              dL_dalpha += gC[ch] * (c * T - (fin.C[ch] - P[ch]) / (1 - alpha));
            }
            const double o = bv.opacity[i];
            if (o * G > st.alpha_max) return;
#pragma omp atomic
            g_op[i] += dL_dalpha * G;
            const double dL_dpower = dL_dalpha * o * G;
            const double dx = bv.mean2d[2 * i] - px, dy = bv.mean2d[2 * i + 1] - py;
            const double A = bv.conic[3 * i], B = bv.conic[3 * i + 1], Cc = bv.conic[3 * i + 2];
#pragma omp atomic
            g_con[3 * i] += dL_dpower * (-0.5 * dx * dx);
#pragma omp atomic
            g_con[3 * i + 1] += dL_dpower * (-dx * dy);
#pragma omp atomic
            g_con[3 * i + 2] += dL_dpower * (-0.5 * dy * dy);
#pragma omp atomic
            g_m2[2 * i] += dL_dpower * (-(A * dx + B * dy));
#pragma omp atomic
            g_m2[2 * i + 1] += dL_dpower * (-(B * dx + Cc * dy));
          });
        }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      if (!vf.visible[i]) continue;
      Gaussian g = read_gaussian(i, K, means, log_scales, quats, opacity_logit, sh);
      project_backward_one(g, K, degree, vf.cam, vf.proj[i], &g_m2[2 * i], &g_con[3 * i], g_op[i], &g_rgb[3 * i],
                           g_means + 3 * i, g_log_scales + 3 * i, g_quats + 4 * i, g_opacity_logit + i,
                           g_sh + (size_t)i * K * 3);
    }
    pix_off += HW;
  }
  return 0;
}

}  // extern "C"
