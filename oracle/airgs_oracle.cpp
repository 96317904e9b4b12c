// AirGS splatting oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, double-precision CPU restatement of the data-parallel path of
// AirGS (arXiv 2512.20943): per-frame decode/apply of streamed Gaussian updates
// (Sec. II, Eq. 3; Sec. III-B, Eq. 5; Sec. III-C, d_t and D_t), EWA projection
// of each 3D Gaussian G = {mu, alpha, c, SH, R, S} with Sigma = R S S^T R^T
// (Sec. II), spherical-harmonic colour (Sec. II), 16x16 tile binning, a stable
// (tile, depth) ordering, front-to-back alpha blending, the per-Gaussian blend
// weight used by usage-frequency pruning (Sec. III-C), the L1 part of Eq. 1,
// and the analytic adjoint of all of it ("differentiable splatting renderer",
// Sec. II).  The paper inherits the rasterizer from 3DGS without restating
// it; the per-pixel rules followed here (alpha = o * exp(-1/2 d^T Sigma'^-1 d),
// clamp 0.99, skip below 1/255, stop when T would fall below 1e-4) are the
// standard 3DGS definitions.
//
// Only the tests, the smoke check and the CPU-baseline leg of the benchmark
// may load this library.  It shares no code, header, table or constant with the
// CUDA path.  Nothing here is blocked, fused or reordered beyond what the
// definitions state: every Gaussian is projected on its own, every tile list is
// built by testing every Gaussian's tile rectangle and ordered with
// std::stable_sort, every pixel walks its tile's list in order.
//
// Where the paper is silent the following readings are used (all listed in the
// design notes): pixel (u, v) is sampled at (u + 0.5, v + 0.5); depth is the
// camera-space z; the near plane culls z <= near; J uses x/z and y/z clamped to
// +-1.3 tan(fov/2); Sigma' gets +dilation on its diagonal; the radius is
// ceil(3 sqrt(lambda_max)) with lambda_max = mid + sqrt(max(0.1, mid^2 - det));
// the tile rectangle holds every tile whose pixel span meets
// [mx - r, mx + r] x [my - r, my + r]; equal depths keep index order; the
// termination test T (1 - alpha) < T_min is taken before Gaussian i is blended
// and i is then not blended; colour is clamped at 0 after adding 0.5 and the
// clamp masks the gradient; a clamped alpha (o G > 0.99) passes no gradient to
// o or G.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;
const int kTile = 16;

// ---------------------------------------------------------------- camera
// Flat layout of one camera (23 doubles):
//   [0] width  [1] height  [2] fx  [3] fy  [4] cx  [5] cy  [6] near
//   [7..22] world->camera 4x4 matrix, row-major; the camera looks down +z,
//   x to the right, y down.
struct Camera {
  int W, H;
  double fx, fy, cx, cy, znear;
  double R[3][3];
  double t[3];
};

Camera read_camera(const double* c) {
  Camera cam;
  cam.W = (int)c[0];
  cam.H = (int)c[1];
  cam.fx = c[2];
  cam.fy = c[3];
  cam.cx = c[4];
  cam.cy = c[5];
  cam.znear = c[6];
  const double* m = c + 7;
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) cam.R[r][k] = m[4 * r + k];
    cam.t[r] = m[4 * r + 3];
  }
  return cam;
}

// Flat layout of the rasterizer settings (11 doubles):
//   [0] dilation added to the 2D covariance diagonal
//   [1] alpha_max (0.99)   [2] alpha_min (1/255)   [3] T_min (1e-4)
//   [4..6] background colour
//   [7] ambiguity tolerance in pixels for tile-rectangle edges
//   [8] relative ambiguity tolerance for alpha / radius / depth-tie tests
//   [9] relative ambiguity tolerance for the termination test
//   [10] relative gap below which two blended depths count as a possible tie
//        (single-precision camera-space z carries about 1.5e-7 relative error)
struct Settings {
  double dilation, alpha_max, alpha_min, T_min, bg[3];
  double tol_px, tol_rel, tol_stop, tol_depth;
};

Settings read_settings(const double* s) {
  Settings o;
  o.dilation = s[0];
  o.alpha_max = s[1];
  o.alpha_min = s[2];
  o.T_min = s[3];
  o.bg[0] = s[4];
  o.bg[1] = s[5];
  o.bg[2] = s[6];
  o.tol_px = s[7];
  o.tol_rel = s[8];
  o.tol_stop = s[9];
  o.tol_depth = s[10];
  return o;
}

// ---------------------------------------------------------------- small linear algebra
typedef double Mat3[3][3];

void mat3_mul(const Mat3 a, const Mat3 b, Mat3 out) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += a[i][k] * b[k][j];
      out[i][j] = s;
    }
}

void mat3_transpose(const Mat3 a, Mat3 out) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) out[i][j] = a[j][i];
}

// Rotation matrix of a unit quaternion (w, x, y, z).
void quat_to_rot(const double q[4], Mat3 R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z);
  R[0][1] = 2 * (x * y - w * z);
  R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);
  R[1][1] = 1 - 2 * (x * x + z * z);
  R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);
  R[2][1] = 2 * (y * z + w * x);
  R[2][2] = 1 - 2 * (x * x + y * y);
}

// Partial derivatives of quat_to_rot with respect to w, x, y, z.
void quat_to_rot_partials(const double q[4], Mat3 dR[4]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  // d/dw
  double dw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
  // d/dx
  double dx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
  // d/dy
  double dy[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
  // d/dz
  double dz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
  std::memcpy(dR[0], dw, sizeof(dw));
  std::memcpy(dR[1], dx, sizeof(dx));
  std::memcpy(dR[2], dy, sizeof(dy));
  std::memcpy(dR[3], dz, sizeof(dz));
}

// ---------------------------------------------------------------- spherical harmonics
// Real spherical harmonics, written out from the Cartesian closed form of the
// real (Condon-Shortley-free) basis:
//   Y_lm = sqrt((2l+1)/(2 pi)) Pi_l^|m|(z) A_m(x, y)      m > 0
//   Y_lm = sqrt((2l+1)/(2 pi)) Pi_l^|m|(z) B_|m|(x, y)    m < 0
//   Y_l0 = sqrt((2l+1)/(4 pi)) Pi_l^0(z)
//   A_m + i B_m = (x + i y)^m
//   Pi_l^m(z) = sqrt((l-m)!/(l+m)!) sum_k (-1)^k 2^-l C(l,k) C(2l-2k,l)
//               (l-2k)!/(l-2k-m)! r^(2k) z^(l-2k-m)
// multiplied by (-1)^m, which is the sign convention of the 3DGS colour model
// (the Condon-Shortley phase kept).  Index k = l^2 + l + m.  The functions are
// evaluated as homogeneous polynomials of (x, y, z) with dual numbers, which
// yields the value and the gradient together; callers project the gradient onto
// the sphere.
struct Dual {
  double v, d[3];
};

Dual dconst(double c) { return Dual{c, {0, 0, 0}}; }
Dual operator+(const Dual& a, const Dual& b) {
  return Dual{a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}};
}
Dual operator-(const Dual& a, const Dual& b) {
  return Dual{a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}};
}
Dual operator*(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v * b.v;
  for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
Dual operator*(double s, const Dual& a) { return Dual{s * a.v, {s * a.d[0], s * a.d[1], s * a.d[2]}}; }

Dual dpow(const Dual& a, int n) {
  Dual r = dconst(1.0);
  for (int i = 0; i < n; ++i) r = r * a;
  return r;
}

double factorial(int n) {
  double f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

double binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  return factorial(n) / (factorial(k) * factorial(n - k));
}

void sh_basis_dual(int degree, const double dir[3], Dual* Y) {
  Dual x{dir[0], {1, 0, 0}}, y{dir[1], {0, 1, 0}}, z{dir[2], {0, 0, 1}};
  Dual r2 = x * x + y * y + z * z;
  for (int l = 0; l <= degree; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      // Pi_l^|m|(z)
      Dual Pi = dconst(0);
      for (int k = 0; k <= (l - am) / 2; ++k) {
        double coef = ((k % 2) ? -1.0 : 1.0) * std::pow(2.0, -l) * binom(l, k) * binom(2 * l - 2 * k, l) *
                      factorial(l - 2 * k) / factorial(l - 2 * k - am);
        Pi = Pi + coef * (dpow(r2, k) * dpow(z, l - 2 * k - am));
      }
      Pi = std::sqrt(factorial(l - am) / factorial(l + am)) * Pi;
      Dual val;
      if (m == 0) {
        val = std::sqrt((2 * l + 1) / (4 * kPi)) * Pi;
      } else {
        // A_m + i B_m = (x + i y)^|m| by the binomial expansion.
        Dual A = dconst(0), B = dconst(0);
        for (int p = 0; p <= am; ++p) {
          Dual term = binom(am, p) * (dpow(x, p) * dpow(y, am - p));
          double ang = (am - p) * kPi / 2;
          A = A + std::cos(ang) * term;
          B = B + std::sin(ang) * term;
        }
        val = std::sqrt((2 * l + 1) / (2 * kPi)) * (Pi * (m > 0 ? A : B));
      }
      double sign = (am % 2) ? -1.0 : 1.0;
      Y[l * l + l + m] = sign * val;
    }
  }
}

// ---------------------------------------------------------------- projection
struct Gaussian {
  double mu[3], log_s[3], q[4], logit;
  const double* sh;  // [K][3]
};

Gaussian read_gaussian(int64_t i, int K, const double* means, const double* log_scales, const double* quats,
                       const double* opacity_logit, const double* sh) {
  Gaussian g;
  for (int k = 0; k < 3; ++k) {
    g.mu[k] = means[3 * i + k];
    g.log_s[k] = log_scales[3 * i + k];
  }
  for (int k = 0; k < 4; ++k) g.q[k] = quats[4 * i + k];
  g.logit = opacity_logit[i];
  g.sh = sh + (size_t)i * K * 3;
  return g;
}

// Everything the forward computes for one (view, Gaussian), kept for the
// adjoint.
struct Proj {
  bool in_front;   // z > near
  bool visible;    // binned into at least one tile
  bool ambig;      // a culling, radius or rectangle decision lies within the tolerance
  double tcam[3];  // camera-space mean
  double qn[4], qnorm;
  Mat3 Rq;         // rotation of the normalised quaternion
  double scale[3];
  Mat3 Sigma;      // 3D covariance
  double ux, uy;   // x/z and y/z after the frustum guard
  bool guard_x, guard_y;  // true when the guard clamped
  double J[2][3];
  double T[2][3];  // J R_cam
  double cov[3];   // Sigma' entries a, b, c (dilation included)
  double det;
  double conic[3];  // A, B, C of Sigma'^-1
  double mean2d[2];
  int radius;
  int rect[4];  // tile x0, y0, x1, y1 (half-open)
  double depth;
  double opacity;
  double dir[3], dist;  // view direction (unit) and distance camera->mean
  double rgb[3];
  bool clamp[3];
  bool clamp_ambig;
};

int64_t floor_div16(int64_t a) { return (int64_t)std::floor((double)a / 16.0); }

// Tile rectangle of a footprint centred at (mx, my) with integer radius r: every
// tile whose pixel span [16k, 16k + 16) meets [m - r, m + r].  For an integer r
// floor((m +- r)/16) equals floor((floor(m) +- r)/16), which is what is
// evaluated.  Centres and radii are limited to +-2^20 pixels first.
void tile_rect(double mx, double my, int64_t r, int W, int H, int rect[4]) {
  const double lim = 1048576.0;
  int TW = (W + kTile - 1) / kTile, TH = (H + kTile - 1) / kTile;
  double cx = std::min(std::max(mx, -lim), lim), cy = std::min(std::max(my, -lim), lim);
  int64_t rr = std::min<int64_t>(r, (int64_t)lim);
  int64_t fx = (int64_t)std::floor(cx), fy = (int64_t)std::floor(cy);
  int64_t x0 = floor_div16(fx - rr), x1 = floor_div16(fx + rr) + 1;
  int64_t y0 = floor_div16(fy - rr), y1 = floor_div16(fy + rr) + 1;
  rect[0] = (int)std::min<int64_t>(std::max<int64_t>(x0, 0), TW);
  rect[1] = (int)std::min<int64_t>(std::max<int64_t>(y0, 0), TH);
  rect[2] = (int)std::min<int64_t>(std::max<int64_t>(x1, 0), TW);
  rect[3] = (int)std::min<int64_t>(std::max<int64_t>(y1, 0), TH);
}

bool rect_empty(const int r[4]) { return r[0] >= r[2] || r[1] >= r[3]; }

int64_t radius_of(double lam) {
  double v = std::ceil(3.0 * std::sqrt(lam));
  if (v > 1048576.0) v = 1048576.0;
  return (int64_t)v;
}

Proj project_one(const Gaussian& g, int K, int degree, const Camera& cam, const Settings& st) {
  Proj p;
  std::memset(&p, 0, sizeof(p));
  // camera-space mean t = R mu + t_w
  for (int r = 0; r < 3; ++r)
    p.tcam[r] = cam.R[r][0] * g.mu[0] + cam.R[r][1] * g.mu[1] + cam.R[r][2] * g.mu[2] + cam.t[r];
  p.depth = p.tcam[2];
  p.in_front = p.tcam[2] > cam.znear;
  if (std::fabs(p.tcam[2] - cam.znear) <= st.tol_rel * std::max(1.0, std::fabs(cam.znear))) p.ambig = true;

  // 3D covariance Sigma = R S S^T R^T with S = diag(exp(log_s)), R from q/|q|
  p.qnorm = std::sqrt(g.q[0] * g.q[0] + g.q[1] * g.q[1] + g.q[2] * g.q[2] + g.q[3] * g.q[3]);
  for (int k = 0; k < 4; ++k) p.qn[k] = g.q[k] / p.qnorm;
  quat_to_rot(p.qn, p.Rq);
  for (int k = 0; k < 3; ++k) p.scale[k] = std::exp(g.log_s[k]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += p.Rq[i][k] * p.scale[k] * p.scale[k] * p.Rq[j][k];
      p.Sigma[i][j] = s;
    }

  p.opacity = 1.0 / (1.0 + std::exp(-g.logit));

  // colour from SH in the direction camera -> mean
  double campos[3];
  for (int k = 0; k < 3; ++k) campos[k] = -(cam.R[0][k] * cam.t[0] + cam.R[1][k] * cam.t[1] + cam.R[2][k] * cam.t[2]);
  double v[3] = {g.mu[0] - campos[0], g.mu[1] - campos[1], g.mu[2] - campos[2]};
  p.dist = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int k = 0; k < 3; ++k) p.dir[k] = v[k] / p.dist;
  std::vector<Dual> Y(K);
  sh_basis_dual(degree, p.dir, Y.data());
  for (int ch = 0; ch < 3; ++ch) {
    double c = 0.5;
    for (int k = 0; k < K; ++k) c += g.sh[3 * k + ch] * Y[k].v;
    p.clamp[ch] = c < 0;
    if (std::fabs(c) <= st.tol_rel) p.clamp_ambig = true;
    p.rgb[ch] = p.clamp[ch] ? 0.0 : c;
  }

  if (!p.in_front) return p;

  // EWA: Sigma' = J R_cam Sigma R_cam^T J^T + dilation I
  double tz = p.tcam[2];
  double limx = 1.3 * (cam.W / (2.0 * cam.fx)), limy = 1.3 * (cam.H / (2.0 * cam.fy));
  double rx = p.tcam[0] / tz, ry = p.tcam[1] / tz;
  p.guard_x = rx < -limx || rx > limx;
  p.guard_y = ry < -limy || ry > limy;
  p.ux = std::min(std::max(rx, -limx), limx);
  p.uy = std::min(std::max(ry, -limy), limy);
  p.J[0][0] = cam.fx / tz;
  p.J[0][1] = 0;
  p.J[0][2] = -cam.fx * p.ux / tz;
  p.J[1][0] = 0;
  p.J[1][1] = cam.fy / tz;
  p.J[1][2] = -cam.fy * p.uy / tz;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += p.J[i][k] * cam.R[k][j];
      p.T[i][j] = s;
    }
  double cov2[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += p.T[i][k] * p.Sigma[k][l] * p.T[j][l];
      cov2[i][j] = s;
    }
  p.cov[0] = cov2[0][0] + st.dilation;
  p.cov[1] = cov2[0][1];
  p.cov[2] = cov2[1][1] + st.dilation;
  p.det = p.cov[0] * p.cov[2] - p.cov[1] * p.cov[1];
  if (std::fabs(p.det) <= st.tol_rel * p.cov[0] * p.cov[2]) p.ambig = true;
  if (!(p.det > 0)) return p;
  p.conic[0] = p.cov[2] / p.det;
  p.conic[1] = -p.cov[1] / p.det;
  p.conic[2] = p.cov[0] / p.det;

  double mid = 0.5 * (p.cov[0] + p.cov[2]);
  double lam = mid + std::sqrt(std::max(0.1, mid * mid - p.det));
  p.radius = (int)radius_of(lam);
  double r3 = 3.0 * std::sqrt(lam);
  if (std::fabs(r3 - std::round(r3)) <= st.tol_rel * r3) p.ambig = true;

  p.mean2d[0] = cam.fx * p.tcam[0] / tz + cam.cx;
  p.mean2d[1] = cam.fy * p.tcam[1] / tz + cam.cy;
  tile_rect(p.mean2d[0], p.mean2d[1], p.radius, cam.W, cam.H, p.rect);
  // rectangle decisions that a tiny change of the centre would flip
  for (int sx = -1; sx <= 1; sx += 2)
    for (int sy = -1; sy <= 1; sy += 2) {
      int alt[4];
      tile_rect(p.mean2d[0] + sx * st.tol_px, p.mean2d[1] + sy * st.tol_px, p.radius, cam.W, cam.H, alt);
      if (std::memcmp(alt, p.rect, sizeof(alt)) != 0) p.ambig = true;
    }
  p.visible = !rect_empty(p.rect);
  return p;
}

// ---------------------------------------------------------------- binning + ordering
// Per-tile lists: the Gaussians whose rectangle holds the tile, in increasing
// depth, equal depths in increasing index.
struct TileLists {
  int TW, TH;
  std::vector<int64_t> start, end;  // per tile, into ids
  std::vector<int32_t> ids;
};

TileLists bin_and_order(int64_t N, const std::vector<const int*>& rects, const std::vector<double>& depth,
                        const std::vector<char>& visible, int W, int H) {
  TileLists tl;
  tl.TW = (W + kTile - 1) / kTile;
  tl.TH = (H + kTile - 1) / kTile;
  int ntiles = tl.TW * tl.TH;
  std::vector<std::vector<int32_t>> per_tile(ntiles);
  for (int64_t i = 0; i < N; ++i) {
    if (!visible[i]) continue;
    const int* r = rects[i];
    for (int ty = r[1]; ty < r[3]; ++ty)
      for (int tx = r[0]; tx < r[2]; ++tx) per_tile[ty * tl.TW + tx].push_back((int32_t)i);
  }
  tl.start.resize(ntiles);
  tl.end.resize(ntiles);
  for (int t = 0; t < ntiles; ++t) {
    std::vector<int32_t>& L = per_tile[t];  // already in index order
    std::stable_sort(L.begin(), L.end(), [&](int32_t a, int32_t b) { return depth[a] < depth[b]; });
    tl.start[t] = (int64_t)tl.ids.size();
    tl.ids.insert(tl.ids.end(), L.begin(), L.end());
    tl.end[t] = (int64_t)tl.ids.size();
  }
  return tl;
}

// ---------------------------------------------------------------- blending
struct BlendView {
  int W, H;
  const double* mean2d;   // [N][2]
  const double* conic;    // [N][3]
  const double* opacity;  // [N]
  const double* rgb;      // [N][3]
  const double* depth;    // [N]
};

struct PixelResult {
  double C[3];
  double T;
  int n_contrib;
  int64_t n_eval;
  bool ambig;
};

// Front-to-back blending of one pixel.  'on_blend' is called for every blended
// pair with (list position, Gaussian id, alpha, T before blending, G).
template <class F>
PixelResult blend_pixel(const BlendView& bv, const TileLists& tl, int u, int v, const Settings& st, F on_blend) {
  PixelResult pr;
  pr.C[0] = pr.C[1] = pr.C[2] = 0;
  pr.T = 1.0;
  pr.n_contrib = 0;
  pr.n_eval = 0;
  pr.ambig = false;
  int tile = (v / kTile) * tl.TW + (u / kTile);
  double px = u + 0.5, py = v + 0.5;
  double prev_depth = 0;  // the previous list entry: its depth and whether it blended here
  bool have_prev = false, prev_sig = false;
  bool last_tied = false;  // the latest blended entry is a near tie of a neighbour that does not blend
  for (int64_t k = tl.start[tile]; k < tl.end[tile]; ++k) {
    int32_t i = tl.ids[k];
    int pos = (int)(k - tl.start[tile]);
    pr.n_eval += 1;
    double dx = bv.mean2d[2 * i] - px, dy = bv.mean2d[2 * i + 1] - py;
    double A = bv.conic[3 * i], B = bv.conic[3 * i + 1], Cc = bv.conic[3 * i + 2];
    double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
    if (std::fabs(power) <= st.tol_rel) pr.ambig = true;
    bool sig = false, stop = false;  // sig: the entry blends or stops the pixel
    double G = 0, alpha = 0, test = 0;
    if (!(power > 0)) {
      G = std::exp(power);
      alpha = std::min(st.alpha_max, bv.opacity[i] * G);
      if (std::fabs(alpha - st.alpha_min) <= st.tol_rel * st.alpha_min) pr.ambig = true;
      // the alpha_max clamp decides whether o and G receive gradient
      if (std::fabs(bv.opacity[i] * G - st.alpha_max) <= st.tol_rel * st.alpha_max) pr.ambig = true;
      if (!(alpha < st.alpha_min)) {
        test = pr.T * (1 - alpha);
        if (std::fabs(test - st.T_min) <= st.tol_stop * st.T_min) pr.ambig = true;
        sig = true;
        stop = test < st.T_min;
      }
    }
    // Two neighbouring list entries closer in depth than a single-precision key
    // resolves may come in the other order there.  When both blend or stop this
    // pixel, the blend depends on that rounding; when only one blends, its list
    // position does, which matters if it is the pixel's last blended entry
    // (n_contrib).
    const double d = bv.depth[i];
    const bool tie = have_prev && std::fabs(d - prev_depth) <= st.tol_depth * std::fabs(d);
    if (tie && sig && prev_sig) pr.ambig = true;
    if (tie && !sig && prev_sig) last_tied = true;
    const bool tie_nonsig_prev = tie && sig && !prev_sig;
    have_prev = true;
    prev_depth = d;
    prev_sig = sig;
    if (!sig) continue;
    if (stop) {
      // the entry after the one that stops the pixel could come first
      if (k + 1 < tl.end[tile]) {
        const double dn = bv.depth[tl.ids[k + 1]];
        if (std::fabs(dn - d) <= st.tol_depth * std::fabs(dn)) pr.ambig = true;
      }
      break;
    }
    last_tied = tie_nonsig_prev;  // this entry is now the latest blended one
    for (int ch = 0; ch < 3; ++ch) pr.C[ch] += bv.rgb[3 * i + ch] * alpha * pr.T;
    on_blend(pos, i, alpha, pr.T, G);
    pr.T = test;
    pr.n_contrib = pos + 1;
  }
  if (last_tied) pr.ambig = true;
  for (int ch = 0; ch < 3; ++ch) pr.C[ch] += pr.T * st.bg[ch];
  return pr;
}

// ---------------------------------------------------------------- one view, forward
struct ViewForward {
  Camera cam;
  std::vector<Proj> proj;
  std::vector<double> mean2d, conic, opacity, rgb, depth;
  std::vector<char> visible;
  TileLists tl;
};

void forward_view(int64_t N, int degree, const double* means, const double* log_scales, const double* quats,
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
  std::vector<const int*> rects(N);
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
  for (int64_t i = 0; i < N; ++i) rects[i] = vf.proj[i].rect;
  vf.tl = bin_and_order(N, rects, vf.depth, vf.visible, vf.cam.W, vf.cam.H);
}

BlendView blend_view_of(const ViewForward& vf) {
  BlendView bv;
  bv.W = vf.cam.W;
  bv.H = vf.cam.H;
  bv.mean2d = vf.mean2d.data();
  bv.conic = vf.conic.data();
  bv.opacity = vf.opacity.data();
  bv.rgb = vf.rgb.data();
  bv.depth = vf.depth.data();
  return bv;
}

// ---------------------------------------------------------------- adjoint of one (view, Gaussian)
// Given dL/d(mean2d), dL/d(conic A, B, C), dL/d(opacity), dL/d(rgb) of one
// projected Gaussian, add dL/d(raw parameters).
void project_backward_one(const Gaussian& g, int K, int degree, const Camera& cam, const Proj& p, const double gm2[2],
                          const double gcon[3], double gop, const double grgb[3], double* g_mu, double* g_logs,
                          double* g_q, double* g_logit, double* g_sh) {
  // opacity = sigmoid(logit)
  *g_logit += gop * p.opacity * (1 - p.opacity);

  // colour: c = sum_k sh_k Y_k(dir) + 0.5, clamped at 0
  std::vector<Dual> Y(K);
  sh_basis_dual(degree, p.dir, Y.data());
  double graw[3];
  for (int ch = 0; ch < 3; ++ch) graw[ch] = p.clamp[ch] ? 0.0 : grgb[ch];
  double gdir[3] = {0, 0, 0};
  for (int k = 0; k < K; ++k)
    for (int ch = 0; ch < 3; ++ch) {
      g_sh[3 * k + ch] += Y[k].v * graw[ch];
      for (int j = 0; j < 3; ++j) gdir[j] += g.sh[3 * k + ch] * Y[k].d[j] * graw[ch];
    }
  // dir = v / |v|, v = mu - campos
  double dd = gdir[0] * p.dir[0] + gdir[1] * p.dir[1] + gdir[2] * p.dir[2];
  for (int j = 0; j < 3; ++j) g_mu[j] += (gdir[j] - p.dir[j] * dd) / p.dist;

  // mean2d = (fx tx/tz + cx, fy ty/tz + cy)
  double tx = p.tcam[0], ty = p.tcam[1], tz = p.tcam[2];
  double gt[3] = {0, 0, 0};
  gt[0] += gm2[0] * cam.fx / tz;
  gt[1] += gm2[1] * cam.fy / tz;
  gt[2] += -gm2[0] * cam.fx * tx / (tz * tz) - gm2[1] * cam.fy * ty / (tz * tz);

  // conic K = Sigma'^-1; with G_K the symmetric matrix gradient,
  // dL/dSigma' = -K G_K K.
  double Km[2][2] = {{p.conic[0], p.conic[1]}, {p.conic[1], p.conic[2]}};
  double GK[2][2] = {{gcon[0], 0.5 * gcon[1]}, {0.5 * gcon[1], gcon[2]}};
  double tmp[2][2], GS2[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) tmp[i][j] = Km[i][0] * GK[0][j] + Km[i][1] * GK[1][j];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) GS2[i][j] = -(tmp[i][0] * Km[0][j] + tmp[i][1] * Km[1][j]);

  // Sigma' = T Sigma T^T (+ dilation), T = J R_cam:
  //   dL/dSigma = T^T G T,   dL/dT = 2 G T Sigma,   dL/dJ = dL/dT R_cam^T
  Mat3 GSig;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) s += p.T[a][i] * GS2[a][b] * p.T[b][j];
      GSig[i][j] = s;
    }
  double GT[2][3];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 3; ++k) s += GS2[a][b] * p.T[b][k] * p.Sigma[k][j];
      GT[a][j] = 2 * s;
    }
  double GJ[2][3];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) {
      double s = 0;
      for (int j = 0; j < 3; ++j) s += GT[a][j] * cam.R[k][j];
      GJ[a][k] = s;
    }
  // J = [[fx/tz, 0, -fx ux/tz], [0, fy/tz, -fy uy/tz]], ux = clamp(tx/tz)
  gt[2] += GJ[0][0] * (-cam.fx / (tz * tz));
  gt[2] += GJ[1][1] * (-cam.fy / (tz * tz));
  if (!p.guard_x) {  // J02 = -fx tx / tz^2
    gt[0] += GJ[0][2] * (-cam.fx / (tz * tz));
    gt[2] += GJ[0][2] * (2 * cam.fx * tx / (tz * tz * tz));
  } else {  // J02 = -fx ux / tz with ux constant
    gt[2] += GJ[0][2] * (cam.fx * p.ux / (tz * tz));
  }
  if (!p.guard_y) {
    gt[1] += GJ[1][2] * (-cam.fy / (tz * tz));
    gt[2] += GJ[1][2] * (2 * cam.fy * ty / (tz * tz * tz));
  } else {
    gt[2] += GJ[1][2] * (cam.fy * p.uy / (tz * tz));
  }
  // t = R_cam mu + t_w
  for (int j = 0; j < 3; ++j) g_mu[j] += cam.R[0][j] * gt[0] + cam.R[1][j] * gt[1] + cam.R[2][j] * gt[2];

  // Sigma = M M^T, M = Rq S:  dL/dM = 2 G_Sigma M
  Mat3 M;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = p.Rq[i][j] * p.scale[j];
  Mat3 GM;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += GSig[i][k] * M[k][j];
      GM[i][j] = 2 * s;
    }
  // M_ij = Rq_ij s_j:  dL/ds_j = sum_i GM_ij Rq_ij, dL/dRq_ij = GM_ij s_j
  for (int j = 0; j < 3; ++j) {
    double s = 0;
    for (int i = 0; i < 3; ++i) s += GM[i][j] * p.Rq[i][j];
    g_logs[j] += s * p.scale[j];  // s_j = exp(log_s_j)
  }
  Mat3 dR[4];
  quat_to_rot_partials(p.qn, dR);
  double gqn[4];
  for (int c = 0; c < 4; ++c) {
    double s = 0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) s += GM[i][j] * p.scale[j] * dR[c][i][j];
    gqn[c] = s;
  }
  // qn = q / |q|
  double dot = gqn[0] * p.qn[0] + gqn[1] * p.qn[1] + gqn[2] * p.qn[2] + gqn[3] * p.qn[3];
  for (int c = 0; c < 4; ++c) g_q[c] += (gqn[c] - p.qn[c] * dot) / p.qnorm;
}

}  // namespace

extern "C" {

// Real SH basis of the given degree at a unit direction; Y has (degree+1)^2
// entries, dY (nullable) the R^3 gradient of each as [K][3].
int orc_sh_eval(int degree, const double* dir, double* Y, double* dY) {
  if (degree < 0 || degree > 8) return -1;
  int K = (degree + 1) * (degree + 1);
  std::vector<Dual> v(K);
  sh_basis_dual(degree, dir, v.data());
  for (int k = 0; k < K; ++k) {
    Y[k] = v[k].v;
    if (dY)
      for (int j = 0; j < 3; ++j) dY[3 * k + j] = v[k].d[j];
  }
  return 0;
}

// Decode one 7-channel 16-bit update map and apply it (Sec. II Eq. 3: one
// Gaussian per pixel, one attribute per channel; Sec. III-B Eq. 5 and Sec.
// III-C: the delta is applied to the previous frame (d_t) or to the anchor
// (D_t)).  Channel c value = lo[c] + u * (hi[c] - lo[c]) / 65535.  Channels:
// dx, dy, dz, qw, qx, qy, qz.  Pixel i in row-major order carries Gaussian i.
// quat_mode 0: q = normalize(dq (x) q_base) (Hamilton product), 1: q = q_base + dq.
int orc_decode_apply(int64_t N, const uint16_t* map, int map_w, int map_h, const double* lo, const double* hi,
                     int quat_mode, const double* base_means, const double* base_quats, double* out_means,
                     double* out_quats) {
  int64_t P = (int64_t)map_w * map_h;
  if (N > P || N < 0) return -1;
  for (int64_t i = 0; i < N; ++i) {
    double val[7];
    for (int c = 0; c < 7; ++c) {
      double scale = (hi[c] - lo[c]) / 65535.0;
      val[c] = lo[c] + (double)map[c * P + i] * scale;
    }
    for (int k = 0; k < 3; ++k) out_means[3 * i + k] = base_means[3 * i + k] + val[k];
    const double* q = base_quats + 4 * i;
    const double* d = val + 3;
    double r[4];
    if (quat_mode == 0) {
      r[0] = d[0] * q[0] - d[1] * q[1] - d[2] * q[2] - d[3] * q[3];
      r[1] = d[0] * q[1] + d[1] * q[0] + d[2] * q[3] - d[3] * q[2];
      r[2] = d[0] * q[2] - d[1] * q[3] + d[2] * q[0] + d[3] * q[1];
      r[3] = d[0] * q[3] + d[1] * q[2] - d[2] * q[1] + d[3] * q[0];
      double n = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
      for (int k = 0; k < 4; ++k) r[k] /= n;
    } else {
      for (int k = 0; k < 4; ++k) r[k] = q[k] + d[k];
    }
    for (int k = 0; k < 4; ++k) out_quats[4 * i + k] = r[k];
  }
  return 0;
}

// Project N Gaussians for one camera.  Outputs per Gaussian: mean2d[2],
// conic[3] (A, B, C), radius, depth, rect[4] (tile x0, y0, x1, y1, half-open),
// rgb[3], clamp mask (bit ch), opacity, visible, ambiguous.
int orc_project(int64_t N, int degree, const double* means, const double* log_scales, const double* quats,
                const double* opacity_logit, const double* sh, const double* camv, const double* settings,
                double* mean2d, double* conic, int32_t* radius, double* depth, int32_t* rect, double* rgb,
                uint8_t* clamp_mask, double* opacity, uint8_t* visible, uint8_t* ambig) {
  if (degree < 0 || degree > 3) return -1;
  int K = (degree + 1) * (degree + 1);
  Camera cam = read_camera(camv);
  Settings st = read_settings(settings);
  for (int64_t i = 0; i < N; ++i) {
    Gaussian g = read_gaussian(i, K, means, log_scales, quats, opacity_logit, sh);
    Proj p = project_one(g, K, degree, cam, st);
    mean2d[2 * i] = p.mean2d[0];
    mean2d[2 * i + 1] = p.mean2d[1];
    for (int k = 0; k < 3; ++k) {
      conic[3 * i + k] = p.conic[k];
      rgb[3 * i + k] = p.rgb[k];
    }
    radius[i] = p.radius;
    depth[i] = p.depth;
    for (int k = 0; k < 4; ++k) rect[4 * i + k] = p.rect[k];
    clamp_mask[i] = (uint8_t)((p.clamp[0] ? 1 : 0) | (p.clamp[1] ? 2 : 0) | (p.clamp[2] ? 4 : 0));
    opacity[i] = p.opacity;
    visible[i] = p.in_front && p.det > 0 && p.visible;
    ambig[i] = p.ambig || p.clamp_ambig;
  }
  return 0;
}

// Bin and order given per-Gaussian centres, radii, depths and visibility
// (these may come from any projection, e.g. single-precision values widened to
// double).  tile_ranges is [ntiles][2] (start, end).  Returns the number of
// list entries; the list is written only if it fits in list_cap.
int64_t orc_bin_sort(int64_t N, const double* mean2d, const int32_t* radius, const double* depth,
                     const uint8_t* visible, int W, int H, int64_t* tile_ranges, int32_t* list, int64_t list_cap) {
  std::vector<int> rect_store(4 * N);
  std::vector<const int*> rects(N);
  std::vector<double> dep(depth, depth + N);
  std::vector<char> vis(N);
  for (int64_t i = 0; i < N; ++i) {
    tile_rect(mean2d[2 * i], mean2d[2 * i + 1], radius[i], W, H, &rect_store[4 * i]);
    rects[i] = &rect_store[4 * i];
    vis[i] = visible[i] && !rect_empty(rects[i]);
  }
  TileLists tl = bin_and_order(N, rects, dep, vis, W, H);
  int ntiles = tl.TW * tl.TH;
  for (int t = 0; t < ntiles; ++t) {
    tile_ranges[2 * t] = tl.start[t];
    tile_ranges[2 * t + 1] = tl.end[t];
  }
  int64_t n = (int64_t)tl.ids.size();
  if (n <= list_cap)
    for (int64_t k = 0; k < n; ++k) list[k] = tl.ids[k];
  return n;
}

// Full forward over n_views cameras.  Outputs are concatenated per view:
// rgb [3][H][W] planar, T [H][W], n_contrib [H][W], pixel ambiguity [H][W].
// imp_w / imp_cnt (nullable, length N) receive the summed blend weight
// alpha_i T_i and the number of blended pairs of each Gaussian over all pixels
// and views; gauss_ambig (nullable) marks Gaussians that were ambiguous in a
// projection or took part in an ambiguous pixel.  pairs (nullable) receives
// the number of evaluated (pixel, list entry) pairs.
// windows (nullable): per view x0, y0, x1, y1; only pixels inside are blended
// (the others keep zero outputs), e.g. to check sampled windows of large views.
int orc_render(int64_t N, int degree, const double* means, const double* log_scales, const double* quats,
               const double* opacity_logit, const double* sh, int n_views, const double* cams,
               const double* settings, double* rgb_out, double* T_out, int32_t* ncontrib_out, double* imp_w,
               int64_t* imp_cnt, uint8_t* pix_ambig, uint8_t* gauss_ambig, int64_t* pairs, const int32_t* windows) {
  if (degree < 0 || degree > 3) return -1;
  Settings st = read_settings(settings);
  if (imp_w)
    for (int64_t i = 0; i < N; ++i) imp_w[i] = 0;
  if (imp_cnt)
    for (int64_t i = 0; i < N; ++i) imp_cnt[i] = 0;
  if (gauss_ambig)
    for (int64_t i = 0; i < N; ++i) gauss_ambig[i] = 0;
  if (pairs) *pairs = 0;
  int64_t pix_off = 0;
  for (int vi = 0; vi < n_views; ++vi) {
    ViewForward vf;
    forward_view(N, degree, means, log_scales, quats, opacity_logit, sh, cams + 23 * vi, st, vf);
    if (gauss_ambig)
      for (int64_t i = 0; i < N; ++i)
        if (vf.proj[i].ambig) gauss_ambig[i] = 1;
    BlendView bv = blend_view_of(vf);
    int W = vf.cam.W, H = vf.cam.H;
    int64_t HW = (int64_t)W * H;
    int wx0 = 0, wy0 = 0, wx1 = W, wy1 = H;
    if (windows) {
      wx0 = windows[4 * vi];
      wy0 = windows[4 * vi + 1];
      wx1 = windows[4 * vi + 2];
      wy1 = windows[4 * vi + 3];
    }
    for (int v = wy0; v < wy1; ++v)
      for (int u = wx0; u < wx1; ++u) {
        PixelResult pr = blend_pixel(bv, vf.tl, u, v, st, [&](int, int32_t i, double alpha, double T, double) {
          if (imp_w) imp_w[i] += alpha * T;
          if (imp_cnt) imp_cnt[i] += 1;
        });
        int64_t pix = (int64_t)v * W + u;
        for (int ch = 0; ch < 3; ++ch) rgb_out[3 * pix_off + ch * HW + pix] = pr.C[ch];
        if (T_out) T_out[pix_off + pix] = pr.T;
        if (ncontrib_out) ncontrib_out[pix_off + pix] = pr.n_contrib;
        if (pairs) *pairs += pr.n_eval;
        bool amb = pr.ambig;
        if (pix_ambig) pix_ambig[pix_off + pix] = amb;
        if (amb && gauss_ambig) {
          int tile = (v / kTile) * vf.tl.TW + (u / kTile);
          for (int64_t k = vf.tl.start[tile]; k < vf.tl.end[tile]; ++k) gauss_ambig[vf.tl.ids[k]] = 1;
        }
      }
    pix_off += HW;
  }
  return 0;
}

// Analytic adjoint of orc_render: given dL/d(rgb) laid out like rgb_out,
// write dL/d(means, log_scales, quats, opacity_logit, sh) (overwritten).
// dens_grad / dens_views (nullable, accumulated) receive, per Gaussian, the sum
// over views of |dL/d mean2d| and the number of views in which it is visible.
int orc_render_backward(int64_t N, int degree, const double* means, const double* log_scales, const double* quats,
                        const double* opacity_logit, const double* sh, int n_views, const double* cams,
                        const double* settings, const double* dL_drgb, double* g_means, double* g_log_scales,
                        double* g_quats, double* g_opacity_logit, double* g_sh, const int32_t* windows,
                        double* dens_grad, int64_t* dens_views) {
  if (degree < 0 || degree > 3) return -1;
  int K = (degree + 1) * (degree + 1);
  Settings st = read_settings(settings);
  std::fill(g_means, g_means + 3 * N, 0.0);
  std::fill(g_log_scales, g_log_scales + 3 * N, 0.0);
  std::fill(g_quats, g_quats + 4 * N, 0.0);
  std::fill(g_opacity_logit, g_opacity_logit + N, 0.0);
  std::fill(g_sh, g_sh + (size_t)N * K * 3, 0.0);
  int64_t pix_off = 0;
  for (int vi = 0; vi < n_views; ++vi) {
    ViewForward vf;
    forward_view(N, degree, means, log_scales, quats, opacity_logit, sh, cams + 23 * vi, st, vf);
    BlendView bv = blend_view_of(vf);
    int W = vf.cam.W, H = vf.cam.H;
    int64_t HW = (int64_t)W * H;
    // per-Gaussian gradients of this view's projected quantities
    std::vector<double> g_m2(2 * N, 0), g_con(3 * N, 0), g_op(N, 0), g_rgb(3 * N, 0);
    int wx0 = 0, wy0 = 0, wx1 = W, wy1 = H;  // pixels outside a window must have zero dL/d(rgb)
    if (windows) {
      wx0 = windows[4 * vi];
      wy0 = windows[4 * vi + 1];
      wx1 = windows[4 * vi + 2];
      wy1 = windows[4 * vi + 3];
    }
    for (int v = wy0; v < wy1; ++v)
      for (int u = wx0; u < wx1; ++u) {
        int64_t pix = (int64_t)v * W + u;
        // the forward result of this pixel
        PixelResult fin = blend_pixel(bv, vf.tl, u, v, st, [](int, int32_t, double, double, double) {});
        double gC[3];
        for (int ch = 0; ch < 3; ++ch) gC[ch] = dL_drgb[3 * pix_off + ch * HW + pix];
        double px = u + 0.5, py = v + 0.5;
        double P[3] = {0, 0, 0};  // colour accumulated through the current Gaussian
        // replay front to back: C = sum_j c_j a_j T_j + T_final bg, so
        //   dC/dc_i = a_i T_i,   dC/da_i = c_i T_i - (C - P_i) / (1 - a_i)
        blend_pixel(bv, vf.tl, u, v, st, [&](int, int32_t i, double alpha, double T, double G) {
          double w = alpha * T;
          double dL_dalpha = 0;
          for (int ch = 0; ch < 3; ++ch) {
            double c = bv.rgb[3 * i + ch];
            P[ch] += c * w;
            g_rgb[3 * i + ch] += w * gC[ch];
            dL_dalpha += gC[ch] * (c * T - (fin.C[ch] - P[ch]) / (1 - alpha));
          }
          double o = bv.opacity[i];
          if (o * G > st.alpha_max) return;  // clamped alpha: constant
          // alpha = o G, G = exp(power)
          g_op[i] += dL_dalpha * G;
          double dL_dpower = dL_dalpha * o * G;
          double dx = bv.mean2d[2 * i] - px, dy = bv.mean2d[2 * i + 1] - py;
          double A = bv.conic[3 * i], B = bv.conic[3 * i + 1], Cc = bv.conic[3 * i + 2];
          // power = -1/2 (A dx^2 + C dy^2) - B dx dy
          g_con[3 * i] += dL_dpower * (-0.5 * dx * dx);
          g_con[3 * i + 1] += dL_dpower * (-dx * dy);
          g_con[3 * i + 2] += dL_dpower * (-0.5 * dy * dy);
          g_m2[2 * i] += dL_dpower * (-(A * dx + B * dy));
          g_m2[2 * i + 1] += dL_dpower * (-(B * dx + Cc * dy));
        });
      }
    for (int64_t i = 0; i < N; ++i) {
      if (!vf.visible[i]) continue;
      // densification statistic: |dL/d mean2d| of this view, and the view count
      if (dens_grad) dens_grad[i] += std::sqrt(g_m2[2 * i] * g_m2[2 * i] + g_m2[2 * i + 1] * g_m2[2 * i + 1]);
      if (dens_views) dens_views[i] += 1;
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
