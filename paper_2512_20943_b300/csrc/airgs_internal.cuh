// Internal device-side definitions shared by the AirGS kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace airgs {

constexpr int kTile = 16;            // 16x16 pixel tiles
constexpr int kTilePixels = kTile * kTile;
constexpr float kLog2e = 1.4426950408889634f;  // 1 / ln 2
constexpr float kLn2 = 0.6931471805599453f;
constexpr int kMaxDevicesAttr = 64;  // devices for which per-device kernel attributes are remembered

// One camera as the kernels see it.
struct CamDev {
  float R[9];       // world -> camera rotation, row-major
  float t[3];       // world -> camera translation
  float campos[3];  // camera centre in world space, -R^T t
  float fx, fy, cx, cy;
  float znear;
  float limx, limy;  // frustum guard 1.3 tan(fov/2) on x/z, y/z
  int W, H, TW, TH;  // image size and tile grid
  int64_t tile_base; // first global tile id of this view
  int64_t pix_base;  // first pixel of this view in concatenated outputs
};

// Rasterizer constants of a launch.
struct RasterParams {
  float dilation, alpha_max, alpha_min, T_min;
  float bg[3];
};

// Per (view, Gaussian) projection record, three 16-byte words:
//   a = {mx, my, a2, b2}
//   b = {c2, opacity, r, g}
//   c = {b, depth, radius (int bits), flags (int bits)}
// with (a2, b2, c2) = log2(e) * (-A/2, -B, -C/2) for the conic (A, B, C) of
// Sigma'^-1, so that  power * log2(e) = a2 dx^2 + b2 dx dy + c2 dy^2.
struct __align__(16) ProjRec {
  float4 a, b, c;
};
constexpr int kFlagVisible = 1;
constexpr int kFlagClampShift = 1;  // bits 1..3: colour channel clamped at 0
constexpr int kFlagGuardX = 16;     // x/z outside the frustum guard
constexpr int kFlagGuardY = 32;

// Per (view, Gaussian) record of the sums the blend backward accumulates over
// the Gaussian's replayed pairs, with d = mean2d - pixel and t = dL/dalpha G on
// unclamped pairs:
//   a = {S_x = sum t dx, S_y = sum t dy, S_xx = sum t dx^2, S_yy = sum t dy^2}
//   b = {S_t = sum t, 0, dL/dr, dL/dg}
//   c = {dL/db, S_xy = sum t dx dy, 0, 0}
// (the order of the backward's accumulator pairs; float 5 is the pair slot of
// the blend weight, which goes to the usage weight instead)
// The projection adjoint turns them into the 2D gradients: with
// power2 = a2 dx^2 + b2 dx dy + c2 dy^2 = log2(e) power and dL/dpower = o t,
// dL/dmean2d = o ln2 (2 a2 S_x + b2 S_y, b2 S_x + 2 c2 S_y),
// dL/dA = -o S_xx / 2, dL/dB = -o S_xy, dL/dC = -o S_yy / 2, dL/dopacity = S_t.
struct __align__(16) GradRec {
  float4 a, b, c;
};
// Slots of a GradRec (as 12 floats) that carry the usage frequency of one
// (view, Gaussian) from the blend backward to the projection adjoint: the sum
// of blend weights, and the blended-pair count as a uint32.
constexpr int kGradWeightSlot = 5;
constexpr int kGradCountSlot = 10;

// ------------------------------------------------------------------ exact-replay arithmetic
// The forward and the backward evaluate every (pixel, Gaussian) pair through
// these helpers, with explicit rounding intrinsics, so that the backward's
// replay takes exactly the forward's skip / blend / stop decisions and
// reproduces its running sums bit for bit.
// 1 / b by the hardware reciprocal, subnormals flushed to zero (the blend
// backward divides the colour still ahead by 1 - alpha, which lies in
// [1 - alpha_max, 1]).
__device__ __forceinline__ float rcp_approx_ftz(float b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
  return r;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Terms that depend only on the pixel row: b2 dy and c2 dy^2.
__device__ __forceinline__ void row_terms(float my, float py, float b2, float c2, float& dy, float& b2dy,
                                          float& c2dy2) {
  dy = __fsub_rn(my, py);
  b2dy = __fmul_rn(b2, dy);
  c2dy2 = __fmul_rn(__fmul_rn(c2, dy), dy);
}

// log2(e) * power for a pixel column offset dx.
__device__ __forceinline__ float power2_of(float dx, float a2, float b2dy, float c2dy2) {
  return __fmaf_rn(__fmaf_rn(a2, dx, b2dy), dx, c2dy2);
}

__device__ __forceinline__ float alpha_of(float o, float G, float alpha_max) { return fminf(alpha_max, __fmul_rn(o, G)); }

// T (1 - alpha) evaluated as T - w with the pair's blend weight w = alpha T (one
// subtraction, the weight being computed for the colour anyway).
__device__ __forceinline__ float blend_weight(float alpha, float T) { return __fmul_rn(alpha, T); }
__device__ __forceinline__ float transmit(float T, float w) { return __fsub_rn(T, w); }

// Tile rectangle of a footprint centred at (mx, my) with integer radius r: the
// tiles whose 16-pixel span meets [m - r, m + r], computed exactly from
// floor(m) (floor((m +- r)/16) = floor((floor(m) +- r)/16) for integer r).
__device__ __forceinline__ void tile_rect(float mx, float my, int r, int TW, int TH, int& x0, int& y0, int& x1,
                                          int& y1) {
  const float lim = 1048576.0f;
  int fx = (int)floorf(fminf(fmaxf(mx, -lim), lim));
  int fy = (int)floorf(fminf(fmaxf(my, -lim), lim));
  int rr = min(r, 1048576);
  // arithmetic shift = floor division by 16 for negative values too
  x0 = min(max((fx - rr) >> 4, 0), TW);
  x1 = min(max(((fx + rr) >> 4) + 1, 0), TW);
  y0 = min(max((fy - rr) >> 4, 0), TH);
  y1 = min(max(((fy + rr) >> 4) + 1, 0), TH);
}

// View that owns a global tile id (binary search over tile_base).
__device__ __forceinline__ int view_of_tile(const int64_t* tile_base, int n_views, int64_t tile) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tile_base[mid] <= tile)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Axis-aligned half-widths of the region where a Gaussian can blend
// (o G >= alpha_min):  Q(d) = -log2(e) power(d) = d^T M d <= L = log2(o/alpha_min),
// half-widths sqrt(L (M^-1)_xx), sqrt(L (M^-1)_yy), widened by a margin far above
// the single-precision error of the per-pair test.  Returns 0 if the Gaussian
// can never blend, 1 with (hx, hy) set, 2 if no bound applies (degenerate or NaN).
__device__ __forceinline__ int alpha_box(float4 ga, float4 gb, float log2_amin, float& hx, float& hy) {
  const float ap = -ga.z, bp = -ga.w, cp = -gb.x;  // Q = ap dx^2 + bp dx dy + cp dy^2
  const float L = lg2_approx(gb.y) - log2_amin + 1e-3f;
  if (L <= 0.f) return 0;
  if (!(L > 0.f)) return 2;
  const float det = ap * cp - 0.25f * bp * bp;
  if (!(det > 0.f)) return 2;
  hx = sqrtf(L * cp / det) * 1.0001f + 0.01f;
  hy = sqrtf(L * ap / det) * 1.0001f + 0.01f;
  return 1;
}

// Instance keys carry the global tile id in the low bits and, in bits 30-31,
// whether the Gaussian can blend in the tile's top / bottom 16x8 half; the
// tile sort orders by the low bits only.
constexpr uint32_t kKeyTileMask = 0x3FFFFFFFu;
constexpr int kKeyHalfShift = 30;

// Largest value over the rectangle [xlo, xhi] x [ylo, yhi] of offsets d = p - m
// of the concave quadratic P(d) = a2 dx^2 + b2 dx dy + c2 dy^2 (negative
// definite), with kx = -b2 / (2 a2), ky = -b2 / (2 c2) the maximisers along a
// row and a column; S receives the sum of the terms' magnitudes there (the
// scale of its rounding error).  When the centre is outside, the maximum lies
// on a face whose outer side holds the centre (the gradient there must point
// out of the rectangle), so only the nearer vertical and horizontal faces are
// searched, each at its clamped 1-D maximiser.  Both faces are evaluated and
// the results selected, so that lanes testing different rectangles do not
// diverge.
__device__ __forceinline__ float rect_max_power2(float a2, float b2, float c2, float kx, float ky, float xlo,
                                                 float xhi, float ylo, float yhi, float& S) {
  const bool in_x = xlo <= 0.f && xhi >= 0.f, in_y = ylo <= 0.f && yhi >= 0.f;
  const float DX = xlo > 0.f ? xlo : xhi;
  const float dy = fminf(fmaxf(ky * DX, ylo), yhi);
  const float pv = fmaf(a2 * DX, DX, fmaf(b2 * DX, dy, c2 * dy * dy));
  const float sv = fabsf(a2) * DX * DX + fabsf(b2 * DX * dy) + fabsf(c2) * dy * dy;
  const float DY = ylo > 0.f ? ylo : yhi;
  const float dx = fminf(fmaxf(kx * DY, xlo), xhi);
  const float ph = fmaf(a2 * dx, dx, fmaf(b2 * dx, DY, c2 * DY * DY));
  const float sh = fabsf(a2) * dx * dx + fabsf(b2 * dx * DY) + fabsf(c2) * DY * DY;
  S = fmaxf(in_x ? 0.f : sv, in_y ? 0.f : sh);
  const float best = fmaxf(in_x ? -INFINITY : pv, in_y ? -INFINITY : ph);
  if (in_x && in_y) S = 0.f;
  return in_x && in_y ? 0.f : best;
}

// Blocks of the tile at (X0, Y0) that the Gaussian's alpha >= alpha_min box
// meets (bit k: block bx = k & 1, by = k >> 1).
__device__ __forceinline__ unsigned block_mask(float4 ga, float4 gb, float log2_amin, float X0, float Y0) {
  const float mx = ga.x, my = ga.y;
  float hx = 0.f, hy = 0.f;
  const int kind = alpha_box(ga, gb, log2_amin, hx, hy);
  if (kind == 0) return 0u;     // o below alpha_min: never blends
  if (kind == 2) return 0xFFu;  // no bound: leave it to the per-pair test
  unsigned xm = 0, m = 0;
#pragma unroll
  for (int bx = 0; bx < 2; ++bx) {
    const float lo = X0 + 8.f * bx + 0.5f, hi = lo + 7.f;
    if (mx + hx >= lo && mx - hx <= hi) xm |= 1u << bx;
  }
#pragma unroll
  for (int by = 0; by < 4; ++by) {
    const float lo = Y0 + 4.f * by + 0.5f, hi = lo + 3.f;
    if (my + hy >= lo && my - hy <= hi) m |= xm << (2 * by);
  }
  return m;
}


// block_mask refined by the exact test of each block's pixel-centre rectangle
// against the ellipse alpha >= alpha_min, i.e. P >= -L with
// L = log2(o / alpha_min): a block is dropped only when the largest P over its
// rectangle lies below -L by a margin far above the single-precision error of
// both this test and the per-pair test.  Pairs in dropped blocks have
// alpha < alpha_min, so results are bit-identical to the unrefined mask.
__device__ __forceinline__ unsigned block_mask_exact(float4 ga, float4 gb, float log2_amin, float X0, float Y0,
                                                     unsigned keep_bits) {
  unsigned m = block_mask(ga, gb, log2_amin, X0, Y0) & keep_bits;
  const float a2 = ga.z, b2 = ga.w, c2 = gb.x;
  if (m == 0u || !(a2 < 0.f && c2 < 0.f && 4.f * a2 * c2 > 1.0001f * b2 * b2)) return m;
  const float L = lg2_approx(gb.y) - log2_amin + 1e-3f;
  const float kx = __fdividef(-b2, 2.f * a2), ky = __fdividef(-b2, 2.f * c2);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (!((m >> k) & 1u)) continue;
    const float xlo = (X0 + 8.f * (k & 1) + 0.5f) - ga.x, xhi = xlo + 7.f;
    const float ylo = (Y0 + 4.f * (k >> 1) + 0.5f) - ga.y, yhi = ylo + 3.f;
    float S;
    const float pm = rect_max_power2(a2, b2, c2, kx, ky, xlo, xhi, ylo, yhi, S);
    if (pm < -L - (0.01f + 1e-5f * S)) m &= ~(1u << k);
  }
  return m;
}

// ------------------------------------------------------------------ culled lists (inference)
// Row-band extents of the region where a Gaussian can blend.  With
// P(d) = a2 dx^2 + b2 dx dy + c2 dy^2 (negative definite, d = pixel - centre) a
// pixel can blend only if P >= -L, L = log2(o / alpha_min).  For fixed dy that
// is an x-interval centred at kx dy (kx = -b2 / (2 a2)) of half-width
// w(dy) = sqrt((L + c' dy^2) / (-a2)), c' = det / a2 (det = a2 c2 - b2^2 / 4),
// nonempty for |dy| <= hy.  Over a band of rows the region's x-extent runs from
// the smallest left end to the largest right end: the right end is concave in
// dy, largest (hx) at the rightmost point dy = -b2 hx / (2 c2) and otherwise at
// the band end nearer to it; the left end mirrors it.  The region is convex, so
// a tile half of the band meets it exactly when its pixel-centre x-range meets
// that extent.  L is widened by 0.01 + 1e-5 S (S bounds the terms' magnitudes
// over the region, the scale of the per-pair test's rounding error) and the
// extent by a small absolute amount, so no dropped tile holds a pair the
// per-pair test would blend.  Every operation has an explicit rounding mode:
// the projection (which counts the live tiles) and the emission (which lists
// them) compute bit-identical extents.
struct EllipseBands {
  float mx, my, kx, cpr, inv_na2, L, hx, hy, dyr, eps;
  int kind;  // 0: never blends, 1: bounded, 2: no bound (every tile of the rectangle is kept)
};

__device__ __forceinline__ EllipseBands ellipse_bands(float mx, float my, float a2, float b2, float c2, float o,
                                                      float log2_amin) {
  EllipseBands e;
  e.mx = mx;
  e.my = my;
  const float L0 = __fadd_rn(__fadd_rn(lg2_approx(o), -log2_amin), 1e-3f);
  const bool definite = a2 < 0.f && c2 < 0.f && __fmul_rn(4.f, __fmul_rn(a2, c2)) > __fmul_rn(1.0001f, __fmul_rn(b2, b2));
  e.kind = L0 <= 0.f ? 0 : ((L0 > 0.f && definite) ? 1 : 2);
  if (e.kind != 1) return e;
  const float det = __fmaf_rn(a2, c2, __fmul_rn(-0.25f, __fmul_rn(b2, b2)));
  const float hx0 = __fsqrt_rn(__fdiv_rn(__fmul_rn(L0, -c2), det));
  const float hy0 = __fsqrt_rn(__fdiv_rn(__fmul_rn(L0, -a2), det));
  const float S = __fadd_rn(__fadd_rn(__fmul_rn(-a2, __fmul_rn(hx0, hx0)), __fmul_rn(fabsf(b2), __fmul_rn(hx0, hy0))),
                            __fmul_rn(-c2, __fmul_rn(hy0, hy0)));
  e.L = __fadd_rn(__fadd_rn(L0, 0.01f), __fmul_rn(1e-5f, S));
  e.hx = __fsqrt_rn(__fdiv_rn(__fmul_rn(e.L, -c2), det));
  e.hy = __fsqrt_rn(__fdiv_rn(__fmul_rn(e.L, -a2), det));
  e.kx = __fdiv_rn(__fmul_rn(-0.5f, b2), a2);
  e.cpr = __fdiv_rn(det, a2);
  e.inv_na2 = __fdiv_rn(-1.f, a2);
  e.dyr = __fdiv_rn(__fmul_rn(__fmul_rn(-0.5f, b2), e.hx), c2);
  e.eps = __fadd_rn(0.01f, __fmul_rn(1e-5f, __fadd_rn(__fadd_rn(e.hx, __fmul_rn(fabsf(e.kx), e.hy)), fabsf(mx))));
  return e;
}

// x-extent [xmin, xmax] (pixel coordinates) of the region over the rows whose
// centres lie in [y0, y1] (pixel coordinates); false when the band misses it.
__device__ __forceinline__ bool band_extent(const EllipseBands& e, float y0, float y1, float& xmin, float& xmax) {
  const float lo = fmaxf(__fadd_rn(y0, -e.my), -e.hy), hi = fminf(__fadd_rn(y1, -e.my), e.hy);
  if (lo > hi) return false;
  const float tr = e.dyr < lo ? lo : (e.dyr > hi ? hi : e.dyr);
  const float tl = -e.dyr < lo ? lo : (-e.dyr > hi ? hi : -e.dyr);
  const float wr = __fsqrt_rn(fmaxf(0.f, __fmul_rn(__fmaf_rn(__fmul_rn(e.cpr, tr), tr, e.L), e.inv_na2)));
  const float wl = __fsqrt_rn(fmaxf(0.f, __fmul_rn(__fmaf_rn(__fmul_rn(e.cpr, tl), tl, e.L), e.inv_na2)));
  const float rmax = tr == e.dyr ? e.hx : __fmaf_rn(e.kx, tr, wr);
  const float lmin = tl == -e.dyr ? -e.hx : __fmaf_rn(e.kx, tl, -wl);
  xmax = __fadd_rn(__fadd_rn(e.mx, rmax), e.eps);
  xmin = __fadd_rn(__fadd_rn(e.mx, lmin), -e.eps);
  return true;
}

// Live tiles of tile row ty within the rectangle's columns [x0, x1): the tiles
// [lo, hi) that either half-row band of the row meets, and the two bands'
// extents for the half flags (ok_* false: the band misses the region).
struct LiveRow {
  int lo, hi;
  bool ok_top, ok_bot;
  float tmin, tmax, bmin, bmax;
};

__device__ __forceinline__ LiveRow live_row(const EllipseBands& e, int ty, int x0, int x1) {
  LiveRow r;
  r.lo = x0;
  r.hi = x1;
  r.ok_top = r.ok_bot = true;
  r.tmin = r.bmin = -INFINITY;
  r.tmax = r.bmax = INFINITY;
  if (e.kind == 2) return r;
  r.lo = r.hi = x0;
  r.ok_top = r.ok_bot = false;
  if (e.kind == 0) return r;
  const float Y0 = (float)(ty * kTile);
  r.ok_top = band_extent(e, Y0 + 0.5f, Y0 + 7.5f, r.tmin, r.tmax);
  r.ok_bot = band_extent(e, Y0 + 8.5f, Y0 + 15.5f, r.bmin, r.bmax);
  if (!r.ok_top && !r.ok_bot) return r;
  const float xmin = fminf(r.ok_top ? r.tmin : INFINITY, r.ok_bot ? r.bmin : INFINITY);
  const float xmax = fmaxf(r.ok_top ? r.tmax : -INFINITY, r.ok_bot ? r.bmax : -INFINITY);
  // tile tx meets [xmin, xmax] iff 16 tx + 0.5 <= xmax and 16 tx + 15.5 >= xmin
  const float lim = 1048576.0f;
  const int first = (int)ceilf(__fdiv_rn(fminf(fmaxf(__fadd_rn(xmin, -15.5f), -lim), lim), 16.f));
  const int last = (int)floorf(__fdiv_rn(fminf(fmaxf(__fadd_rn(xmax, -0.5f), -lim), lim), 16.f));
  r.lo = max(x0, first);
  r.hi = max(r.lo, min(x1, last + 1));
  return r;
}

// The rectangle [x0, x1) x [y0, y1) of tile_rect clipped to the tiles whose
// pixel centres meet the bounding box of the region where the Gaussian can
// blend: P(d) = a2 dx^2 + b2 dx dy + c2 dy^2 >= -L, L = log2(o / alpha_min),
// has half-widths hx = sqrt(L (-c2) / det), hy = sqrt(L (-a2) / det),
// det = a2 c2 - b2^2 / 4.  L is widened by 0.01 + 1e-5 S (S bounds the terms'
// magnitudes over the region, the scale of the per-pair test's rounding
// error) and the box by 0.01 + 1e-5 (h + |m|), as for the row bands above, so
// no dropped tile holds a pair the per-pair test would blend.  Every operation
// has an explicit rounding mode: the projection (which counts the tiles) and
// the emission (which lists them) compute the same rectangle.  A Gaussian that
// can never blend gets an empty rectangle; one with no bound (degenerate or NaN
// terms) keeps the full one.
__device__ __forceinline__ void clip_rect_to_alpha_box(float mx, float my, float a2, float b2, float c2, float o,
                                                       float log2_amin, int& x0, int& y0, int& x1, int& y1) {
  const float L0 = __fadd_rn(__fadd_rn(lg2_approx(o), -log2_amin), 1e-3f);
  if (L0 <= 0.f) {  // o below alpha_min everywhere: never blends
    x1 = x0;
    y1 = y0;
    return;
  }
  const bool definite = a2 < 0.f && c2 < 0.f && __fmul_rn(4.f, __fmul_rn(a2, c2)) > __fmul_rn(1.0001f, __fmul_rn(b2, b2));
  if (!(L0 > 0.f) || !definite) return;
  const float det = __fmaf_rn(a2, c2, __fmul_rn(-0.25f, __fmul_rn(b2, b2)));
  const float hx0 = __fsqrt_rn(__fdiv_rn(__fmul_rn(L0, -c2), det));
  const float hy0 = __fsqrt_rn(__fdiv_rn(__fmul_rn(L0, -a2), det));
  const float S = __fadd_rn(__fadd_rn(__fmul_rn(-a2, __fmul_rn(hx0, hx0)), __fmul_rn(fabsf(b2), __fmul_rn(hx0, hy0))),
                            __fmul_rn(-c2, __fmul_rn(hy0, hy0)));
  const float L = __fadd_rn(__fadd_rn(L0, 0.01f), __fmul_rn(1e-5f, S));
  const float hx = __fsqrt_rn(__fdiv_rn(__fmul_rn(L, -c2), det));
  const float hy = __fsqrt_rn(__fdiv_rn(__fmul_rn(L, -a2), det));
  const float ex = __fadd_rn(hx, __fadd_rn(0.01f, __fmul_rn(1e-5f, __fadd_rn(hx, fabsf(mx)))));
  const float ey = __fadd_rn(hy, __fadd_rn(0.01f, __fmul_rn(1e-5f, __fadd_rn(hy, fabsf(my)))));
  // tile t meets [m - e, m + e] iff 16 t + 0.5 <= m + e and 16 t + 15.5 >= m - e
  const float lim = 1048576.0f;
  const int bx0 = (int)ceilf(__fmul_rn(fminf(fmaxf(__fadd_rn(__fadd_rn(mx, -ex), -15.5f), -lim), lim), 0.0625f));
  const int bx1 = (int)floorf(__fmul_rn(fminf(fmaxf(__fadd_rn(__fadd_rn(mx, ex), -0.5f), -lim), lim), 0.0625f)) + 1;
  const int by0 = (int)ceilf(__fmul_rn(fminf(fmaxf(__fadd_rn(__fadd_rn(my, -ey), -15.5f), -lim), lim), 0.0625f));
  const int by1 = (int)floorf(__fmul_rn(fminf(fmaxf(__fadd_rn(__fadd_rn(my, ey), -0.5f), -lim), lim), 0.0625f)) + 1;
  x0 = max(x0, bx0);
  y0 = max(y0, by0);
  x1 = max(x0, min(x1, bx1));
  y1 = max(y0, min(y1, by1));
}

// Half flags (bit 0 top, bit 1 bottom) of live tile tx of a row.
__device__ __forceinline__ uint32_t live_row_halves(const LiveRow& r, int tx) {
  const float X0 = (float)(tx * kTile);
  uint32_t f = 0u;
  if (r.ok_top && r.tmax >= X0 + 0.5f && r.tmin <= X0 + 15.5f) f |= 1u;
  if (r.ok_bot && r.bmax >= X0 + 0.5f && r.bmin <= X0 + 15.5f) f |= 2u;
  return f;
}

// Half-tile list entries: (Gaussian id, position in the tile's full list in
// bits 0-27 | the half's 8x4 blocks the Gaussian can reach alpha_min in, bits
// 28-31, as block_mask_exact gives them).
constexpr uint32_t kHlPosMask = 0x0FFFFFFFu;
constexpr int kHlMaskShift = 28;

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

}  // namespace airgs
