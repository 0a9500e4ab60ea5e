// Per-tile helpers shared by the split-precision forward and adjoint kernels: the plan fields
// the per-pixel loop reads (held in registers) and the TMA-staged source box of a 32x8 tile.
#pragma once

#include <climits>

#include "dfr_device.cuh"

namespace dfr {

// The plan fields the per-pixel code reads, copied once per tile into registers (the inverse
// SIP coefficient pairs included) so that no plan load sits in the pixel loop.
template <int IDEG, bool PAIRS>
struct HotPlan {
  static constexpr int NC = (IDEG > 0 && PAIRS) ? poly_ncoef(IDEG) : 1;
  float2 cab[NC];
  int32_t W, H, w, h, x0, y0, box_w, box_h;
  bool identity, tsip, newton, use_tma, mask;
  int64_t out_pitch;
  float* out;
  float* fp;
  double* coords;
};

template <int IDEG, bool PAIRS>
__device__ __forceinline__ void load_hot(const FwdPlan& P, HotPlan<IDEG, PAIRS>& Q) {
#pragma unroll
  for (int k = 0; k < HotPlan<IDEG, PAIRS>::NC; ++k)
    Q.cab[k] = (IDEG > 0 && PAIRS) ? make_float2(P.isip_f[0][k], P.isip_f[1][k])
                                   : make_float2(0.f, 0.f);
  Q.W = P.W;
  Q.H = P.H;
  Q.w = P.w;
  Q.h = P.h;
  Q.x0 = P.x0;
  Q.y0 = P.y0;
  Q.box_w = P.box_w;
  Q.box_h = P.box_h;
  Q.identity = P.identity != 0;
  Q.tsip = P.tsip_deg > 0;
  Q.newton = plan_newton(P);
  Q.use_tma = P.use_tma != 0;
  Q.mask = (P.flags & DFR_NAN_MASK) != 0;
  Q.out_pitch = P.out_pitch;
  Q.out = P.out;
  Q.fp = P.fp;
  Q.coords = P.coords;
}

// The plan fields below are read per tile; HP is the form every split kernel uses (the inverse
// SIP is evaluated only at the column-cubic nodes, from the plan itself).
using HP = HotPlan<0, false>;

// FP32 source position of target offset (dx, dy) from the anchor (relative to (bx, by)), the
// split path's exact per-pixel evaluation at the plan's packed inverse-SIP degree. geo: see
// split_coords_core.
// Not inlined (like column_cubic and make_anchor): evaluated a few times per column of a cell,
// it is compiled once per translation unit instead of once per kernel instantiation.
static __device__ __noinline__ bool exact_coords(const FwdPlan& P, const HP& Q, const Anchor& a,
                                          float dx, float dy, float& x, float& y,
                                          float* geo = nullptr) {
  switch (P.isip_deg) {
    case 0:
      return split_coords_core<0, false>(P, nullptr, Q.identity, Q.tsip, Q.newton, a, dx, dy, x,
                                         y, geo);
    case 4:
      return split_coords_core<4, false>(P, nullptr, Q.identity, Q.tsip, Q.newton, a, dx, dy, x,
                                         y, geo);
    case 6:
      return split_coords_core<6, false>(P, nullptr, Q.identity, Q.tsip, Q.newton, a, dx, dy, x,
                                         y, geo);
    default:
      return split_coords_core<9, false>(P, nullptr, Q.identity, Q.tsip, Q.newton, a, dx, dy, x,
                                         y, geo);
  }
}

// ---------------------------------------------------------------- column cubic
// Along one target column of a 32 x 64 cell the split map is a smooth function of the row. Each
// lane evaluates it exactly (exact_coords) at the Chebyshev-Lobatto rows s = -a, -b, b, a of the
// cell (s = row - 31.5, a = 31.5, b = 15.75) and takes the cubic through those four values:
// with E = (f(s) + f(-s)) / 2 and O = (f(s) - f(-s)) / 2,
//   c2 = (E_a - E_b) / (a^2 - b^2),  c0 = E_b - c2 b^2,
//   c3 = (O_a / a - O_b / b) / (a^2 - b^2),  c1 = O_b / b - c3 b^2.
// A fifth exact value at s = 0, where the nodal polynomial (s^2 - a^2)(s^2 - b^2) has its
// largest magnitude on the cell, must equal c0 within kCubicTol; otherwise (and for identity
// maps, where positions must stay exact integers, and cells whose anchor or nodes are
// undefined) the column falls back to the exact evaluation per pixel. Every kernel that needs
// a split-path position (forward rows, coordinate output, adjoint) takes it from here, so all
// agree bit for bit. A valid column has every pixel covered by the projection: the homography
// denominator is linear along the column and positive at both end rows (the outer nodes).
constexpr float kNodeA = 31.5f, kNodeB = 15.75f;
constexpr float kNodeB2 = 248.0625f;  // b^2, exact
constexpr float kInvAB = 1.f / 744.1875f;  // 1 / (a^2 - b^2)
constexpr float kInvA = 1.f / 31.5f, kInvB = 1.f / 15.75f;
constexpr float kCubicTol = 1e-4f;  // px
constexpr float kCellMid = 31.5f;   // s = row - kCellMid; dy = row - kCellH / 2

struct ColCubic {
  float2 c[4];  // (x, y) polynomial coefficients in s, relative to the anchor's (bx, by)
  bool valid;
};

__device__ __forceinline__ float2 v_sub(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

static __device__ __noinline__ ColCubic column_cubic(const FwdPlan& P, const HP& Q, const Anchor& a,
                                              float dx) {
  float2 fam = make_float2(0.f, 0.f), fbm = fam, fbp = fam, fap = fam, f0 = fam;
  bool ok = !Q.identity;
#pragma unroll 1
  for (int k = 0; k < 5; ++k) {
    const float s = k == 0 ? -kNodeA : k == 1 ? -kNodeB : k == 2 ? kNodeB : k == 3 ? kNodeA : 0.f;
    float x = 0.f, y = 0.f;
    ok = exact_coords(P, Q, a, dx, __fsub_rn(s, 0.5f), x, y) && ok;
    const float2 f = make_float2(x, y);
    if (k == 0) fam = f;
    if (k == 1) fbm = f;
    if (k == 2) fbp = f;
    if (k == 3) fap = f;
    if (k == 4) f0 = f;
  }
  const float2 half = make_float2(0.5f, 0.5f);
  const float2 Ea = v_mul(half, v_add(fap, fam)), Eb = v_mul(half, v_add(fbp, fbm));
  const float2 Oa = v_mul(half, v_sub(fap, fam)), Ob = v_mul(half, v_sub(fbp, fbm));
  ColCubic cc;
  cc.c[2] = v_mul(v_sub(Ea, Eb), v_c<float2>(kInvAB));
  cc.c[0] = v_fma(v_c<float2>(-kNodeB2), cc.c[2], Eb);
  const float2 ra = v_mul(Oa, v_c<float2>(kInvA)), rb = v_mul(Ob, v_c<float2>(kInvB));
  cc.c[3] = v_mul(v_sub(ra, rb), v_c<float2>(kInvAB));
  cc.c[1] = v_fma(v_c<float2>(-kNodeB2), cc.c[3], rb);
  // (NaN anywhere fails the comparisons)
  cc.valid = ok && fabsf(cc.c[0].x - f0.x) <= kCubicTol && fabsf(cc.c[0].y - f0.y) <= kCubicTol;
  return cc;
}

// Position of row s of a valid column: c0 + s (c1 + s (c2 + s c3)), both coordinates.
__device__ __forceinline__ float2 cubic_pos(const ColCubic& cc, float s) {
  const float2 ss = make_float2(s, s);
  return v_fma(v_fma(v_fma(cc.c[3], ss, cc.c[2]), ss, cc.c[1]), ss, cc.c[0]);
}

// Source position of row `row` (0..kCellH-1) of the cell column (dx from the anchor): the
// column cubic where valid, else the exact evaluation (whose result says whether the pixel is
// defined). Relative to (a.bx, a.by).
__device__ __forceinline__ bool pixel_coords(const FwdPlan& P, const HP& Q, const Anchor& a,
                                             const ColCubic& cc, float dx, int row, float& x,
                                             float& y) {
  if (cc.valid) {
    const float2 p = cubic_pos(cc, float(row) - kCellMid);
    x = p.x;
    y = p.y;
    return true;
  }
  return exact_coords(P, Q, a, dx, float(row - kCellH / 2), x, y);
}

// Largest deviation of a valid column's positions from the straight line between two rows
// h - 1 apart, for any two such rows of the cell: (h - 1)^2 / 8 max |p''|, |p''| <= 2 |c2| +
// 6 a |c3| (both coordinates).
__device__ __forceinline__ float cubic_bow(const ColCubic& cc, int h) {
  const float hh = float((h - 1) * (h - 1)) * 0.125f;
  const float bx = fmaf(6.f * kNodeA, fabsf(cc.c[3].x), 2.f * fabsf(cc.c[2].x));
  const float by = fmaf(6.f * kNodeA, fabsf(cc.c[3].y), 2.f * fabsf(cc.c[2].y));
  return hh * fmaxf(bx, by);
}

// Source box of the tile of rows [r0, r0 + nrows) of a cell (columns ox .. ox + 31, first row
// oy in the bounding box): the positions of each lane's first and last rows, their floors
// reduced over the warp, widened by the plan's curvature margin (at least 1 px) and the taps,
// and loaded by one TMA copy of kBoxW x box_h floats (when `load`).
struct TileBox {
  int32_t bx0, by0;  // box origin (absolute source pixel)
  int32_t ex0, ey0, ew, eh;  // widened extent of the tile's taps, [ex0, ex0 + ew) etc.
  bool use_box;      // the box was loaded (else gather from global memory)
  bool interior;     // the widened extent lies inside the image: no tap needs masking
  bool empty;        // the widened extent misses the image: nothing in the tile is covered
};

template <int ORDER>
__device__ __forceinline__ TileBox tile_box(const FwdPlan& P, const HP& Q, const Anchor& a,
                                            const ColCubic& cc, int ox, int oy, int r0,
                                            int nrows, int lane, float* box, uint64_t* bar,
                                            bool map_in_gmem, bool load = true,
                                            uint32_t tx_extra = 0) {
  using T = Taps<ORDER>;
  TileBox tb;
  tb.bx0 = tb.by0 = 0;
  tb.ex0 = tb.ey0 = tb.ew = tb.eh = 0;
  tb.use_box = tb.interior = tb.empty = false;
  if (ox >= Q.w || oy >= Q.h) {  // a cell's tile below the bounding box
    tb.empty = true;
    return tb;
  }
  nrows = min(nrows, Q.h - oy);
  const bool active = ox + lane < Q.w;
  const float dx = float(Q.x0 + ox + lane - a.ax);
  float x0 = 0.f, y0 = 0.f, x1 = 0.f, y1 = 0.f;
  bool ok = true;
  if (active) {
    ok = pixel_coords(P, Q, a, cc, dx, r0, x0, y0);
    ok = pixel_coords(P, Q, a, cc, dx, r0 + nrows - 1, x1, y1) && ok;
  }
  // (well inside the |v| < 2^22 range of the fast rows' floor by magic number)
  ok = ok && fabsf(x0) < 2097152.f && fabsf(y0) < 2097152.f && fabsf(x1) < 2097152.f &&
       fabsf(y1) < 2097152.f;
  if (!__all_sync(0xffffffffu, ok)) return tb;  // positions undefined: gather per pixel
  const int lx = int(floorf(fminf(x0, x1))), hx = int(floorf(fmaxf(x0, x1)));
  const int ly = int(floorf(fminf(y0, y1))), hy = int(floorf(fmaxf(y0, y1)));
  const int mnx = __reduce_min_sync(0xffffffffu, active ? lx : INT_MAX);
  const int mxx = __reduce_max_sync(0xffffffffu, active ? hx : INT_MIN);
  const int mny = __reduce_min_sync(0xffffffffu, active ? ly : INT_MAX);
  const int mxy = __reduce_max_sync(0xffffffffu, active ? hy : INT_MIN);
  const int M = max(1, P.box_margin);
  // nearest may step one pixel up from floor(x), so its extent is two taps wide
  constexpr int ext = (ORDER == DFR_NEAREST) ? 2 : T::n;
  const int x_lo = a.bx + mnx - M + T::lo, x_hi = a.bx + mxx + M + T::lo + ext;  // [lo, hi)
  const int y_lo = a.by + mny - M + T::lo, y_hi = a.by + mxy + M + T::lo + ext;
  if (x_hi <= 0 || x_lo >= Q.W || y_hi <= 0 || y_lo >= Q.H) {
    tb.empty = true;
    return tb;
  }
  tb.interior = x_lo >= 0 && x_hi <= Q.W && y_lo >= 0 && y_hi <= Q.H;
  tb.ex0 = x_lo;
  tb.ey0 = y_lo;
  tb.ew = x_hi - x_lo;
  tb.eh = y_hi - y_lo;
  if (!Q.use_tma) return tb;
  tb.bx0 = x_lo & ~3;  // TMA x must be a multiple of 16 bytes
  tb.by0 = y_lo;
  tb.use_box = x_hi - tb.bx0 <= Q.box_w && y_hi - tb.by0 <= Q.box_h;
  if (tb.use_box && load) {  // (load = false: the box geometry only, nothing is copied)
    __syncwarp();  // every lane is done reading this buffer's previous tile
    if (lane == 0) {
      fence_proxy_async();
      if (map_in_gmem) fence_tensormap_acquire(&P.tmap);
      mbar_expect_tx(bar, uint32_t(Q.box_w) * uint32_t(Q.box_h) * 4u + tx_extra);
      tma_load_2d(box, &P.tmap, bar, tb.bx0, tb.by0);
    }
  }
  return tb;
}

}  // namespace dfr
