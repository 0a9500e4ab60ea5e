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
  bool identity, tsip, newton, use_tma, mask, stage_sw;
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
  Q.stage_sw = P.stage_sw != 0;
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
template <bool INL>
__device__ __forceinline__ bool exact_coords_t(const FwdPlan& P, const HP& Q, const Anchor& a,
                                               float dx, float dy, float& x, float& y,
                                               float* geo) {
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

// The per-pixel fallback (cells without valid cubics, the adjoint's chain rule): not inlined,
// compiled once per translation unit instead of once per kernel instantiation.
static __device__ __noinline__ bool exact_coords(const FwdPlan& P, const HP& Q, const Anchor& a,
                                                 float dx, float dy, float& x, float& y,
                                                 float* geo = nullptr) {
  return exact_coords_t<false>(P, Q, a, dx, dy, x, y, geo);
}

// ---------------------------------------------------------------- cell fit
// Cell coordinates: column c = 0..31 (the lane), row r = 0..63; sx = c - 15.5, s = r - 31.5
// (exact). The cell's anchor sits at (sx, s) = (0.5, 0), i.e. target pixel
// (x0 + cox + 16, y0 + coy + 31.5): the exact per-pixel evaluation of a cell pixel is
// exact_coords(anchor, dx = c - 16, dy = s), relative to the anchor's integer base (bx, by).
//
// Along a column the map is a smooth function of s; across the cell, of sx. The warp samples it
// exactly (make_anchor at the point, then exact_coords at offset 0: the double-float homography
// and the FP32 inverse SIP) at the Chebyshev-Lobatto grid sx_i in {-A, -B, B, A} (A = 15.5,
// B = 7.75) by s_j in {-a, -b, b, a} (a = 31.5, b = 15.75): lane i + 4 j takes node (i, j).
// Each lane interpolates the four node rows at its own column, g_j = sum_i L_i(sx) f(i, j) (L
// the Lagrange weights of the x nodes), and takes the cubic in s through g_0..g_3: with
// E = (g(s) + g(-s)) / 2 and O = (g(s) - g(-s)) / 2,
//   c2 = (E_a - E_b) / (a^2 - b^2),  c0 = E_b - c2 b^2,
//   c3 = (O_a / a - O_b / b) / (a^2 - b^2),  c1 = O_b / b - c3 b^2.
// Lanes 16-19 evaluate four check points exactly, at columns 16, 3, 28, 15 and s = 0, 24.875,
// -24.875, -20, where the two nodal polynomials (s^2 - a^2)(s^2 - b^2) and (sx^2 - A^2)(sx^2 -
// B^2) are at or near their largest; the first is the anchor. The cell's cubics are valid
// when every point is defined and each check agrees with its column's cubic within kCubicTol;
// otherwise (and for identity maps, whose positions must stay exact) every pixel of the cell
// takes the exact evaluation. All split-path kernels take positions from here, so all agree
// bit for bit. In a valid cell every pixel is covered by the projection: the homography
// denominator is linear and positive at the four corner nodes.
constexpr float kNodeXA = 15.5f, kNodeXB = 7.75f;
constexpr float kNodeA = 31.5f, kNodeB = 15.75f;
constexpr float kNodeB2 = 248.0625f;  // b^2, exact
constexpr float kInvAB = 1.f / 744.1875f;  // 1 / (a^2 - b^2)
constexpr float kInvA = 1.f / 31.5f, kInvB = 1.f / 15.75f;
constexpr float kCubicTol = 1e-4f;  // px
constexpr float kCellMid = 31.5f;   // s = row - kCellMid
constexpr int kAnchorCol = 16;      // dx = column - kAnchorCol

struct ColCubic {
  float2 c[4];  // (x, y) polynomial coefficients in s, relative to the anchor's (bx, by)
  bool valid;   // the same for the whole cell
};

__device__ __forceinline__ float2 v_sub(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

// Lagrange weights of the x nodes at sx (exact products of quarter-integers, one rounding).
__device__ __forceinline__ void lagrange_x(float sx, float L[4]) {
  const float t[4] = {-kNodeXA, -kNodeXB, kNodeXB, kNodeXA};
  // 1 / prod_{m != i} (t_i - t_m)
  const float kInvDenX[4] = {-1.f / 5585.8125f, 1.f / 2792.90625f, -1.f / 2792.90625f,
                             1.f / 5585.8125f};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float p = 1.f;
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (m != i) p = __fmul_rn(p, __fsub_rn(sx, t[m]));
    L[i] = __fmul_rn(p, kInvDenX[i]);
  }
}

// The cubic in s through the values g[j] at s = -a, -b, b, a.
__device__ __forceinline__ void fit_s(const float2 g[4], float2 c[4]) {
  const float2 half = make_float2(0.5f, 0.5f);
  const float2 Ea = v_mul(half, v_add(g[3], g[0])), Eb = v_mul(half, v_add(g[2], g[1]));
  const float2 Oa = v_mul(half, v_sub(g[3], g[0])), Ob = v_mul(half, v_sub(g[2], g[1]));
  c[2] = v_mul(v_sub(Ea, Eb), v_c<float2>(kInvAB));
  c[0] = v_fma(v_c<float2>(-kNodeB2), c[2], Eb);
  const float2 ra = v_mul(Oa, v_c<float2>(kInvA)), rb = v_mul(Ob, v_c<float2>(kInvB));
  c[3] = v_mul(v_sub(ra, rb), v_c<float2>(kInvAB));
  c[1] = v_fma(v_c<float2>(-kNodeB2), c[3], rb);
}

// Position of row s of a valid column: c0 + s (c1 + s (c2 + s c3)), both coordinates.
__device__ __forceinline__ float2 cubic_pos(const ColCubic& cc, float s) {
  const float2 ss = make_float2(s, s);
  return v_fma(v_fma(v_fma(cc.c[3], ss, cc.c[2]), ss, cc.c[1]), ss, cc.c[0]);
}

// Cell-fit sample k (0-15 nodes, 16-19 checks) as (sx, s).
__device__ __forceinline__ float2 cell_sample(int k) {
  const float xs[4] = {-kNodeXA, -kNodeXB, kNodeXB, kNodeXA};
  const float ss[4] = {-kNodeA, -kNodeB, kNodeB, kNodeA};
  if (k < 16) return make_float2(xs[k & 3], ss[k >> 2]);
  const float cxs[4] = {0.5f, -12.5f, 12.5f, -0.5f};  // columns 16, 3, 28, 15
  const float css[4] = {0.f, 24.875f, -24.875f, -20.f};
  return make_float2(cxs[k - 16], css[k - 16]);
}

// Exact source position at cell point (sx, s): the anchor there and its own offset-0 position
// (relative to that anchor's base). Inlined (with the plan read as kernel-parameter operands
// where the plan is the parameter): the fit's latency is on every cell's critical path.
// Every variant (target SIP, Newton inverse, identity), not inlined: compiled once per
// translation unit (the adjoint kernels, and the rare plans of the forward ones).
static __device__ __noinline__ bool cell_point_call(const FwdPlan& P, const HP& Q, float X,
                                                    float Y, Anchor& an, float& x, float& y) {
  make_anchor(P, X, Y, an);
  return exact_coords_t<true>(P, Q, an, 0.f, 0.f, x, y, nullptr);
}

// The common plan (no target SIP, polynomial or no inverse SIP) inlined: the double-float
// anchor and the inverse SIP by the unrolled Horner of the plan's packed degree at the anchor
// itself (offset 0), with the bits of the general evaluation there.
__device__ __forceinline__ bool cell_point(const FwdPlan& P, const HP& Q, float X, float Y,
                                           Anchor& an, float& x, float& y) {
  make_anchor(P, X, Y, an);
  if (Q.identity || Q.tsip || Q.newton)
    return exact_coords_t<true>(P, Q, an, 0.f, 0.f, x, y, nullptr);
  // at offset 0 the local homography is the anchor itself: (U, V) = (U0, V0) and the position
  // is f0 + (AP, BP)(U0, V0), the bits split_coords_core gives there
  float ga = 0.f, gb = 0.f;
  switch (P.isip_deg) {
    case 0: break;
    case 4: horner_pair<4, float>(P.isip_f[0], P.isip_f[1], an.U0, an.V0, ga, gb); break;
    case 6: horner_pair<6, float>(P.isip_f[0], P.isip_f[1], an.U0, an.V0, ga, gb); break;
    default: horner_pair<9, float>(P.isip_f[0], P.isip_f[1], an.U0, an.V0, ga, gb); break;
  }
  x = __fadd_rn(an.f0x, ga);
  y = __fadd_rn(an.f0y, gb);
  return an.h2 > 0.f;
}

__device__ __forceinline__ Anchor shfl_anchor(const Anchor& a, int src) {
  Anchor r;
  r.bx = __shfl_sync(0xffffffffu, a.bx, src);
  r.by = __shfl_sync(0xffffffffu, a.by, src);
  r.f0x = __shfl_sync(0xffffffffu, a.f0x, src);
  r.f0y = __shfl_sync(0xffffffffu, a.f0y, src);
  r.U0 = __shfl_sync(0xffffffffu, a.U0, src);
  r.V0 = __shfl_sync(0xffffffffu, a.V0, src);
  r.a0 = __shfl_sync(0xffffffffu, a.a0, src);
  r.a1 = __shfl_sync(0xffffffffu, a.a1, src);
  r.b0 = __shfl_sync(0xffffffffu, a.b0, src);
  r.b1 = __shfl_sync(0xffffffffu, a.b1, src);
  r.g20 = __shfl_sync(0xffffffffu, a.g20, src);
  r.g21 = __shfl_sync(0xffffffffu, a.g21, src);
  r.h2 = __shfl_sync(0xffffffffu, a.h2, src);
  r.tu = __shfl_sync(0xffffffffu, a.tu, src);
  r.tv = __shfl_sync(0xffffffffu, a.tv, src);
  r.tA = __shfl_sync(0xffffffffu, a.tA, src);
  r.tB = __shfl_sync(0xffffffffu, a.tB, src);
  return r;
}

// Warp-collective (all 32 lanes, lane = column): the cell's anchor and this lane's column
// cubic. (cox, coy): the cell's first column and row in the bounding box. INL: the sample
// evaluation inlined (forward kernels) or called (adjoint kernels); the same bits either way.
// FULL: every anchor field for every cell (the adjoint's chain rule needs them); otherwise only
// its integer base where the cell's cubics are valid.
template <bool INL = true, bool FULL = false>
__device__ __forceinline__ ColCubic cell_fit(const FwdPlan& P, const HP& Q, int cox, int coy,
                                             int lane, Anchor& anchor) {
  const unsigned full = 0xffffffffu;
  bool ok = true;
  float x = 0.f, y = 0.f;
  Anchor an;
  if (lane < 20) {
    const float2 p = cell_sample(lane);
    const float X = float(Q.x0 + cox) + (p.x + 15.5f), Y = float(Q.y0 + coy) + (p.y + kCellMid);
    ok = INL ? cell_point(P, Q, X, Y, an, x, y) : cell_point_call(P, Q, X, Y, an, x, y);
  }
  // the anchor's integer base (the whole anchor further down, where the cubics do not serve)
  const int abx = __shfl_sync(full, an.bx, 16), aby = __shfl_sync(full, an.by, 16);
  // sample positions relative to the anchor's base
  if (lane < 20) {
    const int ox = an.bx - abx, oy = an.by - aby;
    ok = ok && abs(ox) < (1 << 20) && abs(oy) < (1 << 20);
    x = __fadd_rn(x, float(ox));
    y = __fadd_rn(y, float(oy));
    ok = ok && fabsf(x) < 1048576.f && fabsf(y) < 1048576.f;
  }
  ColCubic cc;
  // this column's values at the four node rows
  float L[4];
  lagrange_x(float(lane) - 15.5f, L);
  float2 g[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = make_float2(__shfl_sync(full, x, i + 4 * j), __shfl_sync(full, y, i + 4 * j));
      const float2 Li = make_float2(L[i], L[i]);
      g[j] = i == 0 ? v_mul(Li, f) : v_fma(Li, f, g[j]);
    }
  }
  fit_s(g, cc.c);
  // checks: lane 16 + k holds the exact value at column kc[k], row s_k
  bool chk = true;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float ex = __shfl_sync(full, x, 16 + k), ey = __shfl_sync(full, y, 16 + k);
    const float2 sk = cell_sample(16 + k);
    if (lane == int(sk.x + 15.5f)) {
      const float2 q = cubic_pos(cc, sk.y);
      chk = fabsf(q.x - ex) <= kCubicTol && fabsf(q.y - ey) <= kCubicTol;
    }
  }
  cc.valid = __all_sync(full, ok && chk) && !Q.identity;
  if (cc.valid && !FULL) {
    anchor.bx = abx;
    anchor.by = aby;
  } else {
    anchor = shfl_anchor(an, 16);
  }
  return cc;
}

// Source position of row `row` (0..kCellH-1) of this lane's column: the column cubic where the
// cell is valid, else the exact evaluation (whose result says whether the pixel is defined).
// Relative to (anchor.bx, anchor.by).
__device__ __forceinline__ bool pixel_coords(const FwdPlan& P, const HP& Q, const Anchor& a,
                                             const ColCubic& cc, int lane, int row, float& x,
                                             float& y) {
  if (cc.valid) {
    const float2 p = cubic_pos(cc, float(row) - kCellMid);
    x = p.x;
    y = p.y;
    return true;
  }
  return exact_coords(P, Q, a, float(lane - kAnchorCol), float(row) - kCellMid, x, y);
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

// Box staging without TMA (stage_sw plans): every lane copies the columns lane and lane + 32
// of the kBoxW-wide box, row by row, with 4-byte asynchronous copies (cp.async), zero-filled
// outside the image like the TMA tile fill, as one commit group per box. The copies land
// before cp_async_wait (by the lane that issued them) plus a warp barrier.
__device__ __forceinline__ void cp_async_f32(float* dst, const float* src, bool inside) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)),
               "l"(src), "r"(inside ? 4 : 0)
               : "memory");
}

__device__ __forceinline__ void stage_box_sw(const FwdPlan& P, const HP& Q, float* box, int bx0,
                                             int by0, int lane) {
  static_assert(kBoxW == 64, "two columns per lane");
  for (int j = 0; j < Q.box_h; ++j) {
    const int gy = by0 + j;
    const bool iny = unsigned(gy) < unsigned(Q.H);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h, gx = bx0 + i;
      const bool in = iny && unsigned(gx) < unsigned(Q.W);
      // (an address inside the image even where nothing is read)
      cp_async_f32(box + j * kBoxW + i, P.img + (in ? int64_t(gy) * P.pitch + gx : 0), in);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Wait for this lane's copies but the newest `keep` commit groups (0 or 1).
template <int KEEP>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(KEEP) : "memory");
}

// SW: the kernel may meet stage_sw plans (the asynchronous-copy staging is compiled in).
template <int ORDER, bool SW = false>
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
  float x0 = 0.f, y0 = 0.f, x1 = 0.f, y1 = 0.f;
  bool ok = true;
  if (active) {
    ok = pixel_coords(P, Q, a, cc, lane, r0, x0, y0);
    ok = pixel_coords(P, Q, a, cc, lane, r0 + nrows - 1, x1, y1) && ok;
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
    if (SW && Q.stage_sw) {
      stage_box_sw(P, Q, box, tb.bx0, tb.by0, lane);
    } else if (lane == 0) {
      fence_proxy_async();
      if (map_in_gmem) fence_tensormap_acquire(&P.tmap);
      mbar_expect_tx(bar, uint32_t(Q.box_w) * uint32_t(Q.box_h) * 4u + tx_extra);
      tma_load_2d(box, &P.tmap, bar, tb.bx0, tb.by0);
    }
  }
  return tb;
}

}  // namespace dfr
