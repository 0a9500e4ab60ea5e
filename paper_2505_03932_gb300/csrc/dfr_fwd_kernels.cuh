// Forward kernel templates (FP64 path and split path), shared by the translation units that
// instantiate them: dfr_fwd.cu (stored outputs) and dfr_coadd.cu (co-add sums, ACC = true).
#pragma once

#include <climits>

#include "dfr_device.cuh"
#include "dfr_tile.cuh"

namespace dfr {

constexpr int kFp64Threads = 256;  // block size of the FP64 kernel

// Output of one pixel: value and footprint stored (ACC = false), or added to the co-add sums
// (ACC = true): sum_vf += value * footprint, sum_f += footprint, uncovered pixels untouched.
// Within one launch every output pixel belongs to one thread, so the read-modify-write needs
// no atomics; frames of a co-add run one after another.
template <bool ACC>
__device__ __forceinline__ void put_pixel(float* po, float* pf, float v, float f) {
  if (ACC) {
    if (f != 0.f) {
      *po = fmaf(v, f, *po);
      *pf += f;
    }
  } else {
    __stcs(po, v);
    if (pf) __stcs(pf, f);
  }
}

// ------------------------------------------------------------------ FP64 tile (plain method)
// Per pixel: the printed formulas in FP64, direct gather, FP64 weights and sums.
template <int ORDER, int NT, bool ACC>
__device__ __forceinline__ void fp64_tile(const FwdPlan& P, int tile) {
  constexpr int PPT = kTilePix / NT;
  const int ox = (tile % P.tiles_x) * kTileW, oy = (tile / P.tiles_x) * kTileH;
  using T = Taps<ORDER>;
#pragma unroll 1
  for (int k = 0; k < PPT; ++k) {
    const int i = threadIdx.x + k * NT;
    const int gx = ox + (i % kTileW), gy = oy + (i / kTileW);
    if (gx >= P.w || gy >= P.h) continue;
    double xs, ys;
    const bool ok = source_from_target_fp64(P, double(P.x0 + gx), double(P.y0 + gy), xs, ys);
    const int64_t o = int64_t(gy) * P.out_pitch + gx;
    if (P.coords) {
      double* c = P.coords + 2 * (int64_t(gy) * P.w + gx);
      c[0] = ok ? xs : __longlong_as_double(0x7ff8000000000000ll);
      c[1] = ok ? ys : __longlong_as_double(0x7ff8000000000000ll);
    }
    float val = 0.f, fpv = 0.f;
    // snap coordinates within kSnap of an integer (FP64 round-off of an exact map)
    const double rx = rint(xs), ry = rint(ys);
    if (fabs(xs - rx) < kSnap) xs = rx;
    if (fabs(ys - ry) < kSnap) ys = ry;
    if (ok && xs >= -0.5 && xs <= P.W - 0.5 && ys >= -0.5 && ys <= P.H - 0.5) {
      double fx = floor(xs), fy = floor(ys);
      const double tx = xs - fx, ty = ys - fy;
      if (ORDER == DFR_NEAREST) {
        if (tx >= 0.5) fx += 1.0;
        if (ty >= 0.5) fy += 1.0;
      }
      double wx[T::n], wy[T::n];
      weights<ORDER, double>(tx, wx);
      weights<ORDER, double>(ty, wy);
      const int ix = int(fx) + T::lo, iy = int(fy) + T::lo;
      if (ORDER == DFR_BSPLINE3) {
        // coefficients continue by mirroring outside the image; footprint 1
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < T::n; ++b) {
          const int yy = mirror_index(iy + b, P.H);
          double row = 0.0;
#pragma unroll
          for (int a = 0; a < T::n; ++a)
            row += wx[a] * double(__ldg(P.img + int64_t(yy) * P.pitch + mirror_index(ix + a, P.W)));
          acc += wy[b] * row;
        }
        if (ACC) {
          put_pixel<true>(P.out + o, P.fp + o, float(acc), 1.f);
        } else {
          P.out[o] = float(acc);
          if (P.fp) P.fp[o] = 1.f;
        }
        continue;
      }
      double num = 0.0, sx = 0.0, sy = 0.0;
#pragma unroll
      for (int a = 0; a < T::n; ++a) {
        if (ix + a < 0 || ix + a >= P.W) wx[a] = 0.0;
        if (iy + a < 0 || iy + a >= P.H) wy[a] = 0.0;
        sx += wx[a];
        sy += wy[a];
      }
      const bool mask = (P.flags & DFR_NAN_MASK) != 0;
      double fm = 0.0;  // masked footprint
#pragma unroll
      for (int b = 0; b < T::n; ++b) {
        double row = 0.0, rowf = 0.0;
        const int yy = iy + b;
        if (wy[b] != 0.0) {
#pragma unroll
          for (int a = 0; a < T::n; ++a) {
            const int xx = ix + a;
            if (wx[a] == 0.0) continue;
            const double s = double(__ldg(P.img + int64_t(yy) * P.pitch + xx));
            if (mask && s != s) continue;  // NaN tap: missing
            row += wx[a] * s;
            rowf += wx[a];
          }
        }
        num += wy[b] * row;
        fm += wy[b] * rowf;
      }
      const double f = mask ? fm : sx * sy;
      if (mask ? f > 0.0 : f != 0.0) {
        val = float(num / f);
        fpv = float(f);
      }
    }
    if (ACC) {
      put_pixel<true>(P.out + o, P.fp + o, val, fpv);
    } else {
      P.out[o] = val;
      if (P.fp) P.fp[o] = fpv;
    }
  }
}

// Co-add launches: ask L2 for a tile's accumulator rows (value and weight sums) one tile ahead,
// so the read-modify-write of put_pixel<true> does not wait on HBM. Addresses inside the
// output box only.
template <bool ACC, int IDEG, bool PAIRS>
__device__ __forceinline__ void prefetch_sums(const HotPlan<IDEG, PAIRS>& Q, int ox, int oy,
                                              int lane) {
  if (!ACC) return;
  const int gx = ox + lane;
  if (gx >= Q.w || oy >= Q.h) return;
  const int nrows = min(kTileH, Q.h - oy);
  for (int r = 0; r < nrows; ++r) {
    const int64_t o = int64_t(oy + r) * Q.out_pitch + gx;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(Q.out + o));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(Q.fp + o));
  }
}

// ------------------------------------------------------------------ split-precision tiles
// One warp owns a 32x8 tile at a time: lane = column, 8 rows per lane. Per pixel the source
// position comes in FP32 from the anchor of the pixel's 32x32 cell; per tile a TMA load
// stages the source box covering the tile's taps in the warp's shared buffer.

// Value and footprint of one pixel from its taps. S(k, q) reads tap (row k, column q) and must
// return 0 outside the image. A pixel whose taps all lie inside the image has footprint
// exactly 1 (the weights sum to 1) and value = sum w S; otherwise out-of-image weights are
// zeroed, footprint = (sum wx)(sum wy) and value = sum w S / footprint. Every gather path
// (shared-memory box, global memory, the fast tile path) runs the same operation sequence:
// row_k = sum_q wx_q S_kq, then value = sum_k wy_k row_k, each a chain of FMAs in index order.
template <int ORDER, bool INTERIOR, typename Tap>
__device__ __forceinline__ float2 interp_pixel(float x, float y, int bx, int by, int W, int H,
                                               const Tap& S) {
  using T = Taps<ORDER>;
  const float flx = floorf(x), fly = floorf(y);
  const float2 t = make_float2(x - flx, y - fly);
  int ix = int(flx), iy = int(fly);
  if (ORDER == DFR_NEAREST) {
    ix += t.x >= 0.5f;
    iy += t.y >= 0.5f;
  }
  ix += bx + T::lo;  // absolute source column / row of the first tap
  iy += by + T::lo;
  const bool interior = INTERIOR || (ix >= 0 && ix + T::n <= W && iy >= 0 && iy + T::n <= H);
  float2 w[T::n];
  weights2<ORDER>(t, w);
  if (ORDER == DFR_NEAREST) {
    const float v = S(ix, iy, 0, 0);
    return interior ? make_float2(v, 1.f) : make_float2(0.f, 0.f);
  }
  if (ORDER == DFR_BSPLINE3 && !interior) {
    // B-spline coefficients continue by mirroring outside the image; footprint 1
    float num = 0.f;
#pragma unroll
    for (int k = 0; k < T::n; ++k) {
      const int yy = mirror_index(iy + k, H);
      float row = 0.f;
#pragma unroll
      for (int q = 0; q < T::n; ++q) {
        const int xx = mirror_index(ix + q, W);
        row = fmaf(w[q].x, S(xx - q, yy - k, k, q), row);
      }
      num = fmaf(w[k].y, row, num);
    }
    return make_float2(num, 1.f);
  }
  float sx = 0.f, sy = 0.f;
  if (!interior) {
#pragma unroll
    for (int q = 0; q < T::n; ++q) {
      w[q].x = (unsigned(ix + q) < unsigned(W)) ? w[q].x : 0.f;
      w[q].y = (unsigned(iy + q) < unsigned(H)) ? w[q].y : 0.f;
      sx += w[q].x;
      sy += w[q].y;
    }
  }
  float num = 0.f;
#pragma unroll
  for (int k = 0; k < T::n; ++k) {
    float row = 0.f;
#pragma unroll
    for (int q = 0; q < T::n; ++q) row = fmaf(w[q].x, S(ix, iy, k, q), row);
    num = fmaf(w[k].y, row, num);
  }
  if (interior) return make_float2(num, 1.f);
  const float f = sx * sy;
  if (f == 0.f) return make_float2(0.f, 0.f);
  return make_float2((f == 1.f) ? num : __fdividef(num, f), f);
}

// NaN-masked form (DFR_NAN_MASK): a tap whose source value is NaN is missing, like a tap
// outside the image. Footprint = sum of the weights of the in-image finite taps, value =
// sum w S / footprint; both 0 unless that sum is positive (signed bicubic weights can leave a
// sum <= 0 once taps are missing). Per tap: row_k = sum_q m_kq wx_q S_kq and
// rowf_k = sum_q m_kq wx_q (m = 0 or 1), then sum_k wy_k row_k and sum_k wy_k rowf_k.
template <int ORDER, typename Tap>
__device__ __forceinline__ float2 interp_pixel_masked(float x, float y, int bx, int by, int W,
                                                      int H, const Tap& S) {
  using T = Taps<ORDER>;
  const float flx = floorf(x), fly = floorf(y);
  const float2 t = make_float2(x - flx, y - fly);
  int ix = int(flx), iy = int(fly);
  if (ORDER == DFR_NEAREST) {
    ix += t.x >= 0.5f;
    iy += t.y >= 0.5f;
  }
  ix += bx + T::lo;
  iy += by + T::lo;
  if (ORDER == DFR_NEAREST) {
    const bool in = unsigned(ix) < unsigned(W) && unsigned(iy) < unsigned(H);
    const float v = in ? S(ix, iy, 0, 0) : 0.f;
    return (in && v == v) ? make_float2(v, 1.f) : make_float2(0.f, 0.f);
  }
  float2 w[T::n];
  weights2<ORDER>(t, w);
#pragma unroll
  for (int q = 0; q < T::n; ++q) {
    w[q].x = (unsigned(ix + q) < unsigned(W)) ? w[q].x : 0.f;
    w[q].y = (unsigned(iy + q) < unsigned(H)) ? w[q].y : 0.f;
  }
  float num = 0.f, f = 0.f;
#pragma unroll
  for (int k = 0; k < T::n; ++k) {
    float row = 0.f, rowf = 0.f;
#pragma unroll
    for (int q = 0; q < T::n; ++q) {
      const float s = S(ix, iy, k, q);
      const bool ok = s == s;
      row = fmaf(ok ? w[q].x : 0.f, ok ? s : 0.f, row);
      rowf += ok ? w[q].x : 0.f;
    }
    num = fmaf(w[k].y, row, num);
    f = fmaf(w[k].y, rowf, f);
  }
  if (!(f > 0.f)) return make_float2(0.f, 0.f);
  return make_float2((f == 1.f) ? num : __fdividef(num, f), f);
}

// Masked gather from a warp's shared-memory box whose origin is (bx0, by0), width bw. Not
// inlined: the masked path is rare, and its registers stay out of the kernels' hot rows.
template <int ORDER>
__device__ __noinline__ float2 gather_box_masked(const float* box, int bw, int bx0, int by0,
                                                 int W, int H, float x, float y, int bx, int by) {
  auto SB = [=](int ixa, int iya, int k, int q) -> float {
    return box[(iya + k - by0) * bw + (ixa + q - bx0)];
  };
  return interp_pixel_masked<ORDER>(x, y, bx, by, W, H, SB);
}

// Fallback gather straight from global memory (tiles whose box does not fit, or no TMA).
template <int ORDER>
__device__ __noinline__ float2 gather_global(const float* __restrict__ img, int64_t pitch, int W,
                                             int H, float x, float y, int bx, int by,
                                             bool mask = false) {
  auto S = [=](int ix, int iy, int k, int q) -> float {
    const int xx = ix + q, yy = iy + k;
    return (unsigned(xx) < unsigned(W) && unsigned(yy) < unsigned(H))
               ? __ldg(img + int64_t(yy) * pitch + xx)
               : 0.f;
  };
  if (mask) return interp_pixel_masked<ORDER>(x, y, bx, by, W, H, S);
  return interp_pixel<ORDER, false>(x, y, bx, by, W, H, S);
}

// Rows of one tile: per pixel the split coordinates, coverage, then the gather from the box
// (fast when the tile is interior) or from global memory.
// Fast rows: the tile lies inside the bounding box, its widened source extent inside the image
// and inside the loaded box, and the plan has no Newton inverse, NaN mask or identity. No
// per-pixel branch: taps are read from the box at clamped positions and the rare pixel whose
// taps leave the box (the curvature margin was too small) is redone from global memory.
template <int ORDER, int IDEG, bool PAIRS, bool ACC, bool TSIP>
__device__ __forceinline__ void tile_rows_fast(const FwdPlan& P, const HotPlan<IDEG, PAIRS>& Q,
                                               const Anchor& a, int ox, int oy, int lane,
                                               const float* box, const TileBox& tb) {
  using T = Taps<ORDER>;
  const int gx = ox + lane;
  const float dx = float(Q.x0 + gx - a.ax);
  float dy = float(Q.y0 + oy - a.ay);
  const int bw = Q.box_w;
  // a pixel is taken here only if all its taps lie in the widened extent, which is inside the
  // image (no masking, footprint 1) and inside the box
  const unsigned uxmax = unsigned(tb.ew - T::n), uymax = unsigned(tb.eh - T::n);
  const int ux0 = a.bx + T::lo - tb.ex0, uy0 = a.by + T::lo - tb.ey0;
  const int sx0 = tb.ex0 - tb.bx0, sy0 = tb.ey0 - tb.by0;  // extent origin within the box
  float* po = Q.out + int64_t(oy) * Q.out_pitch + gx;
  float* pf = Q.fp ? Q.fp + int64_t(oy) * Q.out_pitch + gx : nullptr;
  uint32_t bad = 0;
  // measured: by 4 for the plain kernels (1.6 % over 2; full unrolling costs instruction
  // fetch), by 2 for Lanczos-3 and target-SIP rows (more registers per row)
  constexpr int kUnroll = (ORDER == DFR_LANCZOS3 || TSIP) ? 2 : 4;
#pragma unroll kUnroll
  for (int r = 0; r < kTileH; ++r) {
    float x, y;
    const bool ok = split_coords_core<IDEG, PAIRS, -1, TSIP>(P, Q.cab, false, TSIP, false, a, dx,
                                                             dy, x, y);
    const float flx = floorf(x), fly = floorf(y);
    const float2 t = make_float2(x - flx, y - fly);
    int ux = int(flx) + ux0, uy = int(fly) + uy0;
    if (ORDER == DFR_NEAREST) {
      ux += t.x >= 0.5f;
      uy += t.y >= 0.5f;
    }
    const bool in_ext = ok && unsigned(ux) <= uxmax && unsigned(uy) <= uymax;
    bad |= uint32_t(!in_ext) << r;
    const float* b = box + ((in_ext ? uy : 0) + sy0) * bw + (in_ext ? ux : 0) + sx0;
    float num;
    if (ORDER == DFR_NEAREST) {
      num = b[0];
    } else {
      float2 w[T::n];
      weights2<ORDER>(t, w);
      num = 0.f;
#pragma unroll
      for (int k = 0; k < T::n; ++k) {
        float row = 0.f;
#pragma unroll
        for (int q = 0; q < T::n; ++q) row = fmaf(w[q].x, b[k * bw + q], row);
        num = fmaf(w[k].y, row, num);
      }
    }
    if (ACC) {
      if (in_ext) put_pixel<true>(po + int64_t(r) * Q.out_pitch, pf + int64_t(r) * Q.out_pitch,
                                  num, 1.f);
    } else {
      put_pixel<false>(po + int64_t(r) * Q.out_pitch, pf ? pf + int64_t(r) * Q.out_pitch : nullptr,
                       num, 1.f);
    }
    dy += 1.f;
  }
  if (__any_sync(0xffffffffu, bad != 0) && bad) {
    // pixels outside the box: the general per-pixel path, from global memory
    const float xlo = -0.5f - float(a.bx), xhi = float(Q.W) - 0.5f - float(a.bx);
    const float ylo = -0.5f - float(a.by), yhi = float(Q.H) - 0.5f - float(a.by);
    for (int r = 0; r < kTileH; ++r) {
      if (!((bad >> r) & 1u)) continue;
      float x, y;
      const bool ok = split_coords_core<IDEG, PAIRS>(P, Q.cab, false, TSIP, false, a, dx,
                                                     float(Q.y0 + oy - a.ay) + float(r), x, y);
      float2 vf = make_float2(0.f, 0.f);
      if (ok && x >= xlo && x <= xhi && y >= ylo && y <= yhi)
        vf = gather_global<ORDER>(P.img, P.pitch, Q.W, Q.H, x, y, a.bx, a.by);
      put_pixel<ACC>(po + int64_t(r) * Q.out_pitch, pf ? pf + int64_t(r) * Q.out_pitch : nullptr,
                     vf.x, vf.y);
    }
  }
}

// General rows: per pixel the split coordinates, coverage, then the gather from the box (when
// its taps are in the box) or from global memory.
template <int ORDER, int IDEG, bool PAIRS, bool ACC, bool TSIP>
__device__ __forceinline__ void tile_rows(const FwdPlan& P, const HotPlan<IDEG, PAIRS>& Q,
                                          const Anchor& a, int ox, int oy, int lane,
                                          const float* box, const TileBox& tb) {
  using T = Taps<ORDER>;
  if (oy >= Q.h) return;
  // (the fast rows of a TSIP instantiation serve plans with target SIP, the others plans
  // without; the remaining plans take the general rows)
  const bool plain = !Q.identity && !Q.newton && !Q.mask && Q.tsip == TSIP;
  if (plain && tb.use_box && tb.interior && ox + kTileW <= Q.w && oy + kTileH <= Q.h) {
    tile_rows_fast<ORDER, IDEG, PAIRS, ACC, TSIP>(P, Q, a, ox, oy, lane, box, tb);
    return;
  }
  const int gx = ox + lane;
  if (gx >= Q.w) return;
  const float xlo = -0.5f - float(a.bx), xhi = float(Q.W) - 0.5f - float(a.bx);
  const float ylo = -0.5f - float(a.by), yhi = float(Q.H) - 0.5f - float(a.by);
  const float dx = float(Q.x0 + gx - a.ax);
  const float dy0 = float(Q.y0 + oy - a.ay);
  const int bw = Q.box_w, bh = Q.box_h;
  const int nrows = min(kTileH, Q.h - oy);
  float* po = Q.out + int64_t(oy) * Q.out_pitch + gx;
  float* pf = Q.fp ? Q.fp + int64_t(oy) * Q.out_pitch + gx : nullptr;
#pragma unroll 1
  for (int r = 0; r < nrows; ++r) {
    float x, y;
    const bool ok = split_coords_core<IDEG, PAIRS>(P, Q.cab, Q.identity, Q.tsip, Q.newton, a,
                                                   dx, dy0 + float(r), x, y);
    float2 vf = make_float2(0.f, 0.f);
    if (!tb.empty && ok && x >= xlo && x <= xhi && y >= ylo && y <= yhi) {
      const float flx = floorf(x), fly = floorf(y);
      const float2 t = make_float2(x - flx, y - fly);
      int ix = int(flx), iy = int(fly);
      if (ORDER == DFR_NEAREST) {
        ix += t.x >= 0.5f;
        iy += t.y >= 0.5f;
      }
      // first tap relative to the box origin
      const int cx = ix + a.bx + T::lo - tb.bx0, cy = iy + a.by + T::lo - tb.by0;
      bool in_box = tb.use_box && cx >= 0 && cx + T::n <= bw && cy >= 0 && cy + T::n <= bh;
      if (ORDER == DFR_BSPLINE3) {
        // near the image edge the taps are mirrored: the box must hold the mirrored positions
        const int ixa = ix + a.bx + T::lo, iya = iy + a.by + T::lo;
        int mx0 = INT_MAX, mx1 = INT_MIN, my0 = INT_MAX, my1 = INT_MIN;
#pragma unroll
        for (int q = 0; q < T::n; ++q) {
          const int mx = mirror_index(ixa + q, Q.W), my = mirror_index(iya + q, Q.H);
          mx0 = min(mx0, mx);
          mx1 = max(mx1, mx);
          my0 = min(my0, my);
          my1 = max(my1, my);
        }
        in_box = tb.use_box && mx0 >= tb.bx0 && mx1 < tb.bx0 + bw && my0 >= tb.by0 &&
                 my1 < tb.by0 + bh;
      }
      if (in_box) {
        const int bx0 = tb.bx0, by0 = tb.by0;
        auto SB = [=](int ixa, int iya, int k, int q) -> float {
          return box[(iya + k - by0) * bw + (ixa + q - bx0)];
        };
        vf = Q.mask ? gather_box_masked<ORDER>(box, bw, bx0, by0, Q.W, Q.H, x, y, a.bx, a.by)
                    : interp_pixel<ORDER, false>(x, y, a.bx, a.by, Q.W, Q.H, SB);
      } else {
        vf = gather_global<ORDER>(P.img, P.pitch, Q.W, Q.H, x, y, a.bx, a.by, Q.mask);
      }
    }
    put_pixel<ACC>(po, pf, vf.x, vf.y);
    po += Q.out_pitch;
    if (pf) pf += Q.out_pitch;
  }
}

// ------------------------------------------------------------------ kernels
// CTAs (of kWarps warps) per SM the register budget targets: 6 (80 registers) for single-frame
// launches, whose inverse-SIP coefficients are constant-bank operands; 4 (128) for batch
// launches, which hold them in registers.
// Accumulating (co-add) launches hold the read-modify-write operands as well, and target-SIP
// launches the target polynomial: 5 (96 registers). Lanczos-3 (36 taps): 4 (128 registers).
constexpr int split_min_blocks(bool batch, bool acc, bool tsip, int order) {
  return (batch || order == DFR_LANCZOS3) ? 4 : ((acc || tsip) ? 5 : 6);
}

__device__ __forceinline__ int frame_of(const FwdLaunch& L, int t) {
  int lo = 0, hi = L.nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int ORDER, int NT, bool ACC>
__global__ void __launch_bounds__(NT) fwd_fp64_kernel(const __grid_constant__ FwdPlan p0,
                                                      const FwdLaunch L) {
  if (L.plans == nullptr) {
    fp64_tile<ORDER, NT, ACC>(p0, blockIdx.x);
    return;
  }
  __shared__ int32_t s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(L.counter, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= L.tile_start[L.nframes]) break;
    const int f = frame_of(L, t);
    fp64_tile<ORDER, NT, ACC>(L.plans[f], t - L.tile_start[f]);
  }
}

// BATCH: frame plans in global memory (persistent launch over a frame table), inverse-SIP
// coefficients held in registers as FP32x2 pairs; otherwise one frame whose plan is the kernel
// parameter, read as constant-bank operands by scalar FMAs (fewer registers).
//
// Work unit: kCellsPerCta consecutive 32x32 anchor cells. Warp 0 computes their anchors
// (one lane per cell), then each warp processes the 4 tiles of each of its kCellsPerWarp cells,
// requesting the source box of the next tile before gathering the current one.
template <int ORDER, int IDEG, bool BATCH, bool ACC, bool TSIP = false>
__global__ void __launch_bounds__(kWarps * 32, split_min_blocks(BATCH, ACC, TSIP, ORDER)) fwd_split_kernel(
    const __grid_constant__ FwdPlan p0, const FwdLaunch L) {
  extern __shared__ __align__(128) float box_raw[];
  __shared__ Anchor s_anc[kCellsPerCta];
  __shared__ int32_t s_frame[kCellsPerCta];
  __shared__ int32_t s_cell[kCellsPerCta];
  __shared__ __align__(8) uint64_t s_bar[kWarps][2];
  __shared__ int32_t s_unit;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // 128-byte aligned source-box buffers (the launch reserves 128 bytes of slack); indexing the
  // shared array itself keeps the compiler on shared-memory loads
  const int skew = int((128u - (smem_addr(box_raw) & 127u)) & 127u) / 4;
  float* box = box_raw + skew + warp * 2 * L.box_floats;  // two buffers per warp
  uint64_t* bar = &s_bar[warp][0];
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  uint32_t phase = 0;  // bit b: parity of the next wait on buffer b
  constexpr bool batch = BATCH;
  // cells; a single-frame launch may cover units [unit_begin, unit_begin + grid) only (bands)
  const int total = batch ? L.tile_start[L.nframes] : L.total_tiles;
  const int nunits = (total + kCellsPerCta - 1) / kCellsPerCta;
  // grid launch: one unit per CTA (from unit_begin); persistent: units from a counter
  int unit = blockIdx.x + L.unit_begin;
  if (batch) {
    if (threadIdx.x == 0) s_unit = atomicAdd(L.counter, 1);
    __syncthreads();
    unit = s_unit;
  }
  while (unit < nunits) {
    const int c0 = unit * kCellsPerCta;
    const int nc = min(kCellsPerCta, total - c0);
    if (warp == 0 && lane < nc) {  // anchors of the unit's cells, one per lane
      int f = 0, cell = c0 + lane;
      if (batch) {
        f = frame_of(L, cell);
        cell -= L.tile_start[f];
      }
      const FwdPlan& P = batch ? L.plans[f] : p0;
      const int cox = (cell % P.cells_x) * kCellW, coy = (cell / P.cells_x) * kCellH;
      make_anchor(P, P.x0 + cox + kCellW / 2, P.y0 + coy + kCellH / 2, s_anc[lane]);
      s_frame[lane] = f;
      s_cell[lane] = cell;
    }
    __syncthreads();
    // this warp's tiles: kTilesPerCell per cell, cells warp*kCellsPerWarp ...
    const int j0 = warp * kCellsPerWarp;
    const int ncw = max(0, min(kCellsPerWarp, nc - j0));
    const int nt = ncw * kTilesPerCell;
    if (nt > 0) {
      TileBox cur;
      {
        const FwdPlan& P = batch ? L.plans[s_frame[j0]] : p0;
        HotPlan<IDEG, BATCH> Q;
        load_hot(P, Q);
        const Anchor a = s_anc[j0];
        const int cell = s_cell[j0];
        cur = tile_box<ORDER, IDEG, BATCH, TSIP>(P, Q, a, (cell % P.cells_x) * kCellW,
                                                 (cell / P.cells_x) * kCellH, lane, box, &bar[0],
                                                 batch);
        prefetch_sums<ACC>(Q, (cell % P.cells_x) * kCellW, (cell / P.cells_x) * kCellH, lane);
      }
      for (int t = 0; t < nt; ++t) {
        const int b = t & 1;
        TileBox nxt;
        nxt.use_box = false;
        if (t + 1 < nt) {
          const int jn = j0 + (t + 1) / kTilesPerCell, kn = (t + 1) % kTilesPerCell;
          const FwdPlan& Pn = batch ? L.plans[s_frame[jn]] : p0;
          HotPlan<IDEG, BATCH> Qn;
          load_hot(Pn, Qn);
          const Anchor an = s_anc[jn];
          const int celln = s_cell[jn];
          nxt = tile_box<ORDER, IDEG, BATCH, TSIP>(
              Pn, Qn, an, (celln % Pn.cells_x) * kCellW,
              (celln / Pn.cells_x) * kCellH + kn * kTileH, lane, box + (b ^ 1) * L.box_floats,
              &bar[b ^ 1], batch);
          prefetch_sums<ACC>(Qn, (celln % Pn.cells_x) * kCellW,
                             (celln / Pn.cells_x) * kCellH + kn * kTileH, lane);
        }
        const int j = j0 + t / kTilesPerCell, k = t % kTilesPerCell;
        const FwdPlan& P = batch ? L.plans[s_frame[j]] : p0;
        HotPlan<IDEG, BATCH> Q;
        load_hot(P, Q);
        const Anchor a = s_anc[j];
        const int cell = s_cell[j];
        if (cur.use_box) {
          if (!mbar_wait(&bar[b], (phase >> b) & 1u)) cur.use_box = false;  // timed out
          phase ^= 1u << b;
        }
        tile_rows<ORDER, IDEG, BATCH, ACC, TSIP>(P, Q, a, (cell % P.cells_x) * kCellW,
                                      (cell / P.cells_x) * kCellH + k * kTileH, lane,
                                      box + b * L.box_floats, cur);
        cur = nxt;
      }
    }
    if (!batch) break;
    __syncthreads();  // every warp is done with this unit's anchors
    if (threadIdx.x == 0) s_unit = atomicAdd(L.counter, 1);
    __syncthreads();
    unit = s_unit;
  }
}

}  // namespace dfr
