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
template <bool ACC>
__device__ __forceinline__ void prefetch_sums(const HP& Q, int ox, int oy, int rows, int lane) {
  if (!ACC) return;
  const int gx = ox + lane;
  if (gx >= Q.w || oy >= Q.h) return;
  const int nrows = min(rows, Q.h - oy);
  for (int r = 0; r < nrows; ++r) {
    const int64_t o = int64_t(oy + r) * Q.out_pitch + gx;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(Q.out + o));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(Q.fp + o));
  }
}

// ------------------------------------------------------------------ split-precision tiles
// A warp owns a 32 x 64 cell (lane = column); its rows are processed in tiles of TH rows, each
// with its source box staged in the warp's shared buffer by one TMA load. Per pixel the source
// position comes from the lane's column cubic (cell_fit).

// Value and footprint of one pixel from its taps. S(k, q) reads tap (row k, column q) and must
// return 0 outside the image. A pixel whose taps all lie inside the image has footprint
// exactly 1 (the weights sum to 1) and value = sum w S; otherwise out-of-image weights are
// zeroed, footprint = (sum wx)(sum wy) and value = sum w S / footprint. Every gather path
// (shared-memory box, global memory, the packed two-pixel rows) runs the same operation
// sequence: row_k = wx_0 S_k0 + wx_1 S_k1 + ... (a product, then FMAs in index order), then
// value = wy_0 row_0 + wy_1 row_1 + ... the same way.
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
        const float sv = S(xx - q, yy - k, k, q);
        row = q == 0 ? __fmul_rn(w[q].x, sv) : fmaf(w[q].x, sv, row);
      }
      num = k == 0 ? __fmul_rn(w[k].y, row) : fmaf(w[k].y, row, num);
    }
    return make_float2(num, 1.f);
  }
  float sx = 0.f, sy = 0.f;
  if (!interior) {
#pragma unroll
    for (int q = 0; q < T::n; ++q) {
      w[q].x = (unsigned(ix + q) < unsigned(W)) ? w[q].x : 0.f;
      w[q].y = (unsigned(iy + q) < unsigned(H)) ? w[q].y : 0.f;
      sx = __fadd_rn(sx, w[q].x);
      sy = __fadd_rn(sy, w[q].y);
    }
  }
  float num = 0.f;
#pragma unroll
  for (int k = 0; k < T::n; ++k) {
    float row = 0.f;
#pragma unroll
    for (int q = 0; q < T::n; ++q) {
      const float sv = S(ix, iy, k, q);
      row = q == 0 ? __fmul_rn(w[q].x, sv) : fmaf(w[q].x, sv, row);
    }
    num = k == 0 ? __fmul_rn(w[k].y, row) : fmaf(w[k].y, row, num);
  }
  if (interior) return make_float2(num, 1.f);
  const float f = __fmul_rn(sx, sy);
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

// floor(v) for |v| < 2^22 from v + 1.5 * 2^23 rounded toward minus infinity: the sum lies in
// [2^23, 2^24), where the floats are the integers, so it equals floor(v) + 1.5 * 2^23 exactly
// and its bit pattern is kFloorMagicBits + floor(v).
constexpr float kFloorMagic = 12582912.f;
constexpr uint32_t kFloorMagicBits = 0x4B400000u;

// Shared-memory load at a 32-bit shared-window address. Not volatile: the compiler may schedule
// these freely among the arithmetic; the caller derives every address from a token produced
// after the barrier wait that made the box visible (box_token), so none can move above it.
__device__ __forceinline__ float lds_f32(uint32_t addr) {
  float v;
  asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}

// An opaque 0, ordered after the preceding volatile operations (the mbarrier wait).
__device__ __forceinline__ uint32_t box_token() {
  uint32_t z;
  asm volatile("mov.u32 %0, 0;" : "=r"(z)::"memory");
  return z;
}

// Fast rows of a tile: TH full rows of 32 columns whose taps all lie in the loaded box and in
// the image (footprint 1), positions from a valid column cubic. Two rows per step in packed
// FP32x2 arithmetic (the pair = the same column in rows r and r + 1): positions, floors and
// fractions, weights, and the tap sums, each half the exact operation sequence of the
// per-pixel path (interp_pixel), so both give the same bits. The box pitch is the
// compile-time kBoxW: a pixel's taps are immediate offsets from one shared address.
// edge: the tile's taps may leave the image (the box holds zeros there, the TMA fill): per pixel
// also the coverage test and, unless all its taps are inside, the in-image weight sums as
// footprint and value = sum / footprint, as interp_pixel does (the zero taps add nothing to
// the sum, exactly like the zeroed weights there). fp: the footprint plane is written. Both are
// uniform runtime branches (one copy of the loop: a smaller kernel, at the same speed).
template <int ORDER, bool ACC, int TH>
__device__ __forceinline__ void tile_rows_fast_impl(const HP& Q, const Anchor& a,
                                                    const ColCubic& cc, int gx, int oy, int r0,
                                                    uint32_t sbox, const TileBox& tb,
                                                    const bool fp, const bool edge) {
  using T = Taps<ORDER>;
  constexpr int n = T::n;
  // edge: absolute first-tap column/row = floor bits + (bx + lo - magic bits); coverage bounds
  const int kxa = a.bx + T::lo - int(kFloorMagicBits), kya = a.by + T::lo - int(kFloorMagicBits);
  const float xlo = -0.5f - float(a.bx), xhi = float(Q.W) - 0.5f - float(a.bx);
  const float ylo = -0.5f - float(a.by), yhi = float(Q.H) - 0.5f - float(a.by);
  // shared address of a pixel's first tap: sbox + 4 ((floor(y) + by + lo - by0) kBoxW +
  // floor(x) + bx + lo - bx0), with the floors as bit patterns (modular arithmetic)
  const uint32_t kb = sbox + 4u * (uint32_t((a.by + T::lo - tb.by0) * kBoxW +
                                            (a.bx + T::lo - tb.bx0)) -
                                   kFloorMagicBits * uint32_t(kBoxW + 1));
  const float2 cx0 = v_c<float2>(cc.c[0].x), cx1 = v_c<float2>(cc.c[1].x);
  const float2 cx2 = v_c<float2>(cc.c[2].x), cx3 = v_c<float2>(cc.c[3].x);
  const float2 cy0 = v_c<float2>(cc.c[0].y), cy1 = v_c<float2>(cc.c[1].y);
  const float2 cy2 = v_c<float2>(cc.c[2].y), cy3 = v_c<float2>(cc.c[3].y);
  const float2 magic = v_c<float2>(kFloorMagic);
  const int64_t pitch = Q.out_pitch;
  float* po = Q.out + int64_t(oy) * pitch + gx;
  float* pf = fp ? Q.fp + int64_t(oy) * pitch + gx : nullptr;
  float2 s = make_float2(float(r0) - kCellMid, float(r0 + 1) - kCellMid);
#pragma unroll 2
  for (int i = 0; i < TH / 2; ++i) {
    const float2 X = v_fma(v_fma(v_fma(cx3, s, cx2), s, cx1), s, cx0);
    const float2 Y = v_fma(v_fma(v_fma(cy3, s, cy2), s, cy1), s, cy0);
    const float2 mx = __fadd2_rd(X, magic), my = __fadd2_rd(Y, magic);
    const float2 tx = v_sub(X, v_sub(mx, magic)), ty = v_sub(Y, v_sub(my, magic));
    uint32_t ia = __float_as_uint(my.x) * uint32_t(4 * kBoxW) + __float_as_uint(mx.x) * 4u + kb;
    uint32_t ib = __float_as_uint(my.y) * uint32_t(4 * kBoxW) + __float_as_uint(mx.y) * 4u + kb;
    float2 num;
    float2 wx[n], wy[n];
    auto wxs = [&](int q) { return wx[q]; };
    auto wys = [&](int q) { return wy[q]; };
    if (ORDER == DFR_NEAREST) {
      ia += 4u * (uint32_t(tx.x >= 0.5f) + uint32_t(kBoxW) * uint32_t(ty.x >= 0.5f));
      ib += 4u * (uint32_t(tx.y >= 0.5f) + uint32_t(kBoxW) * uint32_t(ty.y >= 0.5f));
      num = make_float2(lds_f32(ia), lds_f32(ib));
    } else {
      if (ORDER == DFR_LANCZOS3) {
        float ax[6], bxw[6], ay[6], byw[6];
        lanczos3_weights<float>(tx.x, ax);
        lanczos3_weights<float>(tx.y, bxw);
        lanczos3_weights<float>(ty.x, ay);
        lanczos3_weights<float>(ty.y, byw);
#pragma unroll
        for (int q = 0; q < n; ++q) {
          wx[q] = make_float2(ax[q], bxw[q]);
          wy[q] = make_float2(ay[q], byw[q]);
        }
      } else {
        weights_v<ORDER, float2>(tx, wx);
        weights_v<ORDER, float2>(ty, wy);
      }
#pragma unroll
      for (int k = 0; k < n; ++k) {
        float2 row;
#pragma unroll
        for (int q = 0; q < n; ++q) {
          const uint32_t off = uint32_t(4 * (k * kBoxW + q));
          const float2 sv = make_float2(lds_f32(ia + off), lds_f32(ib + off));
          row = q == 0 ? v_mul(wx[q], sv) : v_fma(wx[q], sv, row);
        }
        num = k == 0 ? v_mul(wy[k], row) : v_fma(wy[k], row, num);
      }
    }
    float2 fpv = make_float2(1.f, 1.f);
    if (edge) {
      // per pixel (half h = A, B): coverage, interior taps, else in-image weight sums
      float v2[2] = {num.x, num.y}, f2[2] = {1.f, 1.f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float xh_ = h ? X.y : X.x, yh_ = h ? Y.y : Y.x;
        const float txh = h ? tx.y : tx.x, tyh = h ? ty.y : ty.x;
        int ix = int(__float_as_uint(h ? mx.y : mx.x)) + kxa;
        int iy = int(__float_as_uint(h ? my.y : my.x)) + kya;
        if (ORDER == DFR_NEAREST) {
          ix += txh >= 0.5f;
          iy += tyh >= 0.5f;
        }
        const bool cov = xh_ >= xlo && xh_ <= xhi && yh_ >= ylo && yh_ <= yhi;
        const bool inner = ix >= 0 && ix + n <= Q.W && iy >= 0 && iy + n <= Q.H;
        float f = 1.f;
        if (!inner) {
          if (ORDER == DFR_NEAREST) {
            f = 0.f;
          } else {
            float sx = 0.f, sy = 0.f;
#pragma unroll
            for (int q = 0; q < n; ++q) {
              sx = __fadd_rn(sx, (unsigned(ix + q) < unsigned(Q.W)) ? (h ? wxs(q).y : wxs(q).x) : 0.f);
              sy = __fadd_rn(sy, (unsigned(iy + q) < unsigned(Q.H)) ? (h ? wys(q).y : wys(q).x) : 0.f);
            }
            f = __fmul_rn(sx, sy);
          }
        }
        const float v = v2[h];
        v2[h] = (!cov || f == 0.f) ? 0.f : ((f == 1.f) ? v : __fdividef(v, f));
        f2[h] = (!cov || f == 0.f) ? 0.f : f;
      }
      num = make_float2(v2[0], v2[1]);
      fpv = make_float2(f2[0], f2[1]);
    }
    if (ACC) {
      put_pixel<true>(po, pf, num.x, fpv.x);
      put_pixel<true>(po + pitch, pf + pitch, num.y, fpv.y);
    } else {
      __stcs(po, num.x);
      __stcs(po + pitch, num.y);
      if (fp) {
        __stcs(pf, fpv.x);
        __stcs(pf + pitch, fpv.y);
      }
    }
    po += 2 * pitch;
    if (fp) pf += 2 * pitch;
    s = v_add(s, make_float2(2.f, 2.f));
  }
}

template <int ORDER, bool ACC, int TH>
__device__ __forceinline__ void tile_rows_fast(const HP& Q, const Anchor& a, const ColCubic& cc,
                                               int gx, int oy, int r0, uint32_t sbox,
                                               const TileBox& tb) {
  tile_rows_fast_impl<ORDER, ACC, TH>(Q, a, cc, gx, oy, r0, sbox, tb, ACC || Q.fp != nullptr,
                                      !tb.interior);
}

// General rows of a tile (per pixel): position (column cubic or exact), coverage, then the
// gather from the box when the pixel's taps are in it, else from global memory; masking,
// image edges and B-spline mirroring as the plan needs.
template <int ORDER, bool ACC>
__device__ __forceinline__ void tile_rows(const FwdPlan& P, const HP& Q, const Anchor& a,
                                          const ColCubic& cc, int gx, int oy, int r0, int nrows,
                                          const float* box, const TileBox& tb) {
  using T = Taps<ORDER>;
  if (oy >= Q.h || gx >= Q.w) return;
  const float xlo = -0.5f - float(a.bx), xhi = float(Q.W) - 0.5f - float(a.bx);
  const float ylo = -0.5f - float(a.by), yhi = float(Q.H) - 0.5f - float(a.by);
  const int lane = gx & (kCellW - 1);
  const int bw = Q.box_w, bh = Q.box_h;
  nrows = min(nrows, Q.h - oy);
  float* po = Q.out + int64_t(oy) * Q.out_pitch + gx;
  float* pf = Q.fp ? Q.fp + int64_t(oy) * Q.out_pitch + gx : nullptr;
#pragma unroll 1
  for (int r = 0; r < nrows; ++r) {
    float x, y;
    const bool ok = pixel_coords(P, Q, a, cc, lane, r0 + r, x, y);
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
// Resident one-warp CTAs per SM the register budget targets: 16 (128 registers: the two-pixel
// rows hold two pixels' taps, weights and column coefficients at once).
constexpr int kSplitMinBlocks = 16;

__device__ __forceinline__ int frame_of(const FwdLaunch& L, int t) {
  int lo = 0, hi = L.nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The same frame, found by one warp: a 32-way search over the prefix table, each step one
// coalesced load per lane and a ballot (one step for up to 32 frames, two up to 1024).
__device__ __forceinline__ int frame_of_warp(const FwdLaunch& L, int t, int lane) {
  int lo = 0, n = L.nframes;  // tile_start[lo] <= t; the frame is in [lo, lo + n)
  while (n > 1) {
    const int step = (n + 31) >> 5;
    const bool le = lane * step < n && __ldg(&L.tile_start[lo + lane * step]) <= t;
    const int k = 31 - __clz(int(__ballot_sync(0xffffffffu, le)));  // lane 0 always holds
    lo += k * step;
    n = min(step, n - k * step);
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

// BATCH: frame plans in global memory (a frame table: the cells of all frames in one index
// space, frame by frame, found from the prefix table); otherwise one frame whose plan is the
// kernel parameter, cells [unit_begin, unit_begin + grid) (a band of the box, or all of it).
// Either way one cell per CTA: the hardware scheduler balances the launch; the cells of its
// last partial wave may be split into units of fewer tiles (split_from, split_k).
//
// A CTA is one warp and owns one 32 x 64 cell: the warp fits the cell's column cubics
// (cell_fit), then the cell's rows go by in tiles of TH rows, the next tile's source box
// requested (TMA or asynchronous copies, double buffered) before the current one is gathered.
// After a bounded wait gives up, the warp issues no more box loads and gathers from global
// memory; before exiting it waits (bounded) for any copy still in flight into its buffers.
template <int ORDER, bool BATCH, bool ACC, int TH, bool SW>
__global__ void __launch_bounds__(kFwdWarps * 32, kSplitMinBlocks) fwd_split_kernel(
    const __grid_constant__ FwdPlan p0, const FwdLaunch L) {
  static_assert(kCellH % TH == 0 && TH % 2 == 0, "tile height must divide the cell");
  extern __shared__ __align__(128) float box_raw[];
  __shared__ __align__(8) uint64_t s_bar[2];
  const int lane = threadIdx.x & 31;
  // 128-byte aligned source-box buffers (the launch reserves 128 bytes of slack)
  const int skew = int((128u - (smem_addr(box_raw) & 127u)) & 127u) / 4;
  float* box = box_raw + skew;  // two buffers of L.box_floats
  uint64_t* bar = s_bar;
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncwarp();
  uint32_t phase = 0;    // bit b: parity of the next wait on buffer b
  uint32_t pending = 0;  // bit b: a copy into buffer b has not been waited for
  bool dead = false;     // a wait gave up: no more copies from this warp
  constexpr bool batch = BATCH;
  constexpr int NT = kCellH / TH;
  // the cell of this CTA; cells from split_from on are split into split_k units of NT /
  // split_k tiles each
  const int total = batch ? L.tile_start[L.nframes] : L.total_tiles;
  int id = blockIdx.x + (batch ? 0 : L.unit_begin);
  int t0 = 0, t1 = NT;
  if (L.split_k > 1 && id >= L.split_from) {
    const int u = id - L.split_from, part = u % L.split_k;
    id = L.split_from + u / L.split_k;
    t0 = part * (NT / L.split_k);
    t1 = t0 + NT / L.split_k;
  }
  if (id < total) {
    int f = 0, cell = id;
    if (batch) {
      f = frame_of_warp(L, cell, lane);
      cell -= __ldg(&L.tile_start[f]);
    }
    const FwdPlan& P = batch ? L.plans[f] : p0;
    HP Q;
    load_hot(P, Q);
    Q.use_tma = Q.use_tma && !dead;
    const int cox = (cell % P.cells_x) * kCellW, coy = (cell / P.cells_x) * kCellH;
    const int gx = cox + lane;
    Anchor a;
    const ColCubic cc = cell_fit(P, Q, cox, coy, lane, a);
    // fast rows need every column's cubic, bowing well inside the box margin
    const bool fast_cell = !Q.mask && cc.valid &&
                           __all_sync(0xffffffffu, cubic_bow(cc, TH) <= 0.5f) &&
                           cox + kCellW <= Q.w;
    TileBox cur = tile_box<ORDER, SW>(P, Q, a, cc, cox, coy + t0 * TH, t0 * TH, TH, lane,
                                  box + (t0 & 1) * L.box_floats, &bar[t0 & 1], batch, true,
                                  L.tx_extra);
    const bool sw = SW && Q.stage_sw;
    if (cur.use_box && !sw) pending |= 1u << (t0 & 1);
    prefetch_sums<ACC>(Q, cox, coy + t0 * TH, TH, lane);
    for (int t = t0; t < t1; ++t) {
      const int b = t & 1;
      TileBox nxt;
      nxt.use_box = false;
      if (t + 1 < t1) {
        nxt = tile_box<ORDER, SW>(P, Q, a, cc, cox, coy + (t + 1) * TH, (t + 1) * TH, TH, lane,
                              box + (b ^ 1) * L.box_floats, &bar[b ^ 1], batch, true, L.tx_extra);
        if (nxt.use_box && !sw) pending |= 1u << (b ^ 1);
        prefetch_sums<ACC>(Q, cox, coy + (t + 1) * TH, TH, lane);
      }
      uint32_t tok = 0;
      if (cur.use_box && sw) {
        // this tile's copies (all but the newest group when the next box is on its way)
        if (nxt.use_box)
          cp_async_wait<1>();
        else
          cp_async_wait<0>();
        __syncwarp();
        tok = box_token();
      } else if (cur.use_box) {
        if (mbar_wait(&bar[b], (phase >> b) & 1u)) {
          phase ^= 1u << b;
          pending &= ~(1u << b);
          tok = box_token();
        } else {  // timed out: this buffer's phase is unknown, gather from global memory
          cur.use_box = false;
          dead = true;
          Q.use_tma = false;
        }
      }
      const int oy = coy + t * TH;
      const float* bt = box + b * L.box_floats;
      // fast rows: the box holds every tap (zeros outside the image); the B-spline's mirrored
      // taps near the image edge take the general rows
      if (fast_cell && cur.use_box && oy + TH <= Q.h &&
          (cur.interior || ORDER != DFR_BSPLINE3))
        tile_rows_fast<ORDER, ACC, TH>(Q, a, cc, gx, oy, t * TH, smem_addr(bt) + tok, cur);
      else
        tile_rows<ORDER, ACC>(P, Q, a, cc, gx, oy, t * TH, TH, bt, cur);
      cur = nxt;
    }
  }
  // copies this warp issued and never saw complete (after a wait gave up) must land before
  // the CTA's shared memory is released
  for (int b = 0; b < 2; ++b)
    if ((pending >> b) & 1u) mbar_wait(&bar[b], (phase >> b) & 1u, false);
  if (SW) asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace dfr
