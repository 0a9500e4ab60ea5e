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

// Source box of a tile, decided from the source positions of its four corner pixels (lanes
// 0-3) widened by the plan's curvature margin, and loaded by one TMA copy (when `load`).
struct TileBox {
  int32_t bx0, by0;  // box origin (absolute source pixel)
  int32_t ex0, ey0, ew, eh;  // widened corner extent of the tile's taps, [ex0, ex0 + ew) etc.
  bool use_box;      // the box was loaded (else gather from global memory)
  bool interior;     // the widened extent lies inside the image: no tap needs masking
  bool empty;        // the widened extent misses the image: nothing in the tile is covered
};

template <int ORDER, int IDEG, bool PAIRS, bool TSIP_UNROLL = false>
__device__ __forceinline__ TileBox tile_box(const FwdPlan& P, const HotPlan<IDEG, PAIRS>& Q,
                                            const Anchor& a, int ox, int oy, int lane,
                                            float* box, uint64_t* bar, bool map_in_gmem,
                                            bool load = true) {
  using T = Taps<ORDER>;
  TileBox tb;
  tb.bx0 = tb.by0 = 0;
  tb.ex0 = tb.ey0 = tb.ew = tb.eh = 0;
  tb.use_box = tb.interior = tb.empty = false;
  if (ox >= Q.w || oy >= Q.h) {  // a cell's tile below the bounding box
    tb.empty = true;
    return tb;
  }
  const int cx = (lane & 1) ? min(kTileW, Q.w - ox) - 1 : 0;
  const int cy = (lane & 2) ? min(kTileH, Q.h - oy) - 1 : 0;
  float x = 0.f, y = 0.f;
  bool ok = true;
  if (lane < 4)
    ok = split_coords_core<IDEG, PAIRS, -1, TSIP_UNROLL>(
        P, Q.cab, Q.identity, Q.tsip, Q.newton, a, float(Q.x0 + ox + cx - a.ax),
        float(Q.y0 + oy + cy - a.ay), x, y);
  ok = ok && fabsf(x) < 1e7f && fabsf(y) < 1e7f;
  if (!__all_sync(0xffffffffu, ok)) return tb;  // corners undefined: gather per pixel
  const int fx = int(floorf(x)), fy = int(floorf(y));
  const int mnx = __reduce_min_sync(0xffffffffu, lane < 4 ? fx : INT_MAX);
  const int mxx = __reduce_max_sync(0xffffffffu, lane < 4 ? fx : INT_MIN);
  const int mny = __reduce_min_sync(0xffffffffu, lane < 4 ? fy : INT_MAX);
  const int mxy = __reduce_max_sync(0xffffffffu, lane < 4 ? fy : INT_MIN);
  const int M = P.box_margin;
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
      mbar_expect_tx(bar, uint32_t(Q.box_w) * uint32_t(Q.box_h) * 4u);
      tma_load_2d(box, &P.tmap, bar, tb.bx0, tb.by0);
    }
  }
  return tb;
}

}  // namespace dfr
