// Tile-staged adjoint of the split-precision reprojection (dfr_reproject_backward), sm_103a.
//
// Work decomposition: kBwdCellsPerCta 32x64 cells per CTA, one per warp, each cell as 8 tiles
// of 32x8 (lane = column); source positions from the same cell fits as the forward kernels
// (bit for bit). The chain rule's inverse-SIP Jacobian comes from per-cell cubics as well
// (fit_jacobian), for the polynomial and the Newton inverse. Per tile the source box is
// staged by TMA into the warp's shared buffer (the taps are read from it) and a second buffer
// of the same shape collects the tile's dL/dS contributions with shared-memory atomics; the
// buffer is then added to grad_src with one global atomic per non-zero element (instead of one
// per tap and pixel). Per-pixel parameter terms accumulate per lane in registers over the
// cell's 64 pixels, and are summed over the warp once per cell. CTAs stride over the cells
// (grid sized for residency) so every CTA's partial covers a fixed set of cells: the parameter
// gradients are deterministic.
#include <climits>

#include "dfr_adjoint.cuh"
#include "dfr_tile.cuh"

namespace dfr {

// Source intermediate offsets (U, V) of target offset (dx, dy) from the anchor: the part of
// split_coords_core before the inverse SIP, with the same operations (so the same bits as its
// geo[0], geo[1] added to the anchor's (U0, V0)).
__device__ __forceinline__ void split_uv(const FwdPlan& P, const HP& Q, const Anchor& a, float dx,
                                         float dy, float& U, float& V) {
  if (Q.identity) {
    U = a.U0 + dx;
    V = a.V0 + dy;
    return;
  }
  float dp = dx, dq = dy;
  if (Q.tsip) {
    float fa, fb;
    tsip_pair(P, __fadd_rn(a.tu, dx), __fadd_rn(a.tv, dy), fa, fb);
    dp = __fadd_rn(dx, __fsub_rn(fa, a.tA));
    dq = __fadd_rn(dy, __fsub_rn(fb, a.tB));
  }
  const float nu = fmaf(a.a0, dp, __fmul_rn(a.a1, dq));
  const float nv = fmaf(a.b0, dp, __fmul_rn(a.b1, dq));
  const float den = fmaf(a.g20, dp, fmaf(a.g21, dq, a.h2));
  const float rcp = __fdividef(1.f, den);
  U = a.U0 + __fmul_rn(nu, rcp);
  V = a.V0 + __fmul_rn(nv, rcp);
}

// The inverse-SIP Jacobian M = d(u, v)/d(U, V) over a cell, as the positions are: sampled at
// the 4x4 Lobatto nodes (lane i + 4 j), interpolated across the columns by the Lagrange
// weights and fitted by a cubic in s per column. Polynomial inverse (FD = 0): M = I +
// d(AP, BP)/d(U, V), a polynomial of one degree less than AP/BP in (U, V); Newton inverse: M =
// (I + d(A, B)/d(u, v))^-1 at the node's exact solution (u, v). Either is a smooth function of
// the pixel, which the cubics reproduce to FP32 rounding for polynomials up to degree 4 and
// closely beyond; the per-pixel chain rule then evaluates two cubics instead of polynomial
// gradients (and, with the Newton inverse, instead of the Newton solve).
struct JacCubic {
  float2 r0[4], r1[4];  // (m00, m01) and (m10, m11) coefficients in s
};

template <int IDEG, int FD>
__device__ __forceinline__ JacCubic fit_jacobian(const FwdPlan& P, const HP& Q, const Anchor& a,
                                                 int lane) {
  const unsigned full = 0xffffffffu;
  float m00 = 1.f, m01 = 0.f, m10 = 0.f, m11 = 1.f;
  if (lane < 16) {
    const float2 p = cell_sample(lane);
    float A, Au, Av, Bq, Bu, Bv;
    if (FD == 0) {
      float U, V;
      split_uv(P, Q, a, p.x - 0.5f, p.y, U, V);
      poly_grad<IDEG, float>(P.isip_f[0], P.isip_deg, U, V, A, Au, Av);
      poly_grad<IDEG, float>(P.isip_f[1], P.isip_deg, U, V, Bq, Bu, Bv);
      m00 = 1.f + Au;
      m01 = Av;
      m10 = Bu;
      m11 = 1.f + Bv;
    } else {
      float xe, ye, geo[4];
      split_coords_core<IDEG, false, FD>(P, nullptr, Q.identity, Q.tsip, Q.newton, a,
                                         p.x - 0.5f, p.y, xe, ye, geo);
      const float u = a.U0 + geo[2], v = a.V0 + geo[3];
      poly_grad<FD, float>(P.fsip_f[0], P.fsip_deg, u, v, A, Au, Av);
      poly_grad<FD, float>(P.fsip_f[1], P.fsip_deg, u, v, Bq, Bu, Bv);
      const float j00 = 1.f + Au, j01 = Av, j10 = Bu, j11 = 1.f + Bv;
      const float inv = __fdividef(1.f, fmaf(j00, j11, -j01 * j10));
      m00 = j11 * inv;
      m01 = -j01 * inv;
      m10 = -j10 * inv;
      m11 = j00 * inv;
    }
  }
  float L[4];
  lagrange_x(float(lane) - 15.5f, L);
  float2 g0[4], g1[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int src = i + 4 * j;
      const float2 f0 = make_float2(__shfl_sync(full, m00, src), __shfl_sync(full, m01, src));
      const float2 f1 = make_float2(__shfl_sync(full, m10, src), __shfl_sync(full, m11, src));
      const float2 Li = make_float2(L[i], L[i]);
      g0[j] = i == 0 ? v_mul(Li, f0) : v_fma(Li, f0, g0[j]);
      g1[j] = i == 0 ? v_mul(Li, f1) : v_fma(Li, f1, g1[j]);
    }
  }
  JacCubic J;
  fit_s(g0, J.r0);
  fit_s(g1, J.r1);
  return J;
}

__device__ __forceinline__ float2 jac_row(const float2 c[4], float s) {
  const float2 ss = make_float2(s, s);
  return v_fma(v_fma(v_fma(c[3], ss, c[2]), ss, c[1]), ss, c[0]);
}

template <int ORDER, int IDEG, int FD>
__device__ __forceinline__ void bwd_tile_rows(const FwdPlan& P, const HP& Q, const BwdExtra& B,
                                              const ChainConst& K, const Anchor& a,
                                              const ColCubic& cc, int ox, int oy, int r0,
                                              int lane, const float* box, float* gbox,
                                              const TileBox& tb, bool want_params, float* acc,
                                              const JacCubic& J) {
  using T = Taps<ORDER>;
  constexpr int NTERM = nterms(FD);
  const int gx = ox + lane;
  if (gx >= Q.w) return;
  const float xlo = -0.5f - float(a.bx), xhi = float(Q.W) - 0.5f - float(a.bx);
  const float ylo = -0.5f - float(a.by), yhi = float(Q.H) - 0.5f - float(a.by);
  const float dx0 = float(lane - kAnchorCol);
  // the anchor base in source intermediate offsets (for u, v of the Newton inverse's terms)
  const float ub = float(double(a.bx) - P.crpix_s[0]), vb = float(double(a.by) - P.crpix_s[1]);
  const int bw = Q.box_w, bh = Q.box_h;
  const int nrows = min(kTileH, Q.h - oy);
#pragma unroll 1
  for (int r = 0; r < nrows; ++r) {
    float x, y;
    float U = 0.f, V = 0.f;
    const bool ok = pixel_coords(P, Q, a, cc, lane, r0 + r, x, y);
    // the chain rule's intermediate offsets (U, V) from the local homography; M from the cell's
    // Jacobian cubics
    if (want_params) split_uv(P, Q, a, dx0, float(r0 + r) - kCellMid, U, V);
    const bool cov = !tb.empty && ok && x >= xlo && x <= xhi && y >= ylo && y <= yhi;
    float gxs = 0.f, gys = 0.f;
    if (cov) {
      const float flx = floorf(x), fly = floorf(y);
      const float tx = x - flx, ty = y - fly;
      int ix = int(flx), iy = int(fly);
      if (ORDER == DFR_NEAREST) {
        ix += tx >= 0.5f;
        iy += ty >= 0.5f;
      }
      ix += a.bx + T::lo;  // first tap, absolute source pixel
      iy += a.by + T::lo;
      float wx[T::n], wy[T::n], dwx[T::n], dwy[T::n];
      weights<ORDER, float>(tx, wx);
      weights<ORDER, float>(ty, wy);
      if (want_params) {
        dweights<ORDER, float>(tx, dwx);
        dweights<ORDER, float>(ty, dwy);
      }
      float sx = 0.f, sy = 0.f;
#pragma unroll
      for (int q = 0; q < T::n; ++q) {
        const bool inx = unsigned(ix + q) < unsigned(Q.W);
        const bool iny = unsigned(iy + q) < unsigned(Q.H);
        wx[q] = inx ? wx[q] : 0.f;
        wy[q] = iny ? wy[q] : 0.f;
        if (want_params) {
          dwx[q] = inx ? dwx[q] : 0.f;
          dwy[q] = iny ? dwy[q] : 0.f;
        }
        sx += wx[q];
        sy += wy[q];
      }
      const float F = sx * sy;
      const int cx = ix - tb.bx0, cy = iy - tb.by0;  // first tap within the box
      const bool in_box = tb.use_box && cx >= 0 && cx + T::n <= bw && cy >= 0 && cy + T::n <= bh;
      if (F != 0.f) {
        const float g = B.grad_out[int64_t(oy + r) * B.go_pitch + gx];
        const float gF = __fdividef(g, F);
        if (B.grad_src) {
          if (in_box) {
            // every tap position is in the box; masked taps (outside the image) add 0 there
            // and the flush skips them
#pragma unroll
            for (int k = 0; k < T::n; ++k) {
              const float gw = gF * wy[k];
              float* row = gbox + (cy + k) * bw + cx;
#pragma unroll
              for (int q = 0; q < T::n; ++q) atomicAdd(row + q, gw * wx[q]);
            }
          } else {
#pragma unroll
            for (int k = 0; k < T::n; ++k)
#pragma unroll
              for (int q = 0; q < T::n; ++q) {
                const float w = wx[q] * wy[k];
                if (w != 0.f)
                  atomicAdd(B.grad_src + int64_t(iy + k) * B.gs_pitch + (ix + q), gF * w);
              }
          }
        }
        if (want_params) {
          // value = sum_k wy_k row_k / F with row_k = sum_q wx_q S_kq; the position derivatives
          // d(value)/dx = sum_k wy_k (sum_q dwx_q S_kq - value sum_q dwx_q) / F and
          // d(value)/dy = sum_k dwy_k (row_k - value sum_q wx_q) / F
          float row[T::n], rowd[T::n];
          float num = 0.f, sdx = 0.f;
#pragma unroll
          for (int q = 0; q < T::n; ++q) sdx += dwx[q];
          // taps from the staged box (branch-free), else from global memory (masked)
          if (in_box) {
            const float* b0 = box + cy * bw + cx;
#pragma unroll
            for (int k = 0; k < T::n; ++k) {
              float rw = 0.f, rd = 0.f;
#pragma unroll
              for (int q = 0; q < T::n; ++q) {
                const float sv = b0[k * bw + q];
                rw = fmaf(wx[q], sv, rw);
                rd = fmaf(dwx[q], sv, rd);
              }
              row[k] = rw;
              rowd[k] = rd;
            }
          } else {
#pragma unroll
            for (int k = 0; k < T::n; ++k) {
              const bool iny = unsigned(iy + k) < unsigned(Q.H);
              float rw = 0.f, rd = 0.f;
#pragma unroll
              for (int q = 0; q < T::n; ++q) {
                const bool in = iny && unsigned(ix + q) < unsigned(Q.W);
                const float sv = in ? __ldg(P.img + int64_t(iy + k) * P.pitch + (ix + q)) : 0.f;
                rw = fmaf(wx[q], sv, rw);
                rd = fmaf(dwx[q], sv, rd);
              }
              row[k] = rw;
              rowd[k] = rd;
            }
          }
#pragma unroll
          for (int k = 0; k < T::n; ++k) num = fmaf(wy[k], row[k], num);
          const float val = __fdividef(num, F);
          float ax_ = 0.f, ay_ = 0.f;
#pragma unroll
          for (int k = 0; k < T::n; ++k) {
            ax_ = fmaf(wy[k], fmaf(-val, sdx, rowd[k]), ax_);
            ay_ = fmaf(dwy[k], fmaf(-val, sx, row[k]), ay_);
          }
          gxs = gF * ax_;
          gys = gF * ay_;
        }
      }
    }
    if (!want_params || !cov) continue;
    float lu, lv, c[6];
    const float sr = float(r0 + r) - kCellMid;
    const bool jac = FD > 0 || IDEG != 0;
    const float2 mr0 = jac ? jac_row(J.r0, sr) : make_float2(1.f, 0.f);
    const float2 mr1 = jac ? jac_row(J.r1, sr) : make_float2(0.f, 1.f);
    chain_terms_m(K, gxs, gys, U, V, mr0.x, mr0.y, mr1.x, mr1.y, lu, lv, c);
    // Newton inverse: the SIP coefficient terms at the pixel's intermediate offsets after the
    // inverse, u = x_s - CRPIX1 (the position the cell cubic gives), likewise v
    const float u = ub + x, v = vb + y;
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[q] += c[q];
    if (FD > 0) {
      float up[FD + 1], vp[FD + 1];
      up[0] = vp[0] = 1.f;
#pragma unroll
      for (int e = 1; e <= FD; ++e) {
        up[e] = up[e - 1] * u;
        vp[e] = vp[e - 1] * v;
      }
      int t = 0;
#pragma unroll
      for (int n = 1; n <= FD; ++n)
#pragma unroll
        for (int p = n; p >= 0; --p, ++t) {
          const float m = up[p] * vp[n - p];
          acc[6 + t] = fmaf(-lu, m, acc[6 + t]);
          acc[6 + NTERM + t] = fmaf(-lv, m, acc[6 + NTERM + t]);
        }
    }
  }
}

// Fast rows of a tile (interior tiles of cells with valid cubics: every pixel covered, every tap
// inside the image and inside the staged boxes, all 32 columns and kTileH rows in the box): the
// per-pixel work of bwd_tile_rows with the same arithmetic in the same order (so the same
// terms), without its per-pixel coverage, masking, box and fallback branches, and with the box
// pitch kBoxW as a compile-time constant (tap offsets are immediates).
template <int ORDER, int IDEG, int FD>
__device__ __forceinline__ void bwd_tile_rows_fast(const FwdPlan& P, const HP& Q,
                                                   const BwdExtra& B, const ChainConst& K,
                                                   const Anchor& a, const ColCubic& cc, int ox,
                                                   int oy, int r0, int lane, const float* box,
                                                   float* gbox, const TileBox& tb,
                                                   bool want_params, float* acc,
                                                   const JacCubic& J) {
  using T = Taps<ORDER>;
  constexpr int NTERM = nterms(FD);
  constexpr int BW = kBoxW;
  const int gx = ox + lane;
  const float dx0 = float(lane - kAnchorCol);
  const float ub = float(double(a.bx) - P.crpix_s[0]), vb = float(double(a.by) - P.crpix_s[1]);
  const float* go = B.grad_out + int64_t(oy) * B.go_pitch + gx;
  const int kx = a.bx + T::lo - tb.bx0, ky = a.by + T::lo - tb.by0;  // box offset of the taps
  // The gradient taps of successive rows, summed in registers over the window of box rows
  // they share: when the next row's taps start one box row lower in the same column, the
  // window's first row goes to the gradient box and the window moves down one row; any other
  // step sends the whole window. (Successive target rows of a column usually step one source
  // row: 4 shared-memory atomics per pixel instead of 16.) With the Newton inverse's 46
  // accumulators the window's registers would spill: there every tap goes straight to the box.
  constexpr bool WIN = FD == 0;
  float win[T::n][T::n];
  int wb = -1;  // box index of the window's first tap; -1: empty
  auto send_row = [&](int w) {
#pragma unroll
    for (int q = 0; q < T::n; ++q) atomicAdd(gbox + wb + w * BW + q, win[w][q]);
  };
#pragma unroll 2
  for (int r = 0; r < kTileH; ++r) {
    const float sr = float(r0 + r) - kCellMid;
    const float2 pos = cubic_pos(cc, sr);
    const float x = pos.x, y = pos.y;
    float U = 0.f, V = 0.f;
    if (want_params) split_uv(P, Q, a, dx0, sr, U, V);
    const float flx = floorf(x), fly = floorf(y);
    const float tx = x - flx, ty = y - fly;
    int cx = int(flx) + kx, cy = int(fly) + ky;  // first tap within the box
    if (ORDER == DFR_NEAREST) {
      cx += tx >= 0.5f;
      cy += ty >= 0.5f;
    }
    float wx[T::n], wy[T::n], dwx[T::n], dwy[T::n];
    weights<ORDER, float>(tx, wx);
    weights<ORDER, float>(ty, wy);
    if (want_params) {
      dweights<ORDER, float>(tx, dwx);
      dweights<ORDER, float>(ty, dwy);
    }
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int q = 0; q < T::n; ++q) {
      sx += wx[q];
      sy += wy[q];
    }
    const float F = sx * sy;
    const float g = go[int64_t(r) * B.go_pitch];
    const float gF = __fdividef(g, F);
    const int b0 = cy * BW + cx;
    if (!WIN && B.grad_src) {
#pragma unroll
      for (int k = 0; k < T::n; ++k) {
        const float gw = gF * wy[k];
#pragma unroll
        for (int q = 0; q < T::n; ++q) atomicAdd(gbox + b0 + k * BW + q, gw * wx[q]);
      }
    }
    if (WIN && B.grad_src) {
      float t[T::n][T::n];
#pragma unroll
      for (int k = 0; k < T::n; ++k) {
        const float gw = gF * wy[k];
#pragma unroll
        for (int q = 0; q < T::n; ++q) t[k][q] = gw * wx[q];
      }
      if (b0 == wb + BW) {  // one box row down: send the window's first row, move it down
        send_row(0);
#pragma unroll
        for (int k = 0; k + 1 < T::n; ++k)
#pragma unroll
          for (int q = 0; q < T::n; ++q) win[k][q] = win[k + 1][q];
#pragma unroll
        for (int q = 0; q < T::n; ++q) win[T::n - 1][q] = 0.f;
        wb = b0;
      } else if (b0 != wb) {  // elsewhere: send the whole window, start a new one
        if (wb >= 0) {
#pragma unroll
          for (int k = 0; k < T::n; ++k) send_row(k);
        }
#pragma unroll
        for (int k = 0; k < T::n; ++k)
#pragma unroll
          for (int q = 0; q < T::n; ++q) win[k][q] = 0.f;
        wb = b0;
      }
#pragma unroll
      for (int k = 0; k < T::n; ++k)
#pragma unroll
        for (int q = 0; q < T::n; ++q) win[k][q] += t[k][q];
    }
    if (!want_params) continue;
    float row[T::n], rowd[T::n];
    float num = 0.f, sdx = 0.f;
#pragma unroll
    for (int q = 0; q < T::n; ++q) sdx += dwx[q];
#pragma unroll
    for (int k = 0; k < T::n; ++k) {
      float rw = 0.f, rd = 0.f;
#pragma unroll
      for (int q = 0; q < T::n; ++q) {
        const float sv = box[b0 + k * BW + q];
        rw = fmaf(wx[q], sv, rw);
        rd = fmaf(dwx[q], sv, rd);
      }
      row[k] = rw;
      rowd[k] = rd;
    }
#pragma unroll
    for (int k = 0; k < T::n; ++k) num = fmaf(wy[k], row[k], num);
    const float val = __fdividef(num, F);
    float ax_ = 0.f, ay_ = 0.f;
#pragma unroll
    for (int k = 0; k < T::n; ++k) {
      ax_ = fmaf(wy[k], fmaf(-val, sdx, rowd[k]), ax_);
      ay_ = fmaf(dwy[k], fmaf(-val, sx, row[k]), ay_);
    }
    const float gxs = gF * ax_, gys = gF * ay_;
    float lu, lv, c[6];
    const bool jac = FD > 0 || IDEG != 0;
    const float2 mr0 = jac ? jac_row(J.r0, sr) : make_float2(1.f, 0.f);
    const float2 mr1 = jac ? jac_row(J.r1, sr) : make_float2(0.f, 1.f);
    chain_terms_m(K, gxs, gys, U, V, mr0.x, mr0.y, mr1.x, mr1.y, lu, lv, c);
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[q] += c[q];
    if (FD > 0) {
      const float u = ub + x, v = vb + y;
      float up[FD + 1], vp[FD + 1];
      up[0] = vp[0] = 1.f;
#pragma unroll
      for (int e = 1; e <= FD; ++e) {
        up[e] = up[e - 1] * u;
        vp[e] = vp[e - 1] * v;
      }
      int t = 0;
#pragma unroll
      for (int n = 1; n <= FD; ++n)
#pragma unroll
        for (int p = n; p >= 0; --p, ++t) {
          const float m = up[p] * vp[n - p];
          acc[6 + t] = fmaf(-lu, m, acc[6 + t]);
          acc[6 + NTERM + t] = fmaf(-lv, m, acc[6 + NTERM + t]);
        }
    }
  }
  if (WIN && B.grad_src && wb >= 0) {
#pragma unroll
    for (int k = 0; k < T::n; ++k) send_row(k);
  }
}

// Adds the warp's gradient box to grad_src (non-zero elements inside the image) and clears it.
__device__ __forceinline__ void flush_gbox(const HP& Q, const BwdExtra& B,
                                           const TileBox& tb, float* gbox, int lane) {
  const int bw = Q.box_w, bh = Q.box_h;
  for (int j = 0; j < bh; ++j) {
    const int sy = tb.by0 + j;
    for (int i = lane; i < bw; i += 32) {
      const float v = gbox[j * bw + i];
      if (v == 0.f) continue;
      gbox[j * bw + i] = 0.f;
      const int sx = tb.bx0 + i;
      if (unsigned(sx) < unsigned(Q.W) && unsigned(sy) < unsigned(Q.H))
        atomicAdd(B.grad_src + int64_t(sy) * B.gs_pitch + sx, v);
    }
  }
}

template <int ORDER, int IDEG, int FD>
__global__ void __launch_bounds__(kBwdWarps * 32, 4) bwd_split_kernel(const __grid_constant__ FwdPlan P,
                                                                const __grid_constant__ BwdExtra B) {
  constexpr int NTERM = nterms(FD);
  constexpr int NP = 6 + 2 * NTERM;
  extern __shared__ __align__(128) float bsm_raw[];
  __shared__ double s_acc[kBwdWarps][NP];
  __shared__ __align__(8) uint64_t s_bar[kBwdWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int skew = int((128u - (smem_addr(bsm_raw) & 127u)) & 127u) / 4;
  float* box = bsm_raw + skew + warp * 2 * B.box_floats;  // source box, then gradient box
  float* gbox = box + B.box_floats;
  uint64_t* bar = &s_bar[warp];
  if (lane == 0) mbar_init(bar, 1);
  for (int q = lane; q < NP; q += 32) s_acc[warp][q] = 0.0;
  for (int i = lane; i < B.box_floats; i += 32) gbox[i] = 0.f;
  __syncwarp();
  uint32_t phase = 0;
  bool dead = false;  // a wait gave up: no more box loads from this warp
  bool pending = false;  // a box load has not been waited for
  HP Q;
  load_hot(P, Q);
  const ChainConst K = chain_const(P);
  const bool want_params = B.grad_params != nullptr && ORDER != DFR_NEAREST;
  const int total = P.cells_x * P.cells_y;
  const int nunits = (total + kBwdCellsPerCta - 1) / kBwdCellsPerCta;
  for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
    const int c0 = unit * kBwdCellsPerCta;
    const int nc = min(kBwdCellsPerCta, total - c0);
    if (warp < nc) {
      const int cell = c0 + warp;
      const int cox = (cell % P.cells_x) * kCellW, coy = (cell / P.cells_x) * kCellH;
      Anchor a;
      const ColCubic cc = cell_fit<false, true>(P, Q, cox, coy, lane, a);
      Q.use_tma = P.use_tma != 0 && !P.stage_sw && !dead;
      JacCubic J;
      if ((FD > 0 || IDEG != 0) && want_params) J = fit_jacobian<IDEG, FD>(P, Q, a, lane);
      // the fast rows need every column's cubic, bowing well inside the box margin
      const bool fast_cell = cc.valid && !Q.mask && cox + kCellW <= Q.w &&
                             __all_sync(0xffffffffu, cubic_bow(cc, kTileH) <= 0.5f);
      float acc[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) acc[q] = 0.f;
      for (int k = 0; k < kTilesPerCell; ++k) {
        const int oy = coy + k * kTileH;
        if (oy >= Q.h) break;
        // the source values are needed only for the parameter terms
        TileBox tb = tile_box<ORDER>(P, Q, a, cc, cox, oy, k * kTileH, kTileH, lane, box, bar,
                                     false, want_params);
        if (tb.empty) continue;
        if (tb.use_box && want_params) {
          pending = true;
          if (mbar_wait(bar, phase)) {
            phase ^= 1u;
            pending = false;
          } else {  // timed out: global memory instead, and no more box loads
            tb.use_box = false;
            dead = true;
            Q.use_tma = false;
          }
        }
        // interior tiles of valid cells, all columns and rows present, every tap in the boxes
        if (fast_cell && tb.use_box && tb.interior && oy + kTileH <= Q.h && Q.box_w == kBoxW)
          bwd_tile_rows_fast<ORDER, IDEG, FD>(P, Q, B, K, a, cc, cox, oy, k * kTileH, lane, box,
                                              gbox, tb, want_params, acc, J);
        else
          bwd_tile_rows<ORDER, IDEG, FD>(P, Q, B, K, a, cc, cox, oy, k * kTileH, lane, box,
                                         gbox, tb, want_params, acc, J);
        if (tb.use_box && B.grad_src) {
          __syncwarp();
          flush_gbox(Q, B, tb, gbox, lane);
          __syncwarp();
        }
      }
      if (want_params) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const float t = warp_sum(acc[q]);
          if (lane == 0) s_acc[warp][q] += double(t);
        }
      }
    }
  }
  // a copy still in flight into this warp's buffer must land before the CTA exits
  if (pending) mbar_wait(bar, phase, false);
  if (B.partials) {
    __syncthreads();  // every warp's accumulators are final
    for (int q = threadIdx.x; q < NP; q += kBwdWarps * 32) {
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < kBwdWarps; ++w) sum += s_acc[w][q];
      B.partials[int64_t(blockIdx.x) * NP + q] = sum;
    }
  }
}

// ------------------------------------------------------------------ dispatch
// Instantiations: polynomial inverse (FD = 0) at each packed AP/BP degree; Newton inverse
// (FD = 3 or 5, the padded A/B degree) with the AP/BP initial guess at runtime degree.
template <int ORDER>
static const void* tile_for_order(int ideg, int fd) {
  if (fd == 3) return reinterpret_cast<const void*>(&bwd_split_kernel<ORDER, -1, 3>);
  if (fd == 5) return reinterpret_cast<const void*>(&bwd_split_kernel<ORDER, -1, 5>);
  switch (ideg) {
    case 0: return reinterpret_cast<const void*>(&bwd_split_kernel<ORDER, 0, 0>);
    case 4: return reinterpret_cast<const void*>(&bwd_split_kernel<ORDER, 4, 0>);
    case 6: return reinterpret_cast<const void*>(&bwd_split_kernel<ORDER, 6, 0>);
    default: return reinterpret_cast<const void*>(&bwd_split_kernel<ORDER, 9, 0>);
  }
}

const void* backward_tile_kernel(int order, int ideg, int fd) {
  if (fd != 0 && fd != 3 && fd != 5) return nullptr;
  switch (order) {
    case DFR_NEAREST: return tile_for_order<DFR_NEAREST>(ideg, fd);
    case DFR_BILINEAR: return tile_for_order<DFR_BILINEAR>(ideg, fd);
    default: return tile_for_order<DFR_BICUBIC>(ideg, fd);
  }
}

DFR_DEFINE_STATUS_READER(read_and_clear_status_bwd_tile)

}  // namespace dfr
