// Tile-staged adjoint of the split-precision reprojection (dfr_reproject_backward), sm_103a.
//
// Work decomposition: kBwdCellsPerCta 32x64 cells per CTA, one per warp, each cell as 8 tiles
// of 32x8 (lane = column); source positions from the same cell fits as the forward kernels
// (bit for bit). Per tile the source box is
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

template <int ORDER, int IDEG, int FD>
__device__ __forceinline__ void bwd_tile_rows(const FwdPlan& P, const HP& Q, const BwdExtra& B,
                                              const ChainConst& K, const Anchor& a,
                                              const ColCubic& cc, int ox, int oy, int r0,
                                              int lane, const float* box, float* gbox,
                                              const TileBox& tb, bool want_params, float* acc) {
  using T = Taps<ORDER>;
  constexpr int NTERM = nterms(FD);
  const int gx = ox + lane;
  if (gx >= Q.w) return;
  const float xlo = -0.5f - float(a.bx), xhi = float(Q.W) - 0.5f - float(a.bx);
  const float ylo = -0.5f - float(a.by), yhi = float(Q.H) - 0.5f - float(a.by);
  const float dx0 = float(lane - kAnchorCol);
  const int bw = Q.box_w, bh = Q.box_h;
  const int nrows = min(kTileH, Q.h - oy);
#pragma unroll 1
  for (int r = 0; r < nrows; ++r) {
    float x, y, geo[4];
    const bool ok = pixel_coords(P, Q, a, cc, lane, r0 + r, x, y);
    if (want_params) {
      // the chain rule's intermediate offsets, from the exact per-pixel evaluation
      float xe, ye;
      split_coords_core<IDEG, false, FD>(P, nullptr, Q.identity, Q.tsip, Q.newton, a, dx0,
                                         float(r0 + r) - kCellMid, xe, ye, geo);
    }
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
    const float U = a.U0 + geo[0], V = a.V0 + geo[1];
    const float u = a.U0 + geo[2], v = a.V0 + geo[3];
    float lu, lv, c[6];
    chain_terms<IDEG, FD>(P, K, cov, Q.newton, gxs, gys, U, V, u, v, lu, lv, c);
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
        bwd_tile_rows<ORDER, IDEG, FD>(P, Q, B, K, a, cc, cox, oy, k * kTileH, lane, box, gbox,
                                       tb, want_params, acc);
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
