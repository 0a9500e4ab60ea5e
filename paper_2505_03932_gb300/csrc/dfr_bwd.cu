// Adjoint of the reprojection (dfr_reproject_backward), sm_103a.
//
// For value = N / F with N = sum_k w_k S_k and F = sum_k w_k over in-bounds taps (Sec. 3.1
// footprint normalisation), per covered target pixel with output gradient g:
//   dL/dS_k  += g w_k / F                                  (scatter, global atomics)
//   dL/dx_s   = g / F * sum_k (dw_k/dx_s) (S_k - value)    (and likewise y)
// and the source-WCS parameter gradients follow by the chain rule through the inverse SIP
// (polynomial AP/BP, or the implicit-function derivative of the Newton inverse of A/B), CD^-1
// and the gnomonic projection about (CRVAL1, CRVAL2). Per-pixel terms are FP32; each warp sums
// them with shuffles and adds the warp total to an FP64 shared accumulator; each CTA writes
// one FP64 partial per parameter and a final single-block kernel adds the partials in a fixed
// order (deterministic parameter gradients).
//
// This file holds the per-pixel kernel (FP64 path, and split plans the tile-staged kernel of
// dfr_bwd_tile.cu does not serve), the final sum and the dispatch between the two.
#include <climits>

#include "dfr_adjoint.cuh"
#include "dfr_tile.cuh"

namespace dfr {

constexpr int kBwdThreads = 256;
constexpr float kBelowOne = 0.99999994f;  // the largest float below 1 (1 - 2^-24)

// FP64 geometry of one target pixel: source position, intermediate offsets before (U, V) and
// after (u, v) the inverse SIP. Same arithmetic as the forward FP64 path.
__device__ __forceinline__ bool fp64_geo(const FwdPlan& P, double X, double Y, double& xs,
                                         double& ys, double& U, double& V, double& u, double& v) {
  if (P.identity) {
    xs = X + P.shift[0];
    ys = Y + P.shift[1];
    U = u = X - P.crpix_t[0];
    V = v = Y - P.crpix_t[1];
    return true;
  }
  double ra, dec;
  world_from_target_fp64(P, X, Y, ra, dec);
  const bool ok = intermediate_from_world_fp64(P, ra, dec, U, V);
  u = U;
  v = V;
  if (P.isip_deg > 0) {
    double ga, gb;
    horner_pair_rt<double>(P.isip_d[0], P.isip_d[1], P.isip_deg, U, V, ga, gb);
    u = U + ga;
    v = V + gb;
  }
  if ((P.flags & DFR_EXACT_INVERSE) && P.fsip_deg > 0) newton_fp64(P, U, V, u, v);
  xs = u + P.crpix_s[0];
  ys = v + P.crpix_s[1];
  return ok;
}

template <int ORDER, int FD>
__global__ void __launch_bounds__(kBwdThreads) bwd_kernel(const __grid_constant__ FwdPlan P,
                                                          const __grid_constant__ BwdExtra B) {
  using T = Taps<ORDER>;
  constexpr int NT = kBwdThreads, NW = NT / 32, PPT = kTilePix / NT;
  constexpr int NTERM = nterms(FD);
  constexpr int NP = 6 + 2 * NTERM;
  __shared__ double sacc[NW][NP];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < NW * NP; i += NT) sacc[i / NP][i % NP] = 0.0;
  const bool split = (P.flags & DFR_SPLIT) != 0;
  const bool exact = (P.flags & DFR_EXACT_INVERSE) && P.fsip_deg > 0;
  const bool want_params = B.grad_params != nullptr && ORDER != DFR_NEAREST;
  const int ntiles = P.tiles_x * P.tiles_y;
  const ChainConst K = chain_const(P);
  __syncthreads();

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ox = (tile % P.tiles_x) * kTileW, oy = (tile / P.tiles_x) * kTileH;
#pragma unroll 1
    for (int k = 0; k < PPT; ++k) {
      const int i = tid + k * NT;
      const int gx = ox + (i % kTileW), gy = oy + (i / kTileW);
      const bool inside = gx < P.w && gy < P.h;
      // split plans: the warp (one tile row, 32 columns of one cell) fits the cell, as the
      // forward kernels do
      Anchor a;
      ColCubic cc;
      HP Q;
      if (split) {
        load_hot(P, Q);
        cc = cell_fit<false, true>(P, Q, ox, gy - gy % kCellH, lane, a);
      }
      bool cov = false;
      int bx = 0, by = 0;
      float xr = 0.f, yr = 0.f, U = 0.f, V = 0.f, u = 0.f, v = 0.f;
      if (inside) {
        if (split) {
          // position from the cell fit of the forward kernels (same bits); the chain rule's
          // intermediate offsets from the exact per-pixel evaluation
          const int row = gy % kCellH;
          const bool ok = pixel_coords(P, Q, a, cc, lane, row, xr, yr);
          float geo[4], xe, ye;
          split_coords<-1>(P, a, float(lane - kAnchorCol), float(row) - kCellMid, xe, ye, geo);
          bx = a.bx;
          by = a.by;
          cov = ok && xr >= -0.5f - float(bx) && xr <= float(P.W) - 0.5f - float(bx) &&
                yr >= -0.5f - float(by) && yr <= float(P.H) - 0.5f - float(by);
          U = a.U0 + geo[0];
          V = a.V0 + geo[1];
          u = a.U0 + geo[2];
          v = a.V0 + geo[3];
        } else {
          double xs, ys, Ud, Vd, ud, vd;
          const bool ok = fp64_geo(P, double(P.x0 + gx), double(P.y0 + gy), xs, ys, Ud, Vd, ud, vd);
          const double rx = rint(xs), ry = rint(ys);
          if (fabs(xs - rx) < kSnap) xs = rx;
          if (fabs(ys - ry) < kSnap) ys = ry;
          cov = ok && xs >= -0.5 && xs <= P.W - 0.5 && ys >= -0.5 && ys <= P.H - 0.5;
          if (cov) {
            const double fx = floor(xs), fy = floor(ys);
            bx = int(fx);
            by = int(fy);
            // fractions rounded to FP32 stay below 1, so the taps (and the one-sided slope of
            // the interpolant) are those of the FP64 floor
            xr = fminf(float(xs - fx), kBelowOne);
            yr = fminf(float(ys - fy), kBelowOne);
          }
          U = float(Ud);
          V = float(Vd);
          u = float(ud);
          v = float(vd);
        }
      }
      float gxs = 0.f, gys = 0.f;  // dL/dx_s, dL/dy_s
      if (cov) {
        const float flx = floorf(xr), fly = floorf(yr);
        const float tx = xr - flx, ty = yr - fly;
        int ix = int(flx), iy = int(fly);
        if (ORDER == DFR_NEAREST) {
          ix += tx >= 0.5f;
          iy += ty >= 0.5f;
        }
        ix += bx + T::lo;
        iy += by + T::lo;
        float wx[T::n], wy[T::n], dx[T::n], dy[T::n], s[T::n][T::n];
        weights<ORDER, float>(tx, wx);
        weights<ORDER, float>(ty, wy);
        dweights<ORDER, float>(tx, dx);
        dweights<ORDER, float>(ty, dy);
        float sx = 0.f, sy = 0.f;
#pragma unroll
        for (int q = 0; q < T::n; ++q) {
          const bool inx = unsigned(ix + q) < unsigned(P.W);
          const bool iny = unsigned(iy + q) < unsigned(P.H);
          wx[q] = inx ? wx[q] : 0.f;
          dx[q] = inx ? dx[q] : 0.f;
          wy[q] = iny ? wy[q] : 0.f;
          dy[q] = iny ? dy[q] : 0.f;
          sx += wx[q];
          sy += wy[q];
        }
        float num = 0.f;
#pragma unroll
        for (int r = 0; r < T::n; ++r) {
          const bool iny = unsigned(iy + r) < unsigned(P.H);
          float row = 0.f;
#pragma unroll
          for (int q = 0; q < T::n; ++q) {
            const bool in = iny && unsigned(ix + q) < unsigned(P.W);
            s[r][q] = in ? __ldg(P.img + int64_t(iy + r) * P.pitch + (ix + q)) : 0.f;
            row = fmaf(wx[q], s[r][q], row);
          }
          num = fmaf(wy[r], row, num);
        }
        const float F = sx * sy;
        if (F != 0.f) {
          const float g = B.grad_out[int64_t(gy) * B.go_pitch + gx];
          const float gF = __fdividef(g, F);
          if (B.grad_src) {
#pragma unroll
            for (int r = 0; r < T::n; ++r)
#pragma unroll
              for (int q = 0; q < T::n; ++q) {
                const float w = wx[q] * wy[r];
                if (w != 0.f)
                  atomicAdd(B.grad_src + int64_t(iy + r) * B.gs_pitch + (ix + q), gF * w);
              }
          }
          if (want_params) {
            const float val = __fdividef(num, F);
            float ax_ = 0.f, ay_ = 0.f;
#pragma unroll
            for (int r = 0; r < T::n; ++r)
#pragma unroll
              for (int q = 0; q < T::n; ++q) {
                const float d = s[r][q] - val;
                ax_ = fmaf(dx[q] * wy[r], d, ax_);
                ay_ = fmaf(wx[q] * dy[r], d, ay_);
              }
            gxs = gF * ax_;
            gys = gF * ay_;
          }
        }
      }
      if (!want_params) continue;  // uniform over the launch
      float lu, lv, c[6];
      chain_terms<-1, -1>(P, K, cov, exact, gxs, gys, U, V, u, v, lu, lv, c);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float t = warp_sum(c[q]);
        if (lane == 0) sacc[warp][q] += double(t);
      }
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
            const float ta = warp_sum(-lu * m);
            const float tb = warp_sum(-lv * m);
            if (lane == 0) {
              sacc[warp][6 + t] += double(ta);
              sacc[warp][6 + NTERM + t] += double(tb);
            }
          }
      }
    }
  }
  __syncthreads();  // every warp's accumulators are final
  if (B.partials) {
    for (int q = tid; q < NP; q += NT) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) s += sacc[w][q];
      B.partials[int64_t(blockIdx.x) * NP + q] = s;
    }
  }
}

// Sum the per-CTA partials in a fixed order and scatter them to the public layout.
__global__ void bwd_finalize(const __grid_constant__ BwdExtra B, int np) {
  for (int j = threadIdx.x; j < B.nout; j += blockDim.x) B.grad_params[j] = 0.0;
  __syncthreads();
  for (int q = threadIdx.x; q < np; q += blockDim.x) {
    const int dst = B.pmap[q];
    if (dst < 0) continue;
    double s = 0.0;
    for (int b = 0; b < B.grid; ++b) s += B.partials[int64_t(b) * np + q];
    B.grad_params[dst] = s;
  }
}

int backward_num_padded(int fd) { return 6 + 2 * nterms(fd); }

template <int ORDER>
static const void* bwd_for_order(int fd) {
  switch (fd) {
    case 0: return reinterpret_cast<const void*>(&bwd_kernel<ORDER, 0>);
    case 3: return reinterpret_cast<const void*>(&bwd_kernel<ORDER, 3>);
    case 5: return reinterpret_cast<const void*>(&bwd_kernel<ORDER, 5>);
    default: return reinterpret_cast<const void*>(&bwd_kernel<ORDER, 9>);
  }
}

// The tile-staged kernel serves split-precision plans with a TMA-capable source and exact-inverse
// degree <= 5 (its per-lane accumulators: 6 + 2 * 20 registers); the per-pixel kernel serves
// the rest (FP64 path, degree 9, sources without a tensor map).
static bool staged(const FwdPlan& p0, int fd) {
  return (p0.flags & DFR_SPLIT) && p0.use_tma && !p0.stage_sw && fd <= 5 &&
         p0.order != DFR_LANCZOS3;
}

static const void* bwd_kernel_for(const FwdPlan& p0, int fd) {
  if (staged(p0, fd)) return backward_tile_kernel(p0.order, p0.isip_deg, fd);
  switch (p0.order) {
    case DFR_NEAREST: return bwd_for_order<DFR_NEAREST>(fd);
    case DFR_BILINEAR: return bwd_for_order<DFR_BILINEAR>(fd);
    case DFR_LANCZOS3: return bwd_for_order<DFR_LANCZOS3>(fd);
    default: return bwd_for_order<DFR_BICUBIC>(fd);
  }
}

int backward_threads_for(const FwdPlan& p0, int fd) {
  return staged(p0, fd) ? kBwdWarps * 32 : kBwdThreads;
}

// Dynamic shared memory: per warp a source box and a gradient box, plus alignment slack.
int backward_smem_bytes(const FwdPlan& p0, int fd, int box_floats) {
  return staged(p0, fd) ? kBwdWarps * 2 * box_floats * 4 + 128 : 0;
}

int backward_max_blocks_per_sm(const FwdPlan& p0, int fd, int smem_bytes) {
  const void* k = bwd_kernel_for(p0, fd);
  if (smem_bytes > 0)
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, backward_threads_for(p0, fd),
                                                    size_t(smem_bytes)) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

cudaError_t launch_backward(const FwdPlan& p0, const BwdExtra& B, cudaStream_t s) {
  FwdPlan p = p0;
  BwdExtra b = B;
  void* args[] = {&p, &b};
  const void* k = bwd_kernel_for(p0, B.fd);
  const int smem = backward_smem_bytes(p0, B.fd, B.box_floats);
  if (smem > 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaLaunchKernel(k, dim3(B.grid), dim3(backward_threads_for(p0, B.fd)), args,
                                   size_t(smem), s);
  if (e != cudaSuccess || B.grad_params == nullptr) return e;
  int np = backward_num_padded(B.fd);
  void* fargs[] = {&b, &np};
  return cudaLaunchKernel(reinterpret_cast<const void*>(&bwd_finalize), dim3(1), dim3(128),
                          fargs, 0, s);
}

DFR_DEFINE_STATUS_READER(read_and_clear_status_bwd)

}  // namespace dfr
