// Forward reprojection kernels for sm_103a.
//
// One kernel per (interpolation order, inverse-SIP degree) does the whole per-pixel chain of
// dfreproject Sec. 3.1 steps 1-3 fused: coordinates in registers, the source tile staged into
// shared memory by a 2-D TMA load (or gathered straight from global memory), the footprint
// computed from the in-bounds weights, value and footprint stored coalesced.
//
// Work unit: a 64x16 tile of the target bounding box. A CTA takes one tile (grid launch) or
// loops over tiles taken from an atomic counter (persistent batch launch); the per-pixel
// arithmetic depends only on the pixel and its tile, so both launch forms give equal bits.
#include <climits>

#include "dfr_device.cuh"

namespace dfr {

// ------------------------------------------------------------------ FP64 tile (plain method)
// Per pixel: the printed formulas in FP64, direct gather, FP64 weights and sums.
template <int ORDER, int NT>
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
      double num = 0.0, sx = 0.0, sy = 0.0;
#pragma unroll
      for (int a = 0; a < T::n; ++a) {
        if (ix + a < 0 || ix + a >= P.W) wx[a] = 0.0;
        if (iy + a < 0 || iy + a >= P.H) wy[a] = 0.0;
        sx += wx[a];
        sy += wy[a];
      }
#pragma unroll
      for (int b = 0; b < T::n; ++b) {
        double row = 0.0;
        const int yy = iy + b;
        if (wy[b] != 0.0) {
#pragma unroll
          for (int a = 0; a < T::n; ++a) {
            const int xx = ix + a;
            if (wx[a] != 0.0) row += wx[a] * double(__ldg(P.img + int64_t(yy) * P.pitch + xx));
          }
        }
        num += wy[b] * row;
      }
      const double f = sx * sy;
      if (f != 0.0) {
        val = float(num / f);
        fpv = float(f);
      }
    }
    P.out[o] = val;
    if (P.fp) P.fp[o] = fpv;
  }
}

// ------------------------------------------------------------------ split-precision tile
struct TileShared {
  Anchor anc;
  int32_t red[5];  // min fx, max fx, min fy, max fy, any covered
};

template <int ORDER, int IDEG, int NT>
__device__ __forceinline__ void split_tile(const FwdPlan& P, int tile, float* box, uint64_t* bar,
                                           uint32_t& phase, TileShared& sh) {
  using T = Taps<ORDER>;
  constexpr int PPT = kTilePix / NT;
  const int tid = threadIdx.x;
  const int ox = (tile % P.tiles_x) * kTileW, oy = (tile / P.tiles_x) * kTileH;
  const int ax = P.x0 + ox + kTileW / 2, ay = P.y0 + oy + kTileH / 2;

  if (tid == 0) {
    make_anchor(P, ax, ay, sh.anc);
    sh.red[0] = INT_MAX;
    sh.red[1] = INT_MIN;
    sh.red[2] = INT_MAX;
    sh.red[3] = INT_MIN;
    sh.red[4] = 0;
  }
  __syncthreads();
  const Anchor a = sh.anc;

  float xr[PPT], yr[PPT];
  uint32_t covmask = 0;
  int mnx = INT_MAX, mxx = INT_MIN, mny = INT_MAX, mxy = INT_MIN;
  const float xlo = -0.5f - float(a.bx), xhi = float(P.W) - 0.5f - float(a.bx);
  const float ylo = -0.5f - float(a.by), yhi = float(P.H) - 0.5f - float(a.by);
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int i = tid + k * NT;
    const int lx = i % kTileW, ly = i / kTileW;
    const int gx = ox + lx, gy = oy + ly;
    const bool inside = gx < P.w && gy < P.h;
    float x, y;
    const bool ok = split_coords<IDEG>(P, a, float(ox + lx + P.x0 - ax), float(oy + ly + P.y0 - ay),
                                       x, y);
    xr[k] = x;
    yr[k] = y;
    const bool cov = inside && ok && x >= xlo && x <= xhi && y >= ylo && y <= yhi;
    if (cov) {
      covmask |= 1u << k;
      const int fx = int(floorf(x)), fy = int(floorf(y));
      mnx = min(mnx, fx);
      mxx = max(mxx, fx);
      mny = min(mny, fy);
      mxy = max(mxy, fy);
    }
    if (P.coords && inside) {
      double* c = P.coords + 2 * (int64_t(gy) * P.w + gx);
      c[0] = ok ? double(a.bx) + double(x) : __longlong_as_double(0x7ff8000000000000ll);
      c[1] = ok ? double(a.by) + double(y) : __longlong_as_double(0x7ff8000000000000ll);
    }
  }
  // coverage and source-extent reduction: warp shuffles, then one shared atomic per warp
  const unsigned any = __ballot_sync(0xffffffffu, covmask != 0);
  if (any) {
    mnx = __reduce_min_sync(0xffffffffu, mnx);
    mxx = __reduce_max_sync(0xffffffffu, mxx);
    mny = __reduce_min_sync(0xffffffffu, mny);
    mxy = __reduce_max_sync(0xffffffffu, mxy);
    if ((tid & 31) == 0) {
      atomicMin(&sh.red[0], mnx);
      atomicMax(&sh.red[1], mxx);
      atomicMin(&sh.red[2], mny);
      atomicMax(&sh.red[3], mxy);
      atomicOr(&sh.red[4], 1);
    }
  }
  __syncthreads();
  const bool tile_any = sh.red[4] != 0;
  int bx0 = 0, by0 = 0;
  bool use_box = false;
  if (tile_any && P.use_tma) {
    bx0 = (a.bx + sh.red[0] + T::lo) & ~3;  // TMA x must be a multiple of 16 bytes
    by0 = a.by + sh.red[2] + T::lo;
    // nearest may step one pixel up from floor(x), so its extent is two taps wide
    constexpr int ext = (ORDER == DFR_NEAREST) ? 2 : T::n;
    const int need_w = a.bx + sh.red[1] + T::lo + ext - bx0;
    const int need_h = a.by + sh.red[3] + T::lo + ext - by0;
    use_box = need_w <= P.box_w && need_h <= P.box_h;
  }
  if (use_box) {
    if (tid == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar, uint32_t(P.box_w) * uint32_t(P.box_h) * 4u);
      tma_load_2d(box, &P.tmap, bar, bx0, by0);
    }
    if (!mbar_wait(bar, phase)) use_box = false;  // timed out: gather from global instead
    phase ^= 1u;
  }

#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int i = tid + k * NT;
    const int gx = ox + (i % kTileW), gy = oy + (i / kTileW);
    if (gx >= P.w || gy >= P.h) continue;
    float val = 0.f, fpv = 0.f;
    if (covmask & (1u << k)) {
      const float x = xr[k], y = yr[k];
      const float flx = floorf(x), fly = floorf(y);
      const float tx = x - flx, ty = y - fly;
      int ix = int(flx), iy = int(fly);
      if (ORDER == DFR_NEAREST) {
        ix += tx >= 0.5f;
        iy += ty >= 0.5f;
      }
      ix += a.bx + T::lo;  // absolute source column of the first tap
      iy += a.by + T::lo;
      float wx[T::n], wy[T::n];
      weights<ORDER, float>(tx, wx);
      weights<ORDER, float>(ty, wy);
      float sx = 0.f, sy = 0.f;
#pragma unroll
      for (int q = 0; q < T::n; ++q) {
        wx[q] = (unsigned(ix + q) < unsigned(P.W)) ? wx[q] : 0.f;
        wy[q] = (unsigned(iy + q) < unsigned(P.H)) ? wy[q] : 0.f;
        sx += wx[q];
        sy += wy[q];
      }
      float num = 0.f;
      if (use_box) {
        const float* b = box + (iy - by0) * P.box_w + (ix - bx0);
#pragma unroll
        for (int r = 0; r < T::n; ++r) {
          float row = 0.f;
#pragma unroll
          for (int q = 0; q < T::n; ++q) row = fmaf(wx[q], b[r * P.box_w + q], row);
          num = fmaf(wy[r], row, num);
        }
      } else {
#pragma unroll
        for (int r = 0; r < T::n; ++r) {
          float row = 0.f;
          const bool iny = unsigned(iy + r) < unsigned(P.H);
#pragma unroll
          for (int q = 0; q < T::n; ++q) {
            const bool in = iny && unsigned(ix + q) < unsigned(P.W);
            const float s = in ? __ldg(P.img + int64_t(iy + r) * P.pitch + (ix + q)) : 0.f;
            row = fmaf(wx[q], s, row);
          }
          num = fmaf(wy[r], row, num);
        }
      }
      const float f = sx * sy;
      if (f != 0.f) {
        val = (f == 1.f) ? num : __fdividef(num, f);
        fpv = f;
      }
    }
    const int64_t o = int64_t(gy) * P.out_pitch + gx;
    __stcs(P.out + o, val);
    if (P.fp) __stcs(P.fp + o, fpv);
  }
  __syncthreads();  // the box and the shared anchor are reused by the next tile
}

// ------------------------------------------------------------------ kernels
template <int ORDER, int NT>
__global__ void __launch_bounds__(NT) fwd_fp64_kernel(const __grid_constant__ FwdPlan p0,
                                                      const FwdLaunch L) {
  if (L.plans == nullptr) {
    fp64_tile<ORDER, NT>(p0, blockIdx.x);
    return;
  }
  __shared__ int32_t s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(L.counter, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= L.tile_start[L.nframes]) break;
    int lo = 0, hi = L.nframes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (L.tile_start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    fp64_tile<ORDER, NT>(L.plans[lo], t - L.tile_start[lo]);
  }
}

template <int ORDER, int IDEG, int NT>
__global__ void __launch_bounds__(NT) fwd_split_kernel(const __grid_constant__ FwdPlan p0,
                                                       const FwdLaunch L) {
  extern __shared__ __align__(128) float box_raw[];
  // TMA destinations are kept 128-byte aligned (the launch reserves 128 bytes of slack)
  float* box = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(box_raw) + 127) &
                                        ~uintptr_t(127));
  __shared__ __align__(8) uint64_t bar;
  __shared__ TileShared sh;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  if (L.plans == nullptr) {
    split_tile<ORDER, IDEG, NT>(p0, blockIdx.x, box, &bar, phase, sh);
    return;
  }
  __shared__ int32_t s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(L.counter, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= L.tile_start[L.nframes]) break;
    int lo = 0, hi = L.nframes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (L.tile_start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    split_tile<ORDER, IDEG, NT>(L.plans[lo], t - L.tile_start[lo], box, &bar, phase, sh);
  }
}

// ------------------------------------------------------------------ dispatch
constexpr int kThreads = 256;
int forward_threads_default() { return kThreads; }

template <int ORDER>
static const void* kernel_for_order(bool split, int ideg) {
  if (!split) return reinterpret_cast<const void*>(&fwd_fp64_kernel<ORDER, kThreads>);
  switch (ideg) {
    case 0: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 0, kThreads>);
    case 4: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 4, kThreads>);
    case 6: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 6, kThreads>);
    default: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 9, kThreads>);
  }
}

// The kernel instantiation for a launch: order, flags and the packed inverse-SIP degree are
// uniform over a launch and taken from p0.
const void* forward_kernel(const FwdPlan& p0) {
  const bool split = (p0.flags & DFR_SPLIT) != 0;
  switch (p0.order) {
    case DFR_NEAREST: return kernel_for_order<DFR_NEAREST>(split, p0.isip_deg);
    case DFR_BILINEAR: return kernel_for_order<DFR_BILINEAR>(split, p0.isip_deg);
    default: return kernel_for_order<DFR_BICUBIC>(split, p0.isip_deg);
  }
}

cudaError_t launch_forward(const FwdPlan& p0, const FwdLaunch& L, int grid, int threads,
                           int smem_bytes, cudaStream_t s) {
  const void* k = forward_kernel(p0);
  if (smem_bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
    if (e != cudaSuccess) return e;
  }
  FwdPlan p = p0;
  FwdLaunch l = L;
  void* args[] = {&p, &l};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, size_t(smem_bytes), s);
}

int forward_max_blocks_per_sm(const FwdPlan& p0, int threads, int smem_bytes) {
  const void* k = forward_kernel(p0);
  if (smem_bytes > 48 * 1024)
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, size_t(smem_bytes)) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

cudaError_t read_and_clear_status_fwd(int32_t* out, cudaStream_t s) {
  int32_t zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_status, sizeof(int32_t), 0,
                                            cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (*out != 0) e = cudaMemcpyToSymbol(g_status, &zero, sizeof(int32_t));
  return e;
}

}  // namespace dfr
