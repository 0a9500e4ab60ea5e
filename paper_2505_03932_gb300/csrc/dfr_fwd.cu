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

// ------------------------------------------------------------------ split-precision tiles
// One warp owns a 32x8 tile: lane = column, 8 rows per lane. Per tile: source positions of the
// 256 pixels (FP32, from the tile's FP64 anchor), warp min/max of their integer parts, one TMA
// load of the covering source box into the warp's shared buffer, then the gather. Tiles are
// double-buffered: the box of tile t+1 is in flight while tile t is gathered.
struct TileCoords {
  float x[kTileH], y[kTileH];  // source position relative to (bx, by)
  uint32_t mask;               // covered rows of this lane
  int32_t bx, by;              // anchor base
  int32_t bx0, by0;            // box origin (absolute source pixel)
  bool use_box;
};

template <int ORDER, int IDEG>
__device__ __forceinline__ void split_prepare(const FwdPlan& P, const Anchor& a, int local,
                                              int lane, float* box, uint64_t* bar,
                                              TileCoords& C) {
  using T = Taps<ORDER>;
  const int ox = (local % P.tiles_x) * kTileW, oy = (local / P.tiles_x) * kTileH;
  const int gx = ox + lane;
  const float xlo = -0.5f - float(a.bx), xhi = float(P.W) - 0.5f - float(a.bx);
  const float ylo = -0.5f - float(a.by), yhi = float(P.H) - 0.5f - float(a.by);
  int mnx = INT_MAX, mxx = INT_MIN, mny = INT_MAX, mxy = INT_MIN;
  C.mask = 0;
  C.bx = a.bx;
  C.by = a.by;
  const float dx = float(P.x0 + gx - a.ax);
#pragma unroll
  for (int r = 0; r < kTileH; ++r) {
    const int gy = oy + r;
    const bool inside = gx < P.w && gy < P.h;
    float x, y;
    const bool ok = split_coords<IDEG>(P, a, dx, float(P.y0 + gy - a.ay), x, y);
    C.x[r] = x;
    C.y[r] = y;
    if (inside && ok && x >= xlo && x <= xhi && y >= ylo && y <= yhi) {
      C.mask |= 1u << r;
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
  // coverage and source extent of the tile: warp-level reductions
  const bool any = __ballot_sync(0xffffffffu, C.mask != 0) != 0;
  C.use_box = false;
  C.bx0 = C.by0 = 0;
  if (any && P.use_tma) {
    mnx = __reduce_min_sync(0xffffffffu, mnx);
    mxx = __reduce_max_sync(0xffffffffu, mxx);
    mny = __reduce_min_sync(0xffffffffu, mny);
    mxy = __reduce_max_sync(0xffffffffu, mxy);
    C.bx0 = (a.bx + mnx + T::lo) & ~3;  // TMA x must be a multiple of 16 bytes
    C.by0 = a.by + mny + T::lo;
    // nearest may step one pixel up from floor(x), so its extent is two taps wide
    constexpr int ext = (ORDER == DFR_NEAREST) ? 2 : T::n;
    C.use_box = (a.bx + mxx + T::lo + ext - C.bx0 <= P.box_w) &&
                (a.by + mxy + T::lo + ext - C.by0 <= P.box_h);
  }
  if (C.use_box) {
    __syncwarp();  // every lane is done reading this buffer's previous tile
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar, uint32_t(P.box_w) * uint32_t(P.box_h) * 4u);
      tma_load_2d(box, &P.tmap, bar, C.bx0, C.by0);
    }
  }
}

template <int ORDER>
__device__ __forceinline__ void split_consume(const FwdPlan& P, int local, int lane,
                                              const float* box, uint64_t* bar, uint32_t& phase,
                                              const TileCoords& C) {
  using T = Taps<ORDER>;
  const int ox = (local % P.tiles_x) * kTileW, oy = (local / P.tiles_x) * kTileH;
  const int gx = ox + lane;
  bool use_box = C.use_box;
  if (use_box) {
    if (!mbar_wait(bar, phase)) use_box = false;  // timed out: gather from global instead
    phase ^= 1u;
  }
  if (gx >= P.w) return;
#pragma unroll
  for (int r = 0; r < kTileH; ++r) {
    const int gy = oy + r;
    if (gy >= P.h) break;
    float val = 0.f, fpv = 0.f;
    if (C.mask & (1u << r)) {
      const float x = C.x[r], y = C.y[r];
      const float flx = floorf(x), fly = floorf(y);
      const float tx = x - flx, ty = y - fly;
      int ix = int(flx), iy = int(fly);
      if (ORDER == DFR_NEAREST) {
        ix += tx >= 0.5f;
        iy += ty >= 0.5f;
      }
      ix += C.bx + T::lo;  // absolute source column / row of the first tap
      iy += C.by + T::lo;
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
        const float* b = box + (iy - C.by0) * P.box_w + (ix - C.bx0);
#pragma unroll
        for (int k = 0; k < T::n; ++k) {
          float row = 0.f;
#pragma unroll
          for (int q = 0; q < T::n; ++q) row = fmaf(wx[q], b[k * P.box_w + q], row);
          num = fmaf(wy[k], row, num);
        }
      } else {
#pragma unroll
        for (int k = 0; k < T::n; ++k) {
          float row = 0.f;
          const bool iny = unsigned(iy + k) < unsigned(P.H);
#pragma unroll
          for (int q = 0; q < T::n; ++q) {
            const bool in = iny && unsigned(ix + q) < unsigned(P.W);
            const float s = in ? __ldg(P.img + int64_t(iy + k) * P.pitch + (ix + q)) : 0.f;
            row = fmaf(wx[q], s, row);
          }
          num = fmaf(wy[k], row, num);
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

__device__ __forceinline__ int frame_of(const FwdLaunch& L, int t) {
  int lo = 0, hi = L.nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int ORDER, int IDEG>
__global__ void __launch_bounds__(kWarps * 32) fwd_split_kernel(const __grid_constant__ FwdPlan p0,
                                                                const FwdLaunch L) {
  extern __shared__ __align__(128) float box_raw[];
  __shared__ Anchor s_anc[kWarps][kChunk];
  __shared__ int32_t s_frame[kWarps][kChunk];
  __shared__ int32_t s_local[kWarps][kChunk];
  __shared__ __align__(8) uint64_t s_bar[kWarps][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // two 128-byte aligned source-box buffers per warp (the launch reserves 128 bytes of slack)
  float* box0 = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(box_raw) + 127) &
                                         ~uintptr_t(127)) + warp * 2 * L.box_floats;
  float* box1 = box0 + L.box_floats;
  uint64_t* bar0 = &s_bar[warp][0];
  uint64_t* bar1 = &s_bar[warp][1];
  if (lane == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
  }
  __syncwarp();
  uint32_t ph0 = 0, ph1 = 0;
  const bool batch = L.plans != nullptr;
  const int total = batch ? L.tile_start[L.nframes] : L.total_tiles;
  const int nchunks = (total + kChunk - 1) / kChunk;
  const int stride = gridDim.x * kWarps;
  int chunk = blockIdx.x * kWarps + warp;
  if (batch) {
    int c = 0;
    if (lane == 0) c = atomicAdd(L.counter, 1);
    chunk = __shfl_sync(0xffffffffu, c, 0);
  }
  while (chunk < nchunks) {
    const int t0 = chunk * kChunk;
    const int nt = min(kChunk, total - t0);
    if (lane < nt) {  // FP64 anchors of the chunk's tiles, one per lane
      int f = 0, local = t0 + lane;
      if (batch) {
        f = frame_of(L, local);
        local -= L.tile_start[f];
      }
      const FwdPlan& P = batch ? L.plans[f] : p0;
      const int ox = (local % P.tiles_x) * kTileW, oy = (local / P.tiles_x) * kTileH;
      make_anchor(P, P.x0 + ox + kTileW / 2, P.y0 + oy + kTileH / 2, s_anc[warp][lane]);
      s_frame[warp][lane] = f;
      s_local[warp][lane] = local;
    }
    __syncwarp();
    TileCoords CA, CB;
    {
      const FwdPlan& P = batch ? L.plans[s_frame[warp][0]] : p0;
      split_prepare<ORDER, IDEG>(P, s_anc[warp][0], s_local[warp][0], lane, box0, bar0, CA);
    }
    for (int t = 0; t < nt; t += 2) {
      const FwdPlan& Pa = batch ? L.plans[s_frame[warp][t]] : p0;
      if (t + 1 < nt) {
        const FwdPlan& Pb = batch ? L.plans[s_frame[warp][t + 1]] : p0;
        split_prepare<ORDER, IDEG>(Pb, s_anc[warp][t + 1], s_local[warp][t + 1], lane, box1, bar1,
                                   CB);
      }
      split_consume<ORDER>(Pa, s_local[warp][t], lane, box0, bar0, ph0, CA);
      if (t + 1 < nt) {
        if (t + 2 < nt) {
          const FwdPlan& Pc = batch ? L.plans[s_frame[warp][t + 2]] : p0;
          split_prepare<ORDER, IDEG>(Pc, s_anc[warp][t + 2], s_local[warp][t + 2], lane, box0,
                                     bar0, CA);
        }
        const FwdPlan& Pb = batch ? L.plans[s_frame[warp][t + 1]] : p0;
        split_consume<ORDER>(Pb, s_local[warp][t + 1], lane, box1, bar1, ph1, CB);
      }
    }
    __syncwarp();  // anchors of this chunk are no longer read
    if (batch) {
      int c = 0;
      if (lane == 0) c = atomicAdd(L.counter, 1);
      chunk = __shfl_sync(0xffffffffu, c, 0);
    } else {
      chunk += stride;
    }
  }
}

// ------------------------------------------------------------------ dispatch
constexpr int kThreads = 256;
int forward_threads_default() { return kThreads; }

template <int ORDER>
static const void* kernel_for_order(bool split, int ideg) {
  if (!split) return reinterpret_cast<const void*>(&fwd_fp64_kernel<ORDER, kThreads>);
  switch (ideg) {
    case 0: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 0>);
    case 4: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 4>);
    case 6: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 6>);
    default: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 9>);
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
  if (smem_bytes > 0) {
    // static + dynamic shared memory may exceed the default 48 KB window
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
  if (smem_bytes > 0)
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
