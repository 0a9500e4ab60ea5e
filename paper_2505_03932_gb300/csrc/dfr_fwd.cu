// Forward reprojection kernels for sm_103a.
//
// One kernel per (interpolation order, inverse-SIP degree) does the whole per-pixel chain of
// dfreproject Sec. 3.1 steps 1-3 fused: coordinates in registers, the source tile staged into
// shared memory by a 2-D TMA load (or gathered straight from global memory), the footprint
// computed from the in-bounds weights, value and footprint stored coalesced.
//
// Work units: FP64 path, a 32x8 tile per CTA; split path, kCellsPerCta 32x32 anchor cells per
// CTA (one per warp). A CTA takes one unit (grid launch) or loops over units taken from an
// atomic counter (persistent batch launch); the per-pixel arithmetic depends only on the pixel
// and its cell, so both launch forms give equal bits.
#include <climits>

#include "dfr_fwd_kernels.cuh"

namespace dfr {

// Source positions exactly as the split kernels compute them (same anchors, same arithmetic),
// for the coordinate output of dfr_reproject; one thread per target pixel.
template <int IDEG>
__global__ void __launch_bounds__(256) split_coords_kernel(const __grid_constant__ FwdPlan P) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(P.w) * P.h) return;
  const int gx = int(i % P.w), gy = int(i / P.w);
  Anchor a;
  make_anchor(P, cell_anchor_x(P, gx), cell_anchor_y(P, gy), a);
  float x, y;
  const bool ok = split_coords_core<IDEG, false>(P, nullptr, P.identity != 0, P.tsip_deg > 0,
                                                 plan_newton(P), a, float(P.x0 + gx - a.ax),
                                                 float(P.y0 + gy - a.ay), x, y);
  double* c = P.coords + 2 * i;
  c[0] = ok ? double(a.bx) + double(x) : __longlong_as_double(0x7ff8000000000000ll);
  c[1] = ok ? double(a.by) + double(y) : __longlong_as_double(0x7ff8000000000000ll);
}

cudaError_t launch_split_coords(const FwdPlan& p0, cudaStream_t s) {
  const int64_t n = int64_t(p0.w) * p0.h;
  const int grid = int((n + 255) / 256);
  FwdPlan p = p0;
  void* args[] = {&p};
  const void* k;
  switch (p0.isip_deg) {
    case 0: k = reinterpret_cast<const void*>(&split_coords_kernel<0>); break;
    case 4: k = reinterpret_cast<const void*>(&split_coords_kernel<4>); break;
    case 6: k = reinterpret_cast<const void*>(&split_coords_kernel<6>); break;
    default: k = reinterpret_cast<const void*>(&split_coords_kernel<9>); break;
  }
  return cudaLaunchKernel(k, dim3(grid), dim3(256), args, 0, s);
}

// ------------------------------------------------------------------ dispatch
int forward_threads_default() { return kFp64Threads; }

template <int ORDER, bool BATCH>
static const void* split_for(int ideg) {
  switch (ideg) {
    case 0: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 0, BATCH, false>);
    case 4: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 4, BATCH, false>);
    case 6: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 6, BATCH, false>);
    default: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 9, BATCH, false>);
  }
}

template <int ORDER>
static const void* kernel_for_order(bool split, bool batch, int ideg) {
  if (!split) return reinterpret_cast<const void*>(&fwd_fp64_kernel<ORDER, kFp64Threads, false>);
  return batch ? split_for<ORDER, true>(ideg) : split_for<ORDER, false>(ideg);
}

// The kernel instantiation for a launch: order, flags and the packed inverse-SIP degree are
// uniform over a launch and taken from p0; batch launches read their plans from a table.
static const void* forward_kernel_for(const FwdPlan& p0, bool batch) {
  if (p0.flags & kFlagAccumulate) return batch ? nullptr : coadd_kernel(p0);
  const bool split = (p0.flags & DFR_SPLIT) != 0;
  if (split && !batch && p0.tsip_deg > 0) return tsip_kernel(p0);
  switch (p0.order) {
    case DFR_NEAREST: return kernel_for_order<DFR_NEAREST>(split, batch, p0.isip_deg);
    case DFR_BILINEAR: return kernel_for_order<DFR_BILINEAR>(split, batch, p0.isip_deg);
    case DFR_BICUBIC: return kernel_for_order<DFR_BICUBIC>(split, batch, p0.isip_deg);
    case DFR_LANCZOS3: return kernel_for_order<DFR_LANCZOS3>(split, batch, p0.isip_deg);
    default: return kernel_for_order<DFR_BSPLINE3>(split, batch, p0.isip_deg);
  }
}

const void* forward_kernel(const FwdPlan& p0) { return forward_kernel_for(p0, false); }

// Block size of the kernel that serves this plan.
static int block_threads(const FwdPlan& p0) {
  return (p0.flags & DFR_SPLIT) ? kWarps * 32 : kFp64Threads;
}

cudaError_t launch_forward(const FwdPlan& p0, const FwdLaunch& L, int grid, int threads,
                           int smem_bytes, cudaStream_t s) {
  (void)threads;
  threads = block_threads(p0);
  const void* k = forward_kernel_for(p0, L.plans != nullptr);
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
  (void)threads;
  threads = block_threads(p0);
  const void* k = forward_kernel_for(p0, true);
  if (smem_bytes > 0)
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, size_t(smem_bytes)) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

DFR_DEFINE_STATUS_READER(read_and_clear_status_fwd)

}  // namespace dfr
