// Forward reprojection kernels for sm_103a.
//
// One kernel per (interpolation order, inverse-SIP degree) does the whole per-pixel chain of
// dfreproject Sec. 3.1 steps 1-3 fused: coordinates in registers, the source tile staged into
// shared memory by a 2-D TMA load (or gathered straight from global memory), the footprint
// computed from the in-bounds weights, value and footprint stored coalesced.
//
// Work units: FP64 path, a 32x8 tile per CTA; split path, a 32x64 cell per one-warp CTA. A
// split CTA takes one unit (one frame, or a cell of a frame table); the FP64 batch kernel loops
// over tiles taken from an atomic counter (a persistent grid). The per-pixel arithmetic
// depends only on the pixel and its cell, so every launch form gives equal bits.
#include <climits>

#include "dfr_fwd_kernels.cuh"

namespace dfr {

// Source positions exactly as the split kernels compute them (same cell fits), for the
// coordinate output of dfr_reproject; one warp per cell (lane = column).
__global__ void __launch_bounds__(32) split_coords_kernel(const __grid_constant__ FwdPlan P) {
  const int cell = blockIdx.x, lane = threadIdx.x & 31;
  const int cox = (cell % P.cells_x) * kCellW, coy = (cell / P.cells_x) * kCellH;
  HP Q;
  load_hot(P, Q);
  Anchor a;
  const ColCubic cc = cell_fit(P, Q, cox, coy, lane, a);
  const int gx = cox + lane;
  if (gx >= P.w) return;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  for (int r = 0; r < kCellH && coy + r < P.h; ++r) {
    float x, y;
    const bool ok = pixel_coords(P, Q, a, cc, lane, r, x, y);
    double* c = P.coords + 2 * (int64_t(coy + r) * P.w + gx);
    c[0] = ok ? double(a.bx) + double(x) : nan;
    c[1] = ok ? double(a.by) + double(y) : nan;
  }
}

cudaError_t launch_split_coords(const FwdPlan& p0, cudaStream_t s) {
  FwdPlan p = p0;
  void* args[] = {&p};
  return cudaLaunchKernel(reinterpret_cast<const void*>(&split_coords_kernel),
                          dim3(p0.cells_x * p0.cells_y), dim3(32), args, 0, s);
}

// ------------------------------------------------------------------ dispatch
int forward_threads_default() { return kFp64Threads; }

template <int ORDER>
static const void* fp64_for_order() {
  return reinterpret_cast<const void*>(&fwd_fp64_kernel<ORDER, kFp64Threads, false>);
}

// Split kernel of a launch form, tile height (8, 16 or 32 rows) and staging (sw: a plan of the
// launch stages its boxes by asynchronous copies), from its instantiation unit.
static const void* split_for(int order, bool batch, int th, bool sw) {
  if (sw) {
    if (batch) return th == 8 ? split_batch_sw_t8(order) : th == 32 ? split_batch_sw_t32(order)
                                                                    : split_batch_sw_t16(order);
    return th == 8 ? split_single_sw_t8(order) : th == 32 ? split_single_sw_t32(order)
                                                          : split_single_sw_t16(order);
  }
  if (batch) return th == 8 ? split_batch_t8(order) : th == 32 ? split_batch_t32(order)
                                                               : split_batch_t16(order);
  return th == 8 ? split_single_t8(order) : th == 32 ? split_single_t32(order)
                                                     : split_single_t16(order);
}

// The kernel instantiation for a launch: order, flags and tile height are uniform over a
// launch and taken from p0; batch launches read their plans from a table.
static const void* forward_kernel_for(const FwdPlan& p0, bool batch) {
  if (p0.flags & kFlagAccumulate) return batch ? nullptr : coadd_kernel(p0);
  if (p0.flags & DFR_SPLIT) return split_for(p0.order, batch, p0.th, p0.stage_sw != 0);
  switch (p0.order) {
    case DFR_NEAREST: return fp64_for_order<DFR_NEAREST>();
    case DFR_BILINEAR: return fp64_for_order<DFR_BILINEAR>();
    case DFR_BICUBIC: return fp64_for_order<DFR_BICUBIC>();
    case DFR_LANCZOS3: return fp64_for_order<DFR_LANCZOS3>();
    default: return fp64_for_order<DFR_BSPLINE3>();
  }
}

const void* forward_kernel(const FwdPlan& p0) { return forward_kernel_for(p0, false); }

// Block size of the kernel that serves this plan.
static int block_threads(const FwdPlan& p0) {
  return (p0.flags & DFR_SPLIT) ? kFwdWarps * 32 : kFp64Threads;
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

int forward_max_blocks_per_sm(const FwdPlan& p0, int threads, int smem_bytes, bool batch) {
  (void)threads;
  threads = block_threads(p0);
  const void* k = forward_kernel_for(p0, batch);
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
