// Co-add (stacking) kernels, sm_103a: the forward kernels instantiated with accumulating
// outputs (sum_vf += value * footprint, sum_f += footprint per target pixel; the step after
// reprojection that motivates the method, Sec. 1), and the final normalisation
// mean = sum_vf / sum_f.
#include <algorithm>
#include <cstdint>

#include "dfr_fwd_kernels.cuh"

namespace dfr {

template <int ORDER>
static const void* coadd_for_order(bool split) {
  if (!split) return reinterpret_cast<const void*>(&fwd_fp64_kernel<ORDER, kFp64Threads, true>);
  return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, false, true, kDefaultTileH, true>);
}

// Single-frame accumulating kernel for a plan (frames of a co-add are launched one after
// another, so no two launches touch the sums at once).
const void* coadd_kernel(const FwdPlan& p0) {
  const bool split = (p0.flags & DFR_SPLIT) != 0;
  switch (p0.order) {
    case DFR_NEAREST: return coadd_for_order<DFR_NEAREST>(split);
    case DFR_BILINEAR: return coadd_for_order<DFR_BILINEAR>(split);
    case DFR_BICUBIC: return coadd_for_order<DFR_BICUBIC>(split);
    case DFR_LANCZOS3: return coadd_for_order<DFR_LANCZOS3>(split);
    default: return coadd_for_order<DFR_BSPLINE3>(split);
  }
}

// mean = sum_vf / sum_f where sum_f > min_weight, else 0 (the uncovered-pixel convention of
// the forward outputs); IEEE division. V = 4: float4 accesses (rows of a multiple of 4 values,
// 16-byte aligned rows), else scalar. Columns across threads, rows strided over grid.y.
// (mean may alias sum_vf: each element is read before the same thread writes it.)
__device__ __forceinline__ float mean_of(float v, float f, float min_weight) {
  return f > min_weight ? v / f : 0.f;
}

template <int V>
__global__ void __launch_bounds__(256) coadd_normalize_kernel(const float* sum_vf,
                                                              const float* __restrict__ sum_f,
                                                              int64_t pitch, int32_t w, int32_t h,
                                                              float min_weight, float* mean,
                                                              int64_t mean_pitch) {
  const int x = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (x >= w) return;
  for (int y = blockIdx.y; y < h; y += gridDim.y) {
    const int64_t i = int64_t(y) * pitch + x, o = int64_t(y) * mean_pitch + x;
    if (V == 4) {
      const float4 f = __ldcs(reinterpret_cast<const float4*>(sum_f + i));
      const float4 v = __ldcs(reinterpret_cast<const float4*>(sum_vf + i));
      __stcs(reinterpret_cast<float4*>(mean + o),
             make_float4(mean_of(v.x, f.x, min_weight), mean_of(v.y, f.y, min_weight),
                         mean_of(v.z, f.z, min_weight), mean_of(v.w, f.w, min_weight)));
    } else {
      const float f = __ldcs(sum_f + i);
      const float v = __ldcs(sum_vf + i);
      __stcs(mean + o, mean_of(v, f, min_weight));
    }
  }
}

cudaError_t launch_coadd_normalize(const float* sum_vf, const float* sum_f, int64_t pitch,
                                   int32_t w, int32_t h, float min_weight, float* mean,
                                   int64_t mean_pitch, cudaStream_t s) {
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const bool vec = w % 4 == 0 && pitch % 4 == 0 && mean_pitch % 4 == 0 && a16(sum_vf) &&
                   a16(sum_f) && a16(mean);
  const int V = vec ? 4 : 1;
  const unsigned gx = (unsigned(w / V) + 255u) / 256u;
  // about 4096 CTAs in all: enough to fill the GPU, few enough to amortise each CTA's start
  const unsigned gy = unsigned(std::max(1, std::min(h, int(4096u / gx) > 0 ? int(4096u / gx) : 1)));
  const dim3 grid(gx, std::min(gy, 65535u));
  if (vec)
    coadd_normalize_kernel<4><<<grid, 256, 0, s>>>(sum_vf, sum_f, pitch, w, h, min_weight, mean,
                                                   mean_pitch);
  else
    coadd_normalize_kernel<1><<<grid, 256, 0, s>>>(sum_vf, sum_f, pitch, w, h, min_weight, mean,
                                                   mean_pitch);
  return cudaGetLastError();
}

DFR_DEFINE_STATUS_READER(read_and_clear_status_coadd)

}  // namespace dfr
