// Persistent batch kernels of the split path (frame table in device memory, work units from an
// atomic counter), one per interpolation order and tile height; instantiated apart from the
// single-frame kernels so that the two sets compile in parallel.
#include "dfr_fwd_kernels.cuh"

namespace dfr {

template <int ORDER>
static const void* batch_for_order(int th) {
  switch (th) {
    case 8: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, true, false, 8>);
    case 32: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, true, false, 32>);
    default: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, true, false, 16>);
  }
}

const void* forward_batch_kernel(int order, int th) {
  switch (order) {
    case DFR_NEAREST: return batch_for_order<DFR_NEAREST>(th);
    case DFR_BILINEAR: return batch_for_order<DFR_BILINEAR>(th);
    case DFR_BICUBIC: return batch_for_order<DFR_BICUBIC>(th);
    case DFR_LANCZOS3: return batch_for_order<DFR_LANCZOS3>(th);
    default: return batch_for_order<DFR_BSPLINE3>(th);
  }
}

DFR_DEFINE_STATUS_READER(read_and_clear_status_batch)

}  // namespace dfr
