// Forward kernels for plans whose target grid carries SIP distortion: the split kernel with
// the target forward SIP in its fast rows (instantiated apart so that the kernels for plain
// targets keep their register allocation).
#include "dfr_fwd_kernels.cuh"

namespace dfr {

template <int ORDER>
static const void* tsip_for_order(int ideg) {
  switch (ideg) {
    case 0: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 0, false, false, true>);
    case 4: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 4, false, false, true>);
    case 6: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 6, false, false, true>);
    default: return reinterpret_cast<const void*>(&fwd_split_kernel<ORDER, 9, false, false, true>);
  }
}

// Single-frame split kernel for a plan with target SIP.
const void* tsip_kernel(const FwdPlan& p0) {
  switch (p0.order) {
    case DFR_NEAREST: return tsip_for_order<DFR_NEAREST>(p0.isip_deg);
    case DFR_BILINEAR: return tsip_for_order<DFR_BILINEAR>(p0.isip_deg);
    case DFR_BICUBIC: return tsip_for_order<DFR_BICUBIC>(p0.isip_deg);
    case DFR_LANCZOS3: return tsip_for_order<DFR_LANCZOS3>(p0.isip_deg);
    default: return tsip_for_order<DFR_BSPLINE3>(p0.isip_deg);
  }
}

DFR_DEFINE_STATUS_READER(read_and_clear_status_tsip)

}  // namespace dfr
