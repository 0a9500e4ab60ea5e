// Adjoint (backward) kernels: see dfr_reproject_backward in include/dfr.h.
#include "dfr_device.cuh"

namespace dfr {

cudaError_t read_and_clear_status_bwd(int32_t* out, cudaStream_t s) {
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
