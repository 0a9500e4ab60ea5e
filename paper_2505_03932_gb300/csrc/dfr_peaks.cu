// Throughput of the arithmetic pipes the reprojection kernels use, measured on the device the
// caller has current (dfr_measure_pipe_peaks): FP64 fused multiply-add, FP32 fused multiply-add
// (scalar and packed FP32x2) and the special-function unit (sin.approx.f32). Each thread runs 8
// independent dependent chains (enough to cover the pipe latency at full occupancy) over a grid
// that fills every SM; the count of operations over the CUDA-event time is the pipe's rate.
// These are the denominators of the all-FP64 path's roofline.
#include <cuda_runtime.h>

#include "dfr_internal.h"

namespace dfr {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

// Where a kernel would store its chains' sum if it ever equalled its sentinel (never, for these
// inputs): the results stay live without any allocation.
__device__ double g_peak_sink[2];

__global__ void __launch_bounds__(kPeakThreads) peak_dfma(double m, double c, int iters,
                                                          double* sink) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.678) sink[0] = s;  // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(kPeakThreads) peak_ffma(float m, float c, int iters,
                                                          float* sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * float(threadIdx.x + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.678f) sink[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) peak_ffma2(float m, float c, int iters,
                                                           float* sink) {
  float2 a[kChains];
  const float2 mm = make_float2(m, m), cc = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = make_float2(1e-3f * float(threadIdx.x + k), 0.5f);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], mm, cc);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  if (s == 12345.678f) sink[0] = s;
}

__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(kPeakThreads) peak_mufu(float c, int iters, float* sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * float(threadIdx.x + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = sin_approx(a[k] + c);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.678f) sink[0] = s;
}

// Operations per second of one kernel launch: ops per thread-iteration x threads x iterations
// over the best of three timed launches.
template <typename F>
double rate(F launch, double ops_per_launch, cudaStream_t s, cudaError_t& err) {
  cudaEvent_t e0, e1;
  if ((err = cudaEventCreate(&e0)) != cudaSuccess) return 0.0;
  if ((err = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 0.0;
  }
  launch();  // warm-up (clocks up, code loaded)
  float best = 1e30f;
  for (int r = 0; r < 3 && err == cudaSuccess; ++r) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err == cudaSuccess ? ops_per_launch / (double(best) * 1e-3) : 0.0;
}

}  // namespace
}  // namespace dfr

using namespace dfr;

extern "C" int dfr_measure_pipe_peaks(double* out, void* stream) {
  if (!out) return report_error(DFR_ERR_INVALID_ARG, "NULL argument");
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, reinterpret_cast<const void*>(&peak_dfma), kPeakThreads, 0);
  if (e != cudaSuccess) return report_cuda_error(e, "dfr_measure_pipe_peaks");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const double threads = double(grid) * kPeakThreads;
  void* sink = nullptr;
  e = cudaGetSymbolAddress(&sink, g_peak_sink);
  if (e != cudaSuccess) return report_cuda_error(e, "cudaGetSymbolAddress");
  const int it64 = 2048, it32 = 32768, itmu = 8192;
  out[0] = rate([&] { peak_dfma<<<grid, kPeakThreads, 0, s>>>(0.999999, 1e-9, it64,
                                                            static_cast<double*>(sink)); },
                threads * it64 * kChains * 2.0, s, e);
  if (e == cudaSuccess)
    out[1] = rate([&] { peak_ffma<<<grid, kPeakThreads, 0, s>>>(0.999999f, 1e-9f, it32,
                                                              static_cast<float*>(sink)); },
                  threads * it32 * kChains * 2.0, s, e);
  if (e == cudaSuccess)
    out[2] = rate([&] { peak_ffma2<<<grid, kPeakThreads, 0, s>>>(0.999999f, 1e-9f, it32,
                                                               static_cast<float*>(sink)); },
                  threads * it32 * kChains * 4.0, s, e);
  if (e == cudaSuccess)
    out[3] = rate([&] { peak_mufu<<<grid, kPeakThreads, 0, s>>>(1e-3f, itmu,
                                                              static_cast<float*>(sink)); },
                  threads * itmu * kChains, s, e);
  if (e != cudaSuccess) return report_cuda_error(e, "dfr_measure_pipe_peaks");
  return DFR_OK;
}
