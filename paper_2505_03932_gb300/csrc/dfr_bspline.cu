// Cubic B-spline prefilter (dfr_bspline_prefilter), sm_103a: the coefficients c of the cubic
// B-spline that interpolates the image, c = (B3 sampled)^-1 S, separably along rows then
// columns. Along one line of n samples (Unser, Aldroubi & Eden, 1991; Unser, 1999): scale by the
// gain 6 = (1 - z)(1 - 1/z) with the pole z = sqrt(3) - 2, a causal pass
// c+[k] = s[k] + z c+[k-1] started from sum_j z^j s[mirror(j)] over a horizon where z^j is
// negligible, then an anticausal pass c[k] = z (c[k+1] - c+[k]) started from
// c[n-1] = z / (z^2 - 1) (c+[n-1] + z c+[n-2]) (the closed form for mirror boundaries).
// One thread per line: rows (stride 1, one warp spans 32 rows) and then columns (adjacent
// threads on adjacent columns: coalesced). Not part of the per-pixel hot path: it runs once per
// source image.
#include "dfr_device.cuh"

namespace dfr {

constexpr float kZ = -0.26794919243112270f;  // sqrt(3) - 2
constexpr int kHorizon = 16;                 // |z|^16 < 7e-10

// In-place filter of one line of n values at base[k * step] (values read from src[k * sstep],
// which may be the same memory).
__device__ __forceinline__ void bspline_line(const float* src, int64_t sstep, float* base,
                                             int64_t step, int n) {
  if (n == 1) {
    base[0] = src[0];
    return;
  }
  // causal start: sum over the mirrored horizon
  float c0 = 0.f, zk = 1.f;
  const int hz = kHorizon;
  for (int j = 0; j < hz; ++j) {
    c0 = fmaf(zk, 6.f * src[int64_t(mirror_index(j, n)) * sstep], c0);
    zk *= kZ;
  }
  float prev = c0;
  base[0] = c0;
  for (int k = 1; k < n; ++k) {
    prev = fmaf(kZ, prev, 6.f * src[int64_t(k) * sstep]);
    base[int64_t(k) * step] = prev;
  }
  // anticausal
  const float cp_last = prev, cp_prev = base[int64_t(n - 2) * step];
  float next = (kZ / (kZ * kZ - 1.f)) * fmaf(kZ, cp_prev, cp_last);
  base[int64_t(n - 1) * step] = next;
  for (int k = n - 2; k >= 0; --k) {
    next = kZ * (next - base[int64_t(k) * step]);
    base[int64_t(k) * step] = next;
  }
}

__global__ void __launch_bounds__(128) bspline_rows(const float* img, int64_t pitch, int w, int h,
                                                    float* coef, int64_t coef_pitch) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= h) return;
  bspline_line(img + int64_t(y) * pitch, 1, coef + int64_t(y) * coef_pitch, 1, w);
}

__global__ void __launch_bounds__(128) bspline_cols(float* coef, int64_t coef_pitch, int w, int h) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= w) return;
  bspline_line(coef + x, coef_pitch, coef + x, coef_pitch, h);
}

cudaError_t launch_bspline_prefilter(const float* img, int64_t pitch, int32_t w, int32_t h,
                                     float* coef, int64_t coef_pitch, cudaStream_t s) {
  bspline_rows<<<(h + 127) / 128, 128, 0, s>>>(img, pitch, w, h, coef, coef_pitch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bspline_cols<<<(w + 127) / 128, 128, 0, s>>>(coef, coef_pitch, w, h);
  return cudaGetLastError();
}

}  // namespace dfr
