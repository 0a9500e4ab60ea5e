// Cubic B-spline prefilter (dfr_bspline_prefilter), sm_103a: the coefficients c of the cubic
// B-spline that interpolates the image, c = (B3 sampled)^-1 S, separably along rows then
// columns. Along one line of n samples (Unser, Aldroubi & Eden, 1991; Unser, 1999): scale by the
// gain 6 = (1 - z)(1 - 1/z) with the pole z = sqrt(3) - 2, a causal pass
// c+[k] = 6 s[k] + z c+[k-1] started from sum_j z^j 6 s[mirror(j)] over a horizon where z^j is
// negligible, then an anticausal pass c[k] = z (c[k+1] - c+[k]) started from
// c[n-1] = z / (z^2 - 1) (c+[n-1] + z c+[n-2]) (the closed form for mirror boundaries).
//
// Parallel form: |z| = 0.268, so a value's influence on the recursion falls below 4e-12 (far
// under FP32 rounding) after kWarm = 20 samples. Each line is cut into segments of kSeg samples,
// one thread per segment: the causal pass of a segment starts kWarm samples early from zero (the
// first segment from the mirrored start), the anticausal pass kWarm samples late from zero (the
// last segments from the closed form). Four launches, ping-ponging through a scratch image:
// rows causal (img -> scratch), rows anticausal (scratch -> coef), columns causal (coef ->
// scratch), columns anticausal (scratch -> coef). Column threads of a warp take adjacent
// columns (coalesced); row threads of a warp take the segments of one row (each walks its own
// cache lines, reused from L1).
#include "dfr_device.cuh"

namespace dfr {

constexpr float kZ = -0.26794919243112270f;  // sqrt(3) - 2
constexpr int kHorizon = 16;                 // mirrored start: |z|^16 < 7e-10
constexpr int kSeg = 64;                     // samples per thread
constexpr int kWarm = 20;                    // |z|^20 < 4e-12

// Element k of line `line` (ROWS: line = row, k = column; else line = column, k = row).
template <bool ROWS>
__device__ __forceinline__ int64_t at(int line, int k, int64_t pitch) {
  return ROWS ? int64_t(line) * pitch + k : int64_t(k) * pitch + line;
}

template <bool ROWS>
__device__ __forceinline__ bool seg_of(int w, int h, int& line, int& k0, int& n) {
  n = ROWS ? w : h;
  const int nseg = (n + kSeg - 1) / kSeg, lines = ROWS ? h : w;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(nseg) * lines) return false;
  // rows: a warp's threads are consecutive segments of one row; columns: adjacent columns
  const int seg = ROWS ? int(t % nseg) : int(t / lines);
  line = ROWS ? int(t / nseg) : int(t % lines);
  k0 = seg * kSeg;
  return true;
}

template <bool ROWS>
__global__ void __launch_bounds__(256) bspline_causal(const float* __restrict__ s, int64_t sp,
                                                      float* __restrict__ cp, int64_t cpp, int w,
                                                      int h) {
  int line, k0, n;
  if (!seg_of<ROWS>(w, h, line, k0, n)) return;
  const int k1 = min(n, k0 + kSeg);
  if (n == 1) {
    cp[at<ROWS>(line, 0, cpp)] = 6.f * s[at<ROWS>(line, 0, sp)];  // a single sample is its own
    return;                                                        // coefficient (6 s / 6)
  }
  float c = 0.f;
  if (k0 == 0) {
    // mirrored start
    float zk = 1.f;
    for (int j = 0; j < kHorizon; ++j) {
      c = fmaf(zk, 6.f * s[at<ROWS>(line, mirror_index(j, n), sp)], c);
      zk *= kZ;
    }
    cp[at<ROWS>(line, 0, cpp)] = c;
    k0 = 1;
  } else {
    for (int k = max(0, k0 - kWarm); k < k0; ++k) c = fmaf(kZ, c, 6.f * s[at<ROWS>(line, k, sp)]);
  }
  for (int k = k0; k < k1; ++k) {
    c = fmaf(kZ, c, 6.f * s[at<ROWS>(line, k, sp)]);
    cp[at<ROWS>(line, k, cpp)] = c;
  }
}

template <bool ROWS>
__global__ void __launch_bounds__(256) bspline_anticausal(const float* __restrict__ cp,
                                                          int64_t cpp, float* __restrict__ out,
                                                          int64_t op, int w, int h) {
  int line, k0, n;
  if (!seg_of<ROWS>(w, h, line, k0, n)) return;
  const int k1 = min(n, k0 + kSeg);
  if (n == 1) {
    out[at<ROWS>(line, 0, op)] = cp[at<ROWS>(line, 0, cpp)] / 6.f;  // undo the causal gain
    return;
  }
  float c;
  int k;
  if (k1 + kWarm >= n) {
    // closed-form start at the end of the line, then down to this segment
    c = (kZ / (kZ * kZ - 1.f)) *
        fmaf(kZ, cp[at<ROWS>(line, n - 2, cpp)], cp[at<ROWS>(line, n - 1, cpp)]);
    if (k1 == n) out[at<ROWS>(line, n - 1, op)] = c;
    for (k = n - 2; k >= k1; --k) c = kZ * (c - cp[at<ROWS>(line, k, cpp)]);
    k = (k1 == n) ? n - 2 : k1 - 1;
  } else {
    c = 0.f;
    for (k = k1 + kWarm - 1; k >= k1; --k) c = kZ * (c - cp[at<ROWS>(line, k, cpp)]);
    k = k1 - 1;
  }
  for (; k >= k0; --k) {
    c = kZ * (c - cp[at<ROWS>(line, k, cpp)]);
    out[at<ROWS>(line, k, op)] = c;
  }
}

namespace {
struct Scratch {
  float* p = nullptr;
  size_t cap = 0;
};
Scratch g_scratch[64];  // per device ordinal
}  // namespace

cudaError_t launch_bspline_prefilter(const float* img, int64_t pitch, int32_t w, int32_t h,
                                     float* coef, int64_t coef_pitch, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  Scratch& sc = g_scratch[dev];
  const int64_t sp = (int64_t(w) + 3) & ~int64_t(3);
  const size_t need = size_t(sp) * size_t(h);
  if (need > sc.cap) {
    // the stream's earlier work may still read the old buffer
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (sc.p) cudaFree(sc.p);
    sc.p = nullptr;
    sc.cap = 0;
    e = cudaMalloc(&sc.p, need * sizeof(float));
    if (e != cudaSuccess) return e;
    sc.cap = need;
  }
  const int64_t rows_t = int64_t((w + kSeg - 1) / kSeg) * h;
  const int64_t cols_t = int64_t((h + kSeg - 1) / kSeg) * w;
  const unsigned gr = unsigned((rows_t + 255) / 256), gc = unsigned((cols_t + 255) / 256);
  bspline_causal<true><<<gr, 256, 0, s>>>(img, pitch, sc.p, sp, w, h);
  bspline_anticausal<true><<<gr, 256, 0, s>>>(sc.p, sp, coef, coef_pitch, w, h);
  bspline_causal<false><<<gc, 256, 0, s>>>(coef, coef_pitch, sc.p, sp, w, h);
  bspline_anticausal<false><<<gc, 256, 0, s>>>(sc.p, sp, coef, coef_pitch, w, h);
  return cudaGetLastError();
}

}  // namespace dfr
