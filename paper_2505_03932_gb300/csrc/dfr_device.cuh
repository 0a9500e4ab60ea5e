// Device helpers shared by the forward and backward kernels: SIP polynomials (Horner in
// registers), the FP64 per-pixel transform of Sec. 3.2.1 / 3.2.2, the split-precision tile
// anchor, interpolation weights, and the TMA / mbarrier primitives.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dfr_internal.h"

namespace dfr {

// Device status word of this translation unit (each kernel file has its own copy).
static __device__ int32_t g_status = 0;

// Each translation unit that includes this header has its own status word; this defines the
// host-side reader (copy out on stream s, then clear if set) for the including unit's word.
#define DFR_DEFINE_STATUS_READER(fn)                                                        \
  cudaError_t fn(int32_t* out, cudaStream_t s) {                                           \
    int32_t zero = 0;                                                                      \
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_status, sizeof(int32_t), 0,           \
                                              cudaMemcpyDeviceToHost, s);                  \
    if (e != cudaSuccess) return e;                                                        \
    e = cudaStreamSynchronize(s);                                                          \
    if (e != cudaSuccess) return e;                                                        \
    if (*out != 0) e = cudaMemcpyToSymbol(g_status, &zero, sizeof(int32_t));               \
    return e;                                                                              \
  }

constexpr double kR0 = 57.295779513082320876798154814105;  // 180 / pi
constexpr double kSnap = 1e-9;                               // FP64 integer snap radius, px

// ---------------------------------------------------------------- polynomials (Horner)
// Fixed degree N, coefficients of two polynomials (A and B) evaluated at the same (u, v).
template <int N, typename T>
__device__ __forceinline__ void horner_pair(const T* __restrict__ ca, const T* __restrict__ cb,
                                            T u, T v, T& A, T& B) {
  T pa = T(0), pb = T(0);
#pragma unroll
  for (int p = N; p >= 0; --p) {
    const int off = poly_off(p, N);
    T qa = ca[off + (N - p)], qb = cb[off + (N - p)];
#pragma unroll
    for (int q = N - p - 1; q >= 0; --q) {
      qa = fma(qa, v, ca[off + q]);
      qb = fma(qb, v, cb[off + q]);
    }
    if (p == N) {
      pa = qa;
      pb = qb;
    } else {
      pa = fma(pa, u, qa);
      pb = fma(pb, u, qb);
    }
  }
  A = pa;
  B = pb;
}

// The same Horner scheme for the pair (A, B) in packed FP32x2 arithmetic: c[k] = (a_k, b_k).
// Each half runs exactly the FMA sequence of horner_pair, so the results are the same bits.
template <int N>
__device__ __forceinline__ float2 horner_pair2(const float2* __restrict__ c, float u, float v) {
  const float2 uu = make_float2(u, u), vv = make_float2(v, v);
  float2 pp = make_float2(0.f, 0.f);
#pragma unroll
  for (int p = N; p >= 0; --p) {
    const int off = poly_off(p, N);
    float2 qq = c[off + (N - p)];
#pragma unroll
    for (int q = N - p - 1; q >= 0; --q) qq = __ffma2_rn(qq, vv, c[off + q]);
    pp = (p == N) ? qq : __ffma2_rn(pp, uu, qq);
  }
  return pp;
}

// Runtime degree n (FP64 path and rarely used branches).
template <typename T>
__device__ __forceinline__ void horner_pair_rt(const T* ca, const T* cb, int n, T u, T v,
                                               T& A, T& B) {
  T pa = T(0), pb = T(0);
  for (int p = n; p >= 0; --p) {
    const int off = poly_off(p, n);
    T qa = ca[off + (n - p)], qb = cb[off + (n - p)];
    for (int q = n - p - 1; q >= 0; --q) {
      qa = fma(qa, v, ca[off + q]);
      qb = fma(qb, v, cb[off + q]);
    }
    pa = (p == n) ? qa : fma(pa, u, qa);
    pb = (p == n) ? qb : fma(pb, u, qb);
  }
  A = pa;
  B = pb;
}

// Value and first partials of one polynomial (runtime degree): P, dP/du, dP/dv.
// Compile-time-degree form of horner_grad_rt below: the same FMA sequence, unrolled, so both
// give equal bits for the same (zero-padded) coefficients.
template <int N, typename T>
__device__ __forceinline__ void horner_grad(const T* c, T u, T v, T& P, T& Pu, T& Pv) {
  T p_ = T(0), pu = T(0), pv = T(0);
#pragma unroll
  for (int p = N; p >= 0; --p) {
    const int off = poly_off(p, N);
    T q_ = c[off + (N - p)], qv = T(0);
#pragma unroll
    for (int q = N - p - 1; q >= 0; --q) {
      qv = fma(qv, v, q_);
      q_ = fma(q_, v, c[off + q]);
    }
    pu = fma(pu, u, p_);
    p_ = fma(p_, u, q_);
    pv = fma(pv, u, qv);
  }
  P = p_;
  Pu = pu;
  Pv = pv;
}

template <typename T>
__device__ __forceinline__ void horner_grad_rt(const T* c, int n, T u, T v, T& P, T& Pu, T& Pv) {
  T p_ = T(0), pu = T(0), pv = T(0);
  for (int p = n; p >= 0; --p) {
    const int off = poly_off(p, n);
    T q_ = c[off + (n - p)], qv = T(0);
    for (int q = n - p - 1; q >= 0; --q) {
      qv = fma(qv, v, q_);
      q_ = fma(q_, v, c[off + q]);
    }
    pu = fma(pu, u, p_);
    p_ = fma(p_, u, q_);
    pv = fma(pv, u, qv);
  }
  P = p_;
  Pu = pu;
  Pv = pv;
}

// Value and gradient of a packed polynomial of degree DEG (> 0: compile time; < 0: the runtime
// degree n). Both forms give equal bits.
template <int DEG, typename T>
__device__ __forceinline__ void poly_grad(const T* c, int n, T u, T v, T& P, T& Pu, T& Pv) {
  if (DEG > 0)
    horner_grad<(DEG > 0 ? DEG : 1), T>(c, u, v, P, Pu, Pv);
  else
    horner_grad_rt<T>(c, n, u, v, P, Pu, Pv);
}

// ---------------------------------------------------------------- interpolation weights
// Taps start at floor(x) + kLo[order]; count kTaps[order].
template <int ORDER> struct Taps;
template <> struct Taps<DFR_NEAREST> { static constexpr int n = 1, lo = 0; };
template <> struct Taps<DFR_BILINEAR> { static constexpr int n = 2, lo = 0; };
template <> struct Taps<DFR_BICUBIC> { static constexpr int n = 4, lo = -1; };
template <> struct Taps<DFR_LANCZOS3> { static constexpr int n = 6, lo = -2; };
template <> struct Taps<DFR_BSPLINE3> { static constexpr int n = 4, lo = -1; };

// Whole-sample symmetric (mirror) extension of index i over [0, n): ... 2 1 | 0 1 2 ... n-1 |
// n-2 ... (period 2 (n - 1)). Used for the B-spline taps outside the image.
__device__ __forceinline__ int mirror_index(int i, int n) {
  if (n <= 1) return 0;
  const int p = 2 * (n - 1);
  i %= p;
  if (i < 0) i += p;
  return i < n ? i : p - i;
}

// ---------------------------------------------------------------- explicitly rounded helpers
// One value (float, double) or a pair (float2: packed FP32x2, each half exactly the scalar
// operation). Every step is a rounding the compiler may not fuse or reorder, so an expression
// written with these gives the same bits in every kernel and for either operand width.
__device__ __forceinline__ float v_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float v_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float v_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float v_splat(float a, float) { return a; }
__device__ __forceinline__ double v_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double v_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double v_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double v_splat(float a, double) { return double(a); }
__device__ __forceinline__ float2 v_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 v_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 v_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 v_splat(float a, float2) { return make_float2(a, a); }
template <typename V>
__device__ __forceinline__ V v_c(float a) { return v_splat(a, V()); }

__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// Lanczos-3 (sinc window sinc(d/3), |d| < 3) at the six tap offsets d_k = t + 2 - k, normalised
// to sum 1. With th = pi t / 3: sin(pi d_k) = (-1)^k sin(pi t) and sin(pi d_k / 3) =
// sin(th + pi (2 - k) / 3) (angle addition); the common factor 3 sin(pi t) / pi^2 of
// sinc(d) sinc(d / 3) cancels in the normalisation, leaving w_k proportional to
// (-1)^k sin(th + pi (2 - k) / 3) / d_k^2. Below t = 1e-12 the weights of t = 0 (1 at the node).
template <typename T>
__device__ __forceinline__ void lanczos3_weights(T t, T* w) {
  if (t < T(1e-12)) {
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = (k == 2) ? T(1) : T(0);
    return;
  }
  T s, c;
  sincospi_t(t / T(3), &s, &c);
  const T h = T(0.86602540378443864676);  // sin(pi / 3)
  const T a[6] = {fma(c, h, T(-0.5) * s), fma(c, h, T(0.5) * s), s,
                  fma(-c, h, T(0.5) * s), fma(-c, h, T(-0.5) * s), -s};
  T sum = T(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const T d = t + T(2 - k);
    const T v = ((k & 1) ? -a[k] : a[k]) / (d * d);
    w[k] = v;
    sum += v;
  }
  const T inv = T(1) / sum;
#pragma unroll
  for (int k = 0; k < 6; ++k) w[k] *= inv;
}

// Interpolation weights at fraction t = x - floor(x) in [0, 1) (nearest: the caller shifts the
// index when t >= 1/2). V = float, double, or float2 (two independent fractions at once). The
// operation sequence is the definition: every FP32 gather path (shared-memory box, global
// memory, the packed two-pixel rows) evaluates it, so they agree bit for bit.
//   bilinear: 1 - t, t
//   bicubic (Keys cubic convolution, a = -0.5, taps at distances 1 + t, t, 1 - t, 2 - t):
//     t (t (1 - t/2) - 1/2), t^2 (3t/2 - 5/2) + 1, t (t (2 - 3t/2) + 1/2), t^2 (t/2 - 1/2)
//   cubic B-spline: (1-t)^3/6, 2/3 - t^2 + t^3/2, 2/3 - (1-t)^2 + (1-t)^3/2, t^3/6
template <int ORDER, typename V>
__device__ __forceinline__ void weights_v(V t, V* w) {
  if (ORDER == DFR_NEAREST) {
    w[0] = v_c<V>(1.f);
  } else if (ORDER == DFR_BILINEAR) {
    w[0] = v_add(v_c<V>(1.f), v_mul(v_c<V>(-1.f), t));
    w[1] = t;
  } else if (ORDER == DFR_BSPLINE3) {
    const V s = v_add(v_c<V>(1.f), v_mul(v_c<V>(-1.f), t));
    const V sixth = v_c<V>(1.f / 6.f), two3 = v_c<V>(2.f / 3.f);
    const V half = v_c<V>(0.5f), mone = v_c<V>(-1.f);
    const V s2 = v_mul(s, s), t2 = v_mul(t, t);
    w[0] = v_mul(s2, v_mul(s, sixth));
    w[1] = v_fma(t2, v_fma(half, t, mone), two3);
    w[2] = v_fma(s2, v_fma(half, s, mone), two3);
    w[3] = v_mul(t2, v_mul(t, sixth));
  } else {  // bicubic
    const V t2 = v_mul(t, t);
    w[0] = v_mul(t, v_fma(v_fma(v_c<V>(-0.5f), t, v_c<V>(1.f)), t, v_c<V>(-0.5f)));
    w[1] = v_fma(t2, v_fma(v_c<V>(1.5f), t, v_c<V>(-2.5f)), v_c<V>(1.f));
    w[2] = v_mul(t, v_fma(v_fma(v_c<V>(-1.5f), t, v_c<V>(2.f)), t, v_c<V>(0.5f)));
    w[3] = v_mul(t2, v_fma(v_c<V>(0.5f), t, v_c<V>(-0.5f)));
  }
}

template <int ORDER, typename T>
__device__ __forceinline__ void weights(T t, T* w) {
  if (ORDER == DFR_LANCZOS3)
    lanczos3_weights<T>(t, w);
  else
    weights_v<ORDER, T>(t, w);
}

// weights() for x and y at once: w[k] = (wx_k, wy_k), each half the bits of weights().
template <int ORDER>
__device__ __forceinline__ void weights2(float2 t, float2* w) {
  if (ORDER == DFR_LANCZOS3) {
    float wx[6], wy[6];
    lanczos3_weights<float>(t.x, wx);
    lanczos3_weights<float>(t.y, wy);
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = make_float2(wx[k], wy[k]);
  } else {
    weights_v<ORDER, float2>(t, w);
  }
}

// d/dt of the normalised Lanczos-3 weights. In the form of lanczos3_weights, each unnormalised
// weight times t: v_k = (-1)^k a_k(th) t / d_k^2 for k != 2 and v_2 = sin(th) / t (finite at
// t = 0), th = pi t / 3, a_k the angle-addition terms, a_k' their derivatives in th. Then
// dv_k/dt = (-1)^k (pi/3 a_k' t + a_k (1 - 2 t / d_k)) / d_k^2, and for k = 2, with
// sin(th) / t = (pi/3) sin(th) / th, dv_2/dt = (pi/3)^2 (th cos th - sin th) / th^2, by its
// series -th / 3 + th^3 / 30 below th = 0.05 (the closed form cancels there). The normalised
// weights w = v / S (S = sum v) have dw_k/dt = (dv_k - w_k sum dv) / S. The kernel is even, so
// w_k(t) = w_{5-k}(1 - t): above t = 1/2 the derivatives come from 1 - t, mirrored, so that the
// node nearest t is always k = 2 (where the series keeps the pole out of the arithmetic).
template <typename T>
__device__ __forceinline__ void lanczos3_dweights(T t_in, T* d) {
  const bool mirror = t_in > T(0.5);
  const T t = mirror ? T(1) - t_in : t_in;
  const T pi3 = T(1.04719755119659774615);  // pi / 3
  const T th = pi3 * t;
  T s, c;
  sincospi_t(t / T(3), &s, &c);
  const T h = T(0.86602540378443864676);  // sin(pi / 3)
  const T a[6] = {fma(c, h, T(-0.5) * s), fma(c, h, T(0.5) * s), s,
                  fma(-c, h, T(0.5) * s), fma(-c, h, T(-0.5) * s), -s};
  const T ad[6] = {fma(-s, h, T(-0.5) * c), fma(-s, h, T(0.5) * c), c,
                   fma(s, h, T(0.5) * c), fma(s, h, T(-0.5) * c), -c};
  T v[6], dv[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    if (k == 2) continue;
    const T dk = t + T(2 - k);
    const T sg = (k & 1) ? T(-1) : T(1);
    const T inv2 = T(1) / (dk * dk);
    v[k] = sg * a[k] * t * inv2;
    dv[k] = sg * fma(pi3 * ad[k], t, a[k] * (T(1) - T(2) * t / dk)) * inv2;
  }
  if (th < T(0.05)) {
    const T th2 = th * th;
    v[2] = pi3 * fma(th2, fma(th2, T(1.0 / 120.0), T(-1.0 / 6.0)), T(1));
    dv[2] = pi3 * pi3 * th * fma(th2, T(1.0 / 30.0), T(-1.0 / 3.0));
  } else {
    v[2] = s / t;
    dv[2] = pi3 * pi3 * (th * c - s) / (th * th);
  }
  T S = T(0), Sd = T(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    S += v[k];
    Sd += dv[k];
  }
  const T inv = T(1) / S;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int j = mirror ? 5 - k : k;
    const T dk = (dv[j] - v[j] * inv * Sd) * inv;
    d[k] = mirror ? -dk : dk;
  }
}

// d(weights)/dt for the backward pass.
template <int ORDER, typename T>
__device__ __forceinline__ void dweights(T t, T* d) {
  if (ORDER == DFR_NEAREST) {
    d[0] = T(0);
  } else if (ORDER == DFR_BILINEAR) {
    d[0] = T(-1);
    d[1] = T(1);
  } else if (ORDER == DFR_LANCZOS3) {
    lanczos3_dweights<T>(t, d);
  } else {
    const T s = T(1) - t;
    // w0 = -t s^2 / 2          -> -(s^2)/2 + t s
    // w1 = 1.5 t^3 - 2.5 t^2 + 1 -> 4.5 t^2 - 5 t
    // w2 = 1.5 s^3 - 2.5 s^2 + 1 -> -(4.5 s^2 - 5 s)
    // w3 = -t^2 s / 2          -> -t s + t^2 / 2
    d[0] = fma(T(-0.5) * s, s, t * s);
    d[1] = t * fma(T(4.5), t, T(-5));
    d[2] = -(s * fma(T(4.5), s, T(-5)));
    d[3] = fma(T(0.5) * t, t, -(t * s));
  }
}

// ---------------------------------------------------------------- FP64 per-pixel transform
// Sec. 3.2.1 then Sec. 3.2.2, literally, in FP64 (the two asin steps as atan2(z, hypot(x, y)),
// the same angle, well conditioned near the tangent point and the poles).
__device__ __forceinline__ void world_from_target_fp64(const FwdPlan& P, double X, double Y,
                                                       double& ra, double& dec) {
  double u = X - P.crpix_t[0];
  double v = Y - P.crpix_t[1];
  if (P.tsip_deg > 0) {
    double fa, fb;
    horner_pair_rt<double>(P.tsip_d[0], P.tsip_d[1], P.tsip_deg, u, v, fa, fb);
    u += fa;
    v += fb;
  }
  const double up = P.cd_t[0][0] * u + P.cd_t[0][1] * v;
  const double vp = P.cd_t[1][0] * u + P.cd_t[1][1] * v;
  const double r = sqrt(up * up + vp * vp);
  const double phi = atan2(-up, vp);
  const double theta = atan2(kR0, r);
  double st, ct, sp, cp;
  sincos(theta, &st, &ct);
  sincos(phi, &sp, &cp);
  const double z = st * P.sd0_t + ct * P.cd0_t * cp;
  const double ya = -ct * sp;
  const double xa = st * P.cd0_t - ct * P.sd0_t * cp;
  dec = atan2(z, sqrt(ya * ya + xa * xa));
  ra = P.ra0_t + atan2(ya, xa);
}

// Returns false where the source projection is undefined (sin theta <= 0).
__device__ __forceinline__ bool intermediate_from_world_fp64(const FwdPlan& P, double ra,
                                                             double dec, double& U, double& V) {
  const double dra = ra - P.ra0_s;
  double sd, cdn, sdra, cdra;
  sincos(dec, &sd, &cdn);
  sincos(dra, &sdra, &cdra);
  const double n1 = -cdn * sdra;
  const double n2 = sd * P.cd0_s - cdn * P.sd0_s * cdra;
  const double dd = sd * P.sd0_s + cdn * P.cd0_s * cdra;
  const double phi = atan2(n1, n2);
  const double theta = atan2(dd, sqrt(n1 * n1 + n2 * n2));
  double st, ct, sp, cp;
  sincos(theta, &st, &ct);
  sincos(phi, &sp, &cp);
  const double r = kR0 * ct / st;
  const double up = -r * sp;
  const double vp = r * cp;
  U = P.cdinv_s[0][0] * up + P.cdinv_s[0][1] * vp;
  V = P.cdinv_s[1][0] * up + P.cdinv_s[1][1] * vp;
  return st > 0.0;
}

// Newton solve of u + A(u, v) = U, v + B(u, v) = V (FP64), started from (u, v).
__device__ __forceinline__ void newton_fp64(const FwdPlan& P, double U, double V, double& u,
                                            double& v) {
  for (int it = 0; it < 30; ++it) {
    double A, Au, Av, B, Bu, Bv;
    horner_grad_rt<double>(P.fsip_d[0], P.fsip_deg, u, v, A, Au, Av);
    horner_grad_rt<double>(P.fsip_d[1], P.fsip_deg, u, v, B, Bu, Bv);
    const double fu = u + A - U, fv = v + B - V;
    const double j00 = 1.0 + Au, j01 = Av, j10 = Bu, j11 = 1.0 + Bv;
    const double det = j00 * j11 - j01 * j10;
    const double du = (j11 * fu - j01 * fv) / det;
    const double dv = (j00 * fv - j10 * fu) / det;
    u -= du;
    v -= dv;
    if (fabs(du) < 1e-12 && fabs(dv) < 1e-12) break;
  }
}

__device__ __forceinline__ bool source_from_target_fp64(const FwdPlan& P, double X, double Y,
                                                        double& xs, double& ys) {
  if (P.identity) {
    xs = X + P.shift[0];
    ys = Y + P.shift[1];
    return true;
  }
  double ra, dec, U, V;
  world_from_target_fp64(P, X, Y, ra, dec);
  const bool ok = intermediate_from_world_fp64(P, ra, dec, U, V);
  double u = U, v = V;
  if (P.isip_deg > 0) {
    double ga, gb;
    horner_pair_rt<double>(P.isip_d[0], P.isip_d[1], P.isip_deg, U, V, ga, gb);
    u = U + ga;
    v = V + gb;
  }
  if ((P.flags & DFR_EXACT_INVERSE) && P.fsip_deg > 0) newton_fp64(P, U, V, u, v);
  xs = u + P.crpix_s[0];
  ys = v + P.crpix_s[1];
  return ok;
}

// ---------------------------------------------------------------- split-precision anchor
// Wide-precision part of the split path, at each cell-fit node and at the cell's anchor: the
// homography at that target position (double-float, or FP64 with a target SIP), the source
// position split into integer and fractional parts, and the FP32 coefficients of the local
// expansion around it.
struct Anchor {
  int32_t bx, by;        // integer part of the anchor's source position
  float f0x, f0y;        // anchor source position minus (bx, by)
  float U0, V0;          // anchor source intermediate offsets (for SIP evaluation)
  float a0, a1, b0, b1;  // numerators of the local homography
  float g20, g21, h2;    // its denominator
  float tu, tv, tA, tB;  // target SIP argument and value at the anchor (FP32)
};

// Target forward SIP (A, B) at (u, v) in FP32 at the plan's degree: by the runtime loop, or
// (UNROLL, for the hot rows of target-SIP kernels) degrees 2-5 unrolled. The FMA sequence is the
// same either way, so the results are equal bits.
template <bool UNROLL = false>
__device__ __forceinline__ void tsip_pair(const FwdPlan& P, float u, float v, float& fa,
                                          float& fb) {
  if (!UNROLL) {
    horner_pair_rt<float>(P.tsip_f[0], P.tsip_f[1], P.tsip_deg, u, v, fa, fb);
    return;
  }
  switch (P.tsip_deg) {
    case 2: horner_pair<2, float>(P.tsip_f[0], P.tsip_f[1], u, v, fa, fb); break;
    case 3: horner_pair<3, float>(P.tsip_f[0], P.tsip_f[1], u, v, fa, fb); break;
    case 4: horner_pair<4, float>(P.tsip_f[0], P.tsip_f[1], u, v, fa, fb); break;
    case 5: horner_pair<5, float>(P.tsip_f[0], P.tsip_f[1], u, v, fa, fb); break;
    default: horner_pair_rt<float>(P.tsip_f[0], P.tsip_f[1], P.tsip_deg, u, v, fa, fb); break;
  }
}

// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats with |lo| at
// most half an ulp of hi (about 48 significant bits). Error-free transformations: Knuth's
// TwoSum, the fast form of Dekker's sum (|a| >= |b|) and the FMA form of Dekker's product;
// the addition is the simple one (TwoSum of the high parts, the low parts added in FP32):
// its error, about 2^-48 of |a| + |b|, is far below the 2^-24 relative resolution that the
// anchors' positions need after cancellation (a few 1e-11 px at 4096 px). Every step is an
// explicitly rounded intrinsic, so no contraction or reassociation can change a result
// between the kernels that build anchors.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_quick_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = ff_two_sum(a.hi, b.hi);
  return ff_quick_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_quick_sum(p, e);
}
__device__ __forceinline__ FF ff_load(const float* hl) { return {hl[0], hl[1]}; }

// Anchor without target SIP, in double-float on the FP32 pipes (the FP64 pipe is narrow on
// this part and the anchor is a chain of dependent operations): the homography numerators
// and denominator at the anchor, 1 / h2 by one Newton step from the FP32 reciprocal (24 -> 48
// bits), the source position and its split into integer and fractional parts.
__device__ __forceinline__ void make_anchor_ff(const FwdPlan& P, float X, float Y, Anchor& a) {
  const FF u = ff_add(FF{X, 0.f}, ff_neg(ff_load(P.crpix_t_ff[0])));
  const FF v = ff_add(FF{Y, 0.f}, ff_neg(ff_load(P.crpix_t_ff[1])));
  a.tu = u.hi;
  a.tv = v.hi;
  a.tA = a.tB = 0.f;
  FF h[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    h[i] = ff_add(ff_add(ff_mul(ff_load(P.G_ff[i][0]), u), ff_mul(ff_load(P.G_ff[i][1]), v)),
                  ff_load(P.G_ff[i][2]));
  // 1 / h2 to about 2^-47: the FMA residual of the correctly rounded FP32 reciprocal (exact
  // for the high part), the low part's term and one Newton correction in FP32
  const float r0 = __frcp_rn(h[2].hi);
  const float e = fmaf(-h[2].lo, r0, fmaf(-h[2].hi, r0, 1.f));
  const FF r = ff_quick_sum(r0, __fmul_rn(r0, e));
  const FF U0 = ff_mul(h[0], r), V0 = ff_mul(h[1], r);
  const float U0f = U0.hi, V0f = V0.hi;
  const float g20 = P.G_ff[2][0][0], g21 = P.G_ff[2][1][0];
  a.a0 = fmaf(-U0f, g20, P.G_ff[0][0][0]);
  a.a1 = fmaf(-U0f, g21, P.G_ff[0][1][0]);
  a.b0 = fmaf(-V0f, g20, P.G_ff[1][0][0]);
  a.b1 = fmaf(-V0f, g21, P.G_ff[1][1][0]);
  a.g20 = g20;
  a.g21 = g21;
  a.h2 = h[2].hi;
  a.U0 = U0f;
  a.V0 = V0f;
  const FF X0 = ff_add(U0, ff_load(P.crpix_s_ff[0]));
  const FF Y0 = ff_add(V0, ff_load(P.crpix_s_ff[1]));
  // floor of hi + lo: floor(hi), one less when hi is an integer and lo < 0; exact while
  // |hi| < 2^24, and anchors farther out than that leave their cell uncovered
  const bool finite = fabsf(X0.hi) < 16777216.f && fabsf(Y0.hi) < 16777216.f;
  float fx = floorf(X0.hi), fy = floorf(Y0.hi);
  if (X0.hi == fx && X0.lo < 0.f) fx = __fsub_rn(fx, 1.f);
  if (Y0.hi == fy && Y0.lo < 0.f) fy = __fsub_rn(fy, 1.f);
  a.bx = finite ? int32_t(fx) : 0;
  a.by = finite ? int32_t(fy) : 0;
  a.f0x = finite ? __fadd_rn(__fsub_rn(X0.hi, fx), X0.lo) : 0.f;
  a.f0y = finite ? __fadd_rn(__fsub_rn(Y0.hi, fy), Y0.lo) : 0.f;
  if (!finite || !(h[2].hi > 0.f)) a.h2 = -1.f;  // the whole cell is treated as uncovered
}

// Anchor at target pixel position (X, Y) (absolute, exactly representable: integers or
// quarter-integers).
__device__ __forceinline__ void make_anchor(const FwdPlan& P, float X, float Y, Anchor& a) {
  if (P.identity) {
    // the translation in FP64: exact for the integer and half-integer shifts of dithers
    const double xs = __dadd_rn(double(X), P.shift[0]), ys = __dadd_rn(double(Y), P.shift[1]);
    const double fx = floor(xs), fy = floor(ys);
    a.bx = int32_t(fx);
    a.by = int32_t(fy);
    a.f0x = float(__dsub_rn(xs, fx));
    a.f0y = float(__dsub_rn(ys, fy));
    // true intermediate offsets of the anchor (the same on both sides; used only by the
    // adjoint's chain rule)
    a.U0 = float(double(X) - P.crpix_t[0]);
    a.V0 = float(double(Y) - P.crpix_t[1]);
    a.a0 = 1.f; a.a1 = 0.f; a.b0 = 0.f; a.b1 = 1.f;
    a.g20 = a.g21 = 0.f;
    a.h2 = 1.f;
    a.tu = a.tv = a.tA = a.tB = 0.f;
    return;
  }
  if (P.tsip_deg <= 0) {
    make_anchor_ff(P, X, Y, a);
    return;
  }
  // with target SIP: FP64 where absolute positions need it (the target SIP, the homography at
  // the anchor and the anchor's source position); the local expansion follows in FP32
  const double u = __dsub_rn(double(X), P.crpix_t[0]);
  const double v = __dsub_rn(double(Y), P.crpix_t[1]);
  double p = u, q = v;
  a.tu = float(u);
  a.tv = float(v);
  a.tA = a.tB = 0.f;
  if (P.tsip_deg > 0) {
    double fa, fb;
    horner_pair_rt<double>(P.tsip_d[0], P.tsip_d[1], P.tsip_deg, u, v, fa, fb);
    p = __dadd_rn(p, fa);
    q = __dadd_rn(q, fb);
    float ga, gb;
    tsip_pair(P, a.tu, a.tv, ga, gb);
    a.tA = ga;
    a.tB = gb;
  }
  const double h0 = fma(P.G[0][0], p, fma(P.G[0][1], q, P.G[0][2]));
  const double h1 = fma(P.G[1][0], p, fma(P.G[1][1], q, P.G[1][2]));
  const double h2 = fma(P.G[2][0], p, fma(P.G[2][1], q, P.G[2][2]));
  // 1/h2: FP32 estimate refined by two Newton steps to full FP64 accuracy
  double r = double(__frcp_rn(float(h2)));
  r = fma(r, fma(-h2, r, 1.0), r);
  r = fma(r, fma(-h2, r, 1.0), r);
  // explicit roundings (no contraction of a product into a later sum: every kernel that builds
  // anchors must get the same bits)
  const double U0 = __dmul_rn(h0, r), V0 = __dmul_rn(h1, r);
  const float U0f = float(U0), V0f = float(V0);
  const float g20 = float(P.G[2][0]), g21 = float(P.G[2][1]);
  a.a0 = fmaf(-U0f, g20, float(P.G[0][0]));
  a.a1 = fmaf(-U0f, g21, float(P.G[0][1]));
  a.b0 = fmaf(-V0f, g20, float(P.G[1][0]));
  a.b1 = fmaf(-V0f, g21, float(P.G[1][1]));
  a.g20 = g20;
  a.g21 = g21;
  a.h2 = float(h2);
  a.U0 = U0f;
  a.V0 = V0f;
  const double X0 = __dadd_rn(U0, P.crpix_s[0]), Y0 = __dadd_rn(V0, P.crpix_s[1]);
  const double fx = floor(X0), fy = floor(Y0);
  const bool finite = isfinite(X0) && isfinite(Y0) && fabs(X0) < 1e9 && fabs(Y0) < 1e9;
  a.bx = finite ? int32_t(fx) : 0;
  a.by = finite ? int32_t(fy) : 0;
  a.f0x = finite ? float(__dsub_rn(X0, fx)) : 0.f;
  a.f0y = finite ? float(__dsub_rn(Y0, fy)) : 0.f;
  if (!finite || !(h2 > 0.0)) a.h2 = -1.f;  // the whole cell is treated as uncovered
}

// FP32 per-pixel part of the split path. (dx, dy): target pixel minus anchor position.
// Writes the source position relative to (bx, by); returns false if undefined.
// cab: the packed (AP, BP) coefficient pairs (IDEG > 0 with PAIRS: an unrolled FP32x2 Horner
// of that degree over cab, which may live in registers; IDEG > 0 without PAIRS: the same in
// scalar FMAs over the plan's arrays; IDEG < 0: runtime degree P.isip_deg over the plan's
// arrays; IDEG == 0: no inverse polynomial). All forms run the same FMA sequence, so they
// give the same bits. The rarely used target-SIP and Newton branches read the plan P; the
// Newton step's forward SIP has degree FDEG (the plan's padded degree) or, with FDEG < 0, the
// runtime degree; TSIP_UNROLL selects the unrolled target-SIP evaluation (same bits).
// geo (nullable) receives (du, dv, eu, ev) for the adjoint.
template <int IDEG, bool PAIRS = true, int FDEG = -1, bool TSIP_UNROLL = false>
__device__ __forceinline__ bool split_coords_core(const FwdPlan& P, const float2* cab,
                                                  bool identity, bool tsip, bool newton,
                                                  const Anchor& a, float dx, float dy, float& xr,
                                                  float& yr, float* geo = nullptr) {
  if (identity) {
    xr = __fadd_rn(a.f0x, dx);
    yr = __fadd_rn(a.f0y, dy);
    if (geo) {
      geo[0] = geo[2] = dx;
      geo[1] = geo[3] = dy;
    }
    return true;
  }
  // Every operation is an explicit rounding (fmaf, __fmul_rn, __fadd_rn, ...): the compiler
  // may not contract a product into a later sum, so every kernel that evaluates this (forward
  // fast and general rows, coordinate output, adjoint) produces the same bits.
  float dp = dx, dq = dy;
  if (tsip) {
    float fa, fb;
    tsip_pair<TSIP_UNROLL>(P, __fadd_rn(a.tu, dx), __fadd_rn(a.tv, dy), fa, fb);
    dp = __fadd_rn(dx, __fsub_rn(fa, a.tA));
    dq = __fadd_rn(dy, __fsub_rn(fb, a.tB));
  }
  const float nu = fmaf(a.a0, dp, __fmul_rn(a.a1, dq));
  const float nv = fmaf(a.b0, dp, __fmul_rn(a.b1, dq));
  const float den = fmaf(a.g20, dp, fmaf(a.g21, dq, a.h2));
  const float rcp = __fdividef(1.f, den);
  // (du, dv) = (nu, nv) / den, fused into each use: U = U0 + du, the position f0 + (ga + du)
  const float Uq = fmaf(nu, rcp, a.U0), Vq = fmaf(nv, rcp, a.V0);
  float ga = 0.f, gb = 0.f;  // inverse SIP AP/BP at (U, V)
  if (IDEG > 0 && PAIRS) {
    const float2 g = horner_pair2<(IDEG > 0 ? IDEG : 1)>(cab, Uq, Vq);
    ga = g.x;
    gb = g.y;
  } else if (IDEG > 0) {
    // scalar FMAs reading the plan directly (constant-bank operands for a kernel parameter)
    horner_pair<(IDEG > 0 ? IDEG : 1), float>(P.isip_f[0], P.isip_f[1], Uq, Vq, ga, gb);
  } else if (IDEG < 0 && P.isip_deg > 0) {
    horner_pair_rt<float>(P.isip_f[0], P.isip_f[1], P.isip_deg, Uq, Vq, ga, gb);
  }
  if (!newton) {
    xr = fmaf(nu, rcp, __fadd_rn(a.f0x, ga));
    yr = fmaf(nv, rcp, __fadd_rn(a.f0y, gb));
    if (geo) {
      const float du = __fmul_rn(nu, rcp), dv = __fmul_rn(nv, rcp);
      geo[0] = du;  // source intermediate offsets before the inverse SIP, relative to (U0, V0)
      geo[1] = dv;
      geo[2] = __fadd_rn(du, ga);  // ... and after it
      geo[3] = __fadd_rn(dv, gb);
    }
    return den > 0.f && a.h2 > 0.f;
  }
  const float du = __fmul_rn(nu, rcp), dv = __fmul_rn(nv, rcp);
  float eu = __fadd_rn(du, ga), ev = __fadd_rn(dv, gb);
  // Newton on e = u - U0: e + A(U0 + e) = du, started from the AP/BP estimate.
  for (int it = 0; it < P.newton_iters; ++it) {
    float A, Au, Av, B, Bu, Bv;
    const float Ue = __fadd_rn(a.U0, eu), Ve = __fadd_rn(a.V0, ev);
    poly_grad<FDEG, float>(P.fsip_f[0], P.fsip_deg, Ue, Ve, A, Au, Av);
    poly_grad<FDEG, float>(P.fsip_f[1], P.fsip_deg, Ue, Ve, B, Bu, Bv);
    const float ru = __fadd_rn(__fsub_rn(eu, du), A), rv = __fadd_rn(__fsub_rn(ev, dv), B);
    const float j00 = __fadd_rn(1.f, Au), j11 = __fadd_rn(1.f, Bv);
    const float det = fmaf(j00, j11, -__fmul_rn(Av, Bu));
    const float inv = __fdividef(1.f, det);
    eu = __fsub_rn(eu, __fmul_rn(fmaf(j11, ru, -__fmul_rn(Av, rv)), inv));
    ev = __fsub_rn(ev, __fmul_rn(fmaf(j00, rv, -__fmul_rn(Bu, ru)), inv));
  }
  xr = __fadd_rn(a.f0x, eu);
  yr = __fadd_rn(a.f0y, ev);
  if (geo) {
    geo[0] = du;
    geo[1] = dv;
    geo[2] = eu;
    geo[3] = ev;
  }
  return den > 0.f && a.h2 > 0.f;
}

__device__ __forceinline__ bool plan_newton(const FwdPlan& P) {
  return (P.flags & DFR_EXACT_INVERSE) && P.fsip_deg > 0;
}

// Plan-reading form (runtime degree), used where the plan is read once per pixel anyway.
template <int IDEG>
__device__ __forceinline__ bool split_coords(const FwdPlan& P, const Anchor& a, float dx,
                                             float dy, float& xr, float& yr,
                                             float* geo = nullptr) {
  static_assert(IDEG <= 0, "the plan-reading form evaluates the inverse SIP at runtime degree");
  return split_coords_core<IDEG>(P, nullptr, P.identity != 0, P.tsip_deg > 0, plan_newton(P), a,
                                 dx, dy, xr, yr, geo);
}

// ---------------------------------------------------------------- TMA and mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: gives up after kWaitNs of the global timer (or 2^26 polls,
// whichever comes first), then, when `flag`, sets the device status word; returns false.
constexpr uint64_t kWaitNs = 500000000ull;  // 0.5 s: far beyond any copy's latency
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, bool flag = true) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) break;
  }
  if (flag) atomicOr(&g_status, kStatusTimeout);
  return false;
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// A tensor map that sits in global memory and was rewritten (by a copy) since the TMA unit
// last read it must be re-acquired by the tensormap proxy before use; without this a TMA load
// can use a stale cached descriptor from an earlier launch.
__device__ __forceinline__ void fence_tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                   reinterpret_cast<uint64_t>(map))
               : "memory");
}

// 2-D tiled TMA load of the box at (x, y) (x a multiple of 4 floats) into shared memory.
__device__ __forceinline__ void tma_load_2d(float* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t x, int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

}  // namespace dfr
