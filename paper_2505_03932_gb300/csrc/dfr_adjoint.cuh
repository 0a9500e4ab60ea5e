// Pieces shared by the adjoint kernels (per-pixel and tile-staged): the parameter layout, warp
// sums and the per-pixel chain rule to the source-WCS parameters.
#pragma once

#include "dfr_device.cuh"

namespace dfr {

constexpr float kR0f = 57.29577951308232f;

// A/B coefficients (1 <= p + q <= fd) of one polynomial in the padded parameter layout.
__host__ __device__ constexpr int nterms(int fd) { return fd > 0 ? (fd + 1) * (fd + 2) / 2 - 1 : 0; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Source CD, CD^-1 and tangent point in FP32 for the per-pixel chain rule.
struct ChainConst {
  float cd00, cd01, cd10, cd11, ci00, ci01, ci10, ci11, sd0, cd0;
};

__device__ __forceinline__ ChainConst chain_const(const FwdPlan& P) {
  ChainConst K;
  K.cd00 = float(P.cd_s[0][0]);
  K.cd01 = float(P.cd_s[0][1]);
  K.cd10 = float(P.cd_s[1][0]);
  K.cd11 = float(P.cd_s[1][1]);
  K.ci00 = float(P.cdinv_s[0][0]);
  K.ci01 = float(P.cdinv_s[0][1]);
  K.ci10 = float(P.cdinv_s[1][0]);
  K.ci11 = float(P.cdinv_s[1][1]);
  K.sd0 = float(P.sd0_s);
  K.cd0 = float(P.cd0_s);
  return K;
}

// Chain rule of one pixel from (gxs, gys) = dL/d(source position): lambda = (lu, lv) =
// dL/d(U, V) through the inverse SIP (M = I + d(AP, BP)/d(U, V), or the implicit-function
// derivative (I + J_AB)^-1 of the Newton inverse), then nu = CD^-T lambda = dL/d(u', v') and
// the CRVAL and CD terms c[0..5]. (U, V): intermediate offsets before the inverse SIP; (u, v):
// after it. IDEG / FDEG: the plan's padded inverse / forward SIP degrees, or -1 (runtime).
template <int IDEG, int FDEG>
__device__ __forceinline__ void chain_terms(const FwdPlan& P, const ChainConst& K, bool cov,
                                            bool exact, float gxs, float gys, float U, float V,
                                            float u, float v, float& lu, float& lv,
                                            float c[6]) {
  float m00 = 1.f, m01 = 0.f, m10 = 0.f, m11 = 1.f;
  if (cov) {
    if (exact) {
      float A, Au, Av, Bq, Bu, Bv;
      poly_grad<FDEG, float>(P.fsip_f[0], P.fsip_deg, u, v, A, Au, Av);
      poly_grad<FDEG, float>(P.fsip_f[1], P.fsip_deg, u, v, Bq, Bu, Bv);
      const float j00 = 1.f + Au, j01 = Av, j10 = Bu, j11 = 1.f + Bv;
      const float inv = __fdividef(1.f, fmaf(j00, j11, -j01 * j10));
      m00 = j11 * inv;
      m01 = -j01 * inv;
      m10 = -j10 * inv;
      m11 = j00 * inv;
    } else if (IDEG != 0 && P.isip_deg > 0) {
      float A, Au, Av, Bq, Bu, Bv;
      poly_grad<IDEG, float>(P.isip_f[0], P.isip_deg, U, V, A, Au, Av);
      poly_grad<IDEG, float>(P.isip_f[1], P.isip_deg, U, V, Bq, Bu, Bv);
      m00 = 1.f + Au;
      m01 = Av;
      m10 = Bu;
      m11 = 1.f + Bv;
    }
  }
  lu = fmaf(gxs, m00, gys * m10);
  lv = fmaf(gxs, m01, gys * m11);
  const float nx = fmaf(K.ci00, lu, K.ci10 * lv);
  const float ny = fmaf(K.ci01, lu, K.ci11 * lv);
  const float xi = fmaf(K.cd00, U, K.cd01 * V) / kR0f;
  const float eta = fmaf(K.cd10, U, K.cd11 * V) / kR0f;
  c[0] = nx * fmaf(-K.cd0, fmaf(xi, xi, 1.f), K.sd0 * eta) + ny * (-xi * fmaf(K.cd0, eta, K.sd0));
  c[1] = nx * (-xi * eta) + ny * (-fmaf(eta, eta, 1.f));
  c[2] = -nx * U;
  c[3] = -nx * V;
  c[4] = -ny * U;
  c[5] = -ny * V;
}

// The same chain rule with M given (its entries m00, m01, m10, m11): the CRVAL and CD terms
// from dL/d(source position) through M, CD^-1 and the TAN projection.
__device__ __forceinline__ void chain_terms_m(const ChainConst& K, float gxs, float gys, float U,
                                              float V, float m00, float m01, float m10,
                                              float m11, float& lu, float& lv, float c[6]) {
  lu = fmaf(gxs, m00, gys * m10);
  lv = fmaf(gxs, m01, gys * m11);
  const float nx = fmaf(K.ci00, lu, K.ci10 * lv);
  const float ny = fmaf(K.ci01, lu, K.ci11 * lv);
  const float xi = fmaf(K.cd00, U, K.cd01 * V) / kR0f;
  const float eta = fmaf(K.cd10, U, K.cd11 * V) / kR0f;
  c[0] = nx * fmaf(-K.cd0, fmaf(xi, xi, 1.f), K.sd0 * eta) + ny * (-xi * fmaf(K.cd0, eta, K.sd0));
  c[1] = nx * (-xi * eta) + ny * (-fmaf(eta, eta, 1.f));
  c[2] = -nx * U;
  c[3] = -nx * V;
  c[4] = -ny * U;
  c[5] = -ny * V;
}

}  // namespace dfr
