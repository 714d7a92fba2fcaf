// Adam step of one site with the paper's clamps (Sec. 6.1), shared by the
// stand-alone Adam kernel and the fused training step.
#pragma once

#include "sad_device.cuh"

namespace sad {

struct AdamArgs {
  float lr[kNParams];
  float beta1, beta2, eps;
  float log_tau_min, log_tau_max, r_min, r_max, a_min, a_max, b_min, b_max;
};

__device__ __forceinline__ void adam_site_mv(float (&p)[kNParams], const float (&g)[kNParams],
                                             const float (&m0)[kNParams], const float (&v0)[kNParams],
                                             float* __restrict__ m, float* __restrict__ v, size_t c,
                                             size_t i, const AdamArgs& A, float bc1, float bc2,
                                             int H, int W);

// Bias-corrected Adam on the 11 planes of site i (planes of stride c) with
// gradient g: x, y and r step in normalised units (gradient / s, step * 1/s);
// then positions clamp to [0,W]x[0,H], log_tau/r/a/b to their ranges, colours
// to [0,1], and (ux,uy) is re-normalised.  bc1 = 1 - b1^t, bc2 = 1 - b2^t.
// p holds the site's parameters on entry and the updated ones on exit.
__device__ __forceinline__ void adam_site(float (&p)[kNParams], const float (&g)[kNParams],
                                          float* __restrict__ m, float* __restrict__ v, size_t c,
                                          size_t i, const AdamArgs& A, float bc1, float bc2,
                                          int H, int W) {
  float m0[kNParams], v0[kNParams];
#pragma unroll
  for (int j = 0; j < kNParams; ++j) {
    m0[j] = m[j * c + i];
    v0[j] = v[j * c + i];
  }
  adam_site_mv(p, g, m0, v0, m, v, c, i, A, bc1, bc2, H, W);
}

// adam_site with the site's m and v already loaded (m0, v0), so that a
// caller can issue those loads early.
__device__ __forceinline__ void adam_site_mv(float (&p)[kNParams], const float (&g)[kNParams],
                                             const float (&m0)[kNParams], const float (&v0)[kNParams],
                                             float* __restrict__ m, float* __restrict__ v, size_t c,
                                             size_t i, const AdamArgs& A, float bc1, float bc2,
                                             int H, int W) {
  const float inv_s = static_cast<float>(H > W ? H : W);
#pragma unroll
  for (int j = 0; j < kNParams; ++j) {
    const size_t o = j * c + i;
    const bool norm_units = (j == PX || j == PY || j == PR);
    const float gj = norm_units ? g[j] * inv_s : g[j];
    const float mj = A.beta1 * m0[j] + (1.f - A.beta1) * gj;
    const float vj = A.beta2 * v0[j] + (1.f - A.beta2) * gj * gj;
    m[o] = mj;
    v[o] = vj;
    const float mhat = mj / bc1, vhat = vj / bc2;
    float step = A.lr[j] * mhat / (sqrtf(vhat) + A.eps);
    if (norm_units) step *= inv_s;
    p[j] = p[j] - step;
  }
  p[PX] = fminf(fmaxf(p[PX], 0.f), static_cast<float>(W));
  p[PY] = fminf(fmaxf(p[PY], 0.f), static_cast<float>(H));
  p[PLOGTAU] = fminf(fmaxf(p[PLOGTAU], A.log_tau_min), A.log_tau_max);
  p[PR] = fminf(fmaxf(p[PR], A.r_min), A.r_max);
  p[PA] = fminf(fmaxf(p[PA], A.a_min), A.a_max);
  p[PB] = fminf(fmaxf(p[PB], A.b_min), A.b_max);
#pragma unroll
  for (int j = PCR; j <= PCB; ++j) p[j] = fminf(fmaxf(p[j], 0.f), 1.f);
  const float n2 = p[PUX] * p[PUX] + p[PUY] * p[PUY];
  if (n2 > 0.f) {
    const float inv = 1.f / sqrtf(n2);
    p[PUX] *= inv;
    p[PUY] *= inv;
  }
}

}  // namespace sad
