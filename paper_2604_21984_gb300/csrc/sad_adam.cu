// Adam step with the paper's clamps and direction re-normalisation (Sec. 6.1).
#include <cmath>

#include "sad_device.cuh"
#include "sad_host.h"

namespace sad {

struct AdamArgs {
  float lr[kNParams];
  float beta1, beta2, eps, bc1, bc2;
  float lo[kNParams], hi[kNParams];
  float inv_s;
};

__global__ void k_adam(float* __restrict__ params, const float* __restrict__ grads,
                       float* __restrict__ m, float* __restrict__ v, int cap, AdamArgs A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  if (!(params[PX * c + i] >= 0.f)) return;  // inactive
  float p[kNParams];
#pragma unroll
  for (int j = 0; j < kNParams; ++j) {
    const size_t o = j * c + i;
    const bool norm_units = (j == PX || j == PY || j == PR);
    const float gj = norm_units ? grads[o] * A.inv_s : grads[o];
    const float mj = A.beta1 * m[o] + (1.f - A.beta1) * gj;
    const float vj = A.beta2 * v[o] + (1.f - A.beta2) * gj * gj;
    m[o] = mj;
    v[o] = vj;
    const float mhat = mj / A.bc1, vhat = vj / A.bc2;
    float step = A.lr[j] * mhat / (sqrtf(vhat) + A.eps);
    if (norm_units) step *= A.inv_s;
    p[j] = fminf(fmaxf(params[o] - step, A.lo[j]), A.hi[j]);
  }
  const float n2 = p[PUX] * p[PUX] + p[PUY] * p[PUY];
  if (n2 > 0.f) {
    const float inv = 1.f / sqrtf(n2);
    p[PUX] *= inv;
    p[PUY] *= inv;
  }
#pragma unroll
  for (int j = 0; j < kNParams; ++j) params[j * c + i] = p[j];
}

}  // namespace sad

using namespace sad;

extern "C" int sad_adam_step(float* params, const float* grads, float* m, float* v,
                             int32_t capacity, int32_t H, int32_t W, int32_t t,
                             const sad_adam_hparams* hp, void* stream) {
  if (int e = check_problem(capacity, H, W, 4, false)) return e;
  if (!hp) return einval("sad_adam_step: null hyper-parameters");
  if (t < 1) return einval("sad_adam_step: step t must be >= 1 (got %d)", t);
  if (capacity == 0) return SAD_OK;
  if (!params || !grads || !m || !v) return einval("sad_adam_step: null pointer");
  AdamArgs A;
  for (int j = 0; j < kNParams; ++j) {
    A.lr[j] = hp->lr[j];
    A.lo[j] = -INFINITY;
    A.hi[j] = INFINITY;
  }
  A.beta1 = hp->beta1;
  A.beta2 = hp->beta2;
  A.eps = hp->eps;
  A.bc1 = static_cast<float>(1.0 - std::pow(static_cast<double>(hp->beta1), t));
  A.bc2 = static_cast<float>(1.0 - std::pow(static_cast<double>(hp->beta2), t));
  A.inv_s = static_cast<float>(H > W ? H : W);
  A.lo[PX] = 0.f; A.hi[PX] = static_cast<float>(W);
  A.lo[PY] = 0.f; A.hi[PY] = static_cast<float>(H);
  A.lo[PLOGTAU] = hp->log_tau_min; A.hi[PLOGTAU] = hp->log_tau_max;
  A.lo[PR] = hp->r_min; A.hi[PR] = hp->r_max;
  A.lo[PA] = hp->a_min; A.hi[PA] = hp->a_max;
  A.lo[PB] = hp->b_min; A.hi[PB] = hp->b_max;
  for (int j = PCR; j <= PCB; ++j) {
    A.lo[j] = 0.f;
    A.hi[j] = 1.f;
  }
  const int bs = 256;
  k_adam<<<(capacity + bs - 1) / bs, bs, 0, as_stream(stream)>>>(params, grads, m, v, capacity, A);
  return check_launch("k_adam");
}
