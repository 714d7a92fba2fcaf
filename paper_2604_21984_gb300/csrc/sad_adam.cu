// Adam step with the paper's clamps and direction re-normalisation (Sec. 6.1).
#include <cmath>

#include "sad_adam.cuh"
#include "sad_host.h"

namespace sad {

__global__ void k_adam(float* __restrict__ params, const float* __restrict__ grads,
                       float* __restrict__ m, float* __restrict__ v, int cap, int H, int W,
                       AdamArgs A, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  if (!(params[PX * c + i] >= 0.f)) return;  // inactive
  float p[kNParams], g[kNParams];
#pragma unroll
  for (int j = 0; j < kNParams; ++j) {
    p[j] = params[j * c + i];
    g[j] = grads[j * c + i];
  }
  adam_site(p, g, m, v, c, i, A, bc1, bc2, H, W);
#pragma unroll
  for (int j = 0; j < kNParams; ++j) params[j * c + i] = p[j];
}

AdamArgs adam_args(const sad_adam_hparams* hp) {
  AdamArgs A;
  for (int j = 0; j < kNParams; ++j) A.lr[j] = hp->lr[j];
  A.beta1 = hp->beta1;
  A.beta2 = hp->beta2;
  A.eps = hp->eps;
  A.log_tau_min = hp->log_tau_min;
  A.log_tau_max = hp->log_tau_max;
  A.r_min = hp->r_min;
  A.r_max = hp->r_max;
  A.a_min = hp->a_min;
  A.a_max = hp->a_max;
  A.b_min = hp->b_min;
  A.b_max = hp->b_max;
  return A;
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
  const AdamArgs A = adam_args(hp);
  const float bc1 = static_cast<float>(1.0 - std::pow(static_cast<double>(hp->beta1), t));
  const float bc2 = static_cast<float>(1.0 - std::pow(static_cast<double>(hp->beta2), t));
  const int bs = 256;
  { TraceScope tr_(as_stream(stream), "k_adam"); k_adam<<<(capacity + bs - 1) / bs, bs, 0, as_stream(stream)>>>(params, grads, m, v, capacity, H, W,
                                                                 A, bc1, bc2); }
  return check_launch("k_adam");
}
