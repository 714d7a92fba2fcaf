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

// Tau diffusion (App. "Tau Diffusion"): one Jacobi step mixing each active
// site's log tau gradient with the mean over the other valid, active sites
// listed at the pixel that contains it.
__global__ void k_tau_diffusion(const float* __restrict__ params, int cap, int H, int W, int K,
                                const uint32_t* __restrict__ map, float lam,
                                const float* __restrict__ g_in, float* __restrict__ g_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  const float gi = g_in[i];
  const float x = params[PX * c + i];
  if (!(x >= 0.f)) {
    g_out[i] = gi;
    return;
  }
  int col = static_cast<int>(floorf(x)), row = static_cast<int>(floorf(params[PY * c + i]));
  col = col < 0 ? 0 : (col >= W ? W - 1 : col);
  row = row < 0 ? 0 : (row >= H ? H - 1 : row);
  const size_t P = static_cast<size_t>(H) * W;
  const size_t q = static_cast<size_t>(row) * W + col;
  float sum = 0.f;
  int n = 0;
  for (int k = 0; k < K; ++k) {
    const uint32_t j = map[(k >> 2) * P * 4 + q * 4 + (k & 3)];
    if (j >= static_cast<uint32_t>(cap) || j == static_cast<uint32_t>(i)) continue;
    if (!(params[PX * c + j] >= 0.f)) continue;
    sum += g_in[j];
    ++n;
  }
  g_out[i] = n ? (1.f - lam) * gi + lam * (sum / static_cast<float>(n)) : gi;
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

extern "C" int sad_tau_diffusion(const float* params, int32_t capacity, int32_t H, int32_t W,
                                 int32_t K, const uint32_t* map, float lambda,
                                 const float* g_logtau, float* g_out, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (capacity == 0) return SAD_OK;
  if (!params || !map || !g_logtau || !g_out) return einval("sad_tau_diffusion: null pointer");
  if (g_logtau == g_out) return einval("sad_tau_diffusion: g_out must not alias g_logtau (Jacobi step)");
  if (!(lambda >= 0.f && lambda <= 1.f)) return einval("sad_tau_diffusion: lambda must be in [0, 1]");
  cudaStream_t st = as_stream(stream);
  {
    TraceScope tr_(st, "k_tau_diffusion");
    k_tau_diffusion<<<(capacity + 255) / 256, 256, 0, st>>>(params, capacity, H, W, K, map, lambda,
                                                            g_logtau, g_out);
  }
  return check_launch("k_tau_diffusion");
}
