// 1-D SAD (Sec. "1D Signal Fitting"): the soft partition of unity of
// Sec. 4.2 over a line.  A batch of independent signals, each with its own N
// sites {p, c, log tau, r} and L samples (sample k at x = k + 0.5, s = 1/L):
//   l_i(x) = tau_i s (r_i - |x - p_i|),
// the value at x is the softmax blend of the K sites of largest logit (ties to
// the smaller index; K >= N blends all sites), trained with the MSE loss and
// Adam.
//
// One block per signal, 256 threads, the signal's sites in shared memory:
//  pass 1 (sample-major, chunks of samples): each sample's logits over all N
//    sites, its top-K set (keys of the propagation's order: logit descending,
//    index ascending), max logit m, 1/Z and blend; residual -> g = 2 (c - y) / L;
//    per sample {m, 1/Z, g, g cbar, K-th key} parked in shared memory;
//  pass 2 (site-major): each site's threads walk the chunk's samples,
//    recompute the site's logit (the same fp32 operations, so the same key),
//    and where the site is in the sample's set add w g, delta, delta l and
//    delta sign(x - p) (delta = w g (c_i - cbar) = dL/dl_i) in a fixed
//    order -- no atomics;
//  then the partial sums of each site's threads (fixed order), the chain rule
//  (dl/dc = w, dl/dlog tau = l, dl/dr = tau s, dl/dp = tau s sign(x - p), 0 at
//  the kink x = p) and Adam, with the per-signal loss from a fixed-order
//  block sum.
#include <cmath>

#include "sad_device.cuh"
#include "sad_host.h"
#include "sad_topk.cuh"

namespace sad {

constexpr int k1dThreads = 256;
constexpr int k1dMaxN = 1024;
constexpr int k1dMaxKSel = 16;  // K < N: the selected set is kept in registers
constexpr int k1dChunk = 1024;  // samples per pass

struct Sad1dAdam {
  float lr[4];
  float beta1, beta2, eps, log_tau_min, log_tau_max;
  float bc1, bc2;  // 1 - beta1^t, 1 - beta2^t
};

struct Sad1dShared {
  float p[k1dMaxN], c[k1dMaxN], ts[k1dMaxN], tr[k1dMaxN];
  float sm[k1dChunk], siz[k1dChunk], sg[k1dChunk], sgc[k1dChunk];
  uint64_t thr[k1dChunk];
  float red[k1dThreads / 32];
  float part[4][k1dThreads];
};

// logit of site i at x (one fixed fp32 form, used by both passes)
__device__ __forceinline__ float logit1d(const Sad1dShared& S, int i, float x) {
  return __fsub_rn(S.tr[i], __fmul_rn(S.ts[i], fabsf(__fsub_rn(x, S.p[i]))));
}

// Pass 1 for one sample: blend over the top-K set (or all sites).  Returns the
// blend; m, iz and thr describe the set.
template <bool ALL, int KS>
__device__ __forceinline__ float sample_blend(const Sad1dShared& S, int N, int K, float x, float& m,
                                              float& iz, uint64_t& thr) {
  float z = 0.f, cb = 0.f;
  m = -INFINITY;
  if (ALL) {
    for (int i = 0; i < N; ++i) {
      const float l = logit1d(S, i, x);
      if (l > m) {
        const float a = __expf(m - l);
        z *= a;
        cb *= a;
        m = l;
      }
      const float b = __expf(l - m);
      z += b;
      cb += b * S.c[i];
    }
    thr = 0ull;  // every site's key is above 0
  } else {
    uint64_t v[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) v[k] = 0ull;
    for (int i = 0; i < N; ++i) {
      const uint64_t key = make_key(logit1d(S, i, x), static_cast<uint32_t>(i));
      if (key > v[KS - 1]) list_insert<KS>(v, key);
    }
    // the K best (K <= KS): v[0..K-1]; the K-th key is the set's threshold
    m = key_logit(v[0]);
    thr = v[0];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      if (k < K && v[k] != 0ull) {
        const float l = key_logit(v[k]);
        const float b = __expf(l - m);
        z += b;
        cb += b * S.c[key_id(v[k])];
        thr = v[k];
      }
    }
  }
  iz = z > 0.f ? 1.f / z : 0.f;
  return cb * iz;
}

template <bool ALL, int KS>
__global__ void __launch_bounds__(k1dThreads) k_sad1d(float* __restrict__ params, float* __restrict__ mo,
                                                      float* __restrict__ vo, const float* __restrict__ target,
                                                      float* __restrict__ values, float* __restrict__ loss,
                                                      float* __restrict__ grads_out, int B, int N, int L,
                                                      int K, Sad1dAdam A, bool train) {
  __shared__ Sad1dShared S;
  const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const size_t BN = static_cast<size_t>(B) * N;
  const size_t base = static_cast<size_t>(b) * N;
  const float s = 1.0f / static_cast<float>(L);
  for (int i = t; i < N; i += k1dThreads) {
    const float pi = params[base + i];
    const float ts = __fmul_rn(__expf(params[2 * BN + base + i]), s);
    S.p[i] = pi;
    S.c[i] = params[BN + base + i];
    S.ts[i] = ts;
    S.tr[i] = __fmul_rn(ts, params[3 * BN + base + i]);
  }
  __syncthreads();
  // pass-2 work split: R threads per site (N <= 256), or sites strided over
  // the threads (N > 256)
  const int R = N <= k1dThreads ? k1dThreads / N : 1;
  const int site0 = N <= k1dThreads ? t % N : t;
  const int part = N <= k1dThreads ? t / N : 0;
  const bool p2 = N <= k1dThreads ? t < N * R : t < N;
  float acc[4][k1dMaxN / k1dThreads] = {};
  float lsum = 0.f;
  const float* y = target ? target + static_cast<size_t>(b) * L : nullptr;
  for (int x0 = 0; x0 < L; x0 += k1dChunk) {
    const int nx = min(k1dChunk, L - x0);
    for (int k = t; k < nx; k += k1dThreads) {
      const float x = static_cast<float>(x0 + k) + 0.5f;
      float m, iz;
      uint64_t thr;
      const float v = sample_blend<ALL, KS>(S, N, K, x, m, iz, thr);
      if (!train) {
        values[static_cast<size_t>(b) * L + x0 + k] = v;
        continue;
      }
      const float r = v - y[x0 + k];
      lsum += r * r;
      const float g = 2.f * r * s;
      S.sm[k] = m;
      S.siz[k] = iz;
      S.sg[k] = g;
      S.sgc[k] = g * v;
      S.thr[k] = thr;
    }
    if (!train) continue;
    __syncthreads();
    if (p2) {
#pragma unroll
      for (int j = 0; j < k1dMaxN / k1dThreads; ++j) {
        const int i = j * k1dThreads + site0;
        if (i >= N) break;
        const float ci = S.c[i], pi = S.p[i];
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int k = part; k < nx; k += R) {
          const float x = static_cast<float>(x0 + k) + 0.5f;
          const float l = logit1d(S, i, x);
          if (make_key(l, static_cast<uint32_t>(i)) < S.thr[k]) continue;  // not in the sample's set
          const float w = __expf(l - S.sm[k]) * S.siz[k];
          const float wg = w * S.sg[k];
          const float d = w * (S.sg[k] * ci - S.sgc[k]);
          const float dx = x - pi;
          a0 += wg;
          a1 += d;
          a2 += d * l;
          a3 += dx > 0.f ? d : (dx < 0.f ? -d : 0.f);
        }
        acc[0][j] += a0;
        acc[1][j] += a1;
        acc[2][j] += a2;
        acc[3][j] += a3;
      }
    }
    __syncthreads();
  }
  if (!train) return;
  // per-signal loss: fixed-order block sum
  float v = lsum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) S.red[warp] = v;
  // each site's R partial sums, in order of the part index
#pragma unroll
  for (int j = 0; j < k1dMaxN / k1dThreads; ++j) {
    if (j * k1dThreads >= N) break;  // uniform over the block
    __syncthreads();
    if (p2 && j * k1dThreads + site0 < N)
      for (int q = 0; q < 4; ++q) S.part[q][t] = acc[q][j];
    __syncthreads();
    const int i = j * k1dThreads + t;
    if (t < k1dThreads && i < N && (N > k1dThreads || t < N)) {
      float sum[4] = {0.f, 0.f, 0.f, 0.f};
      for (int q = 0; q < 4; ++q)
        for (int r = 0; r < R; ++r) sum[q] += S.part[q][r * N + t];
      // chain rule: dL/dc, dL/dp, dL/dlog tau, dL/dr
      const float ts = S.ts[i];
      float g[4];
      g[1] = sum[0];
      g[0] = ts * sum[3];
      g[2] = sum[2];
      g[3] = ts * sum[1];
      const size_t q0 = base + i;
      if (grads_out)
        for (int pl = 0; pl < 4; ++pl) grads_out[pl * BN + q0] = g[pl];
      // Adam (Kingma & Ba 2015), p and r in normalised units
      float pv[4];
      for (int pl = 0; pl < 4; ++pl) {
        const bool norm = pl == 0 || pl == 3;
        const float gj = norm ? g[pl] / s : g[pl];
        const float mj = A.beta1 * mo[pl * BN + q0] + (1.f - A.beta1) * gj;
        const float vj = A.beta2 * vo[pl * BN + q0] + (1.f - A.beta2) * gj * gj;
        mo[pl * BN + q0] = mj;
        vo[pl * BN + q0] = vj;
        const float step = A.lr[pl] * (mj / A.bc1) / (sqrtf(vj / A.bc2) + A.eps);
        pv[pl] = params[pl * BN + q0] - (norm ? step / s : step);
      }
      const float Lf = static_cast<float>(L);
      pv[0] = fminf(fmaxf(pv[0], 0.f), Lf);
      pv[3] = fminf(fmaxf(pv[3], 0.f), Lf);
      pv[2] = fminf(fmaxf(pv[2], A.log_tau_min), A.log_tau_max);
      for (int pl = 0; pl < 4; ++pl) params[pl * BN + q0] = pv[pl];
    }
  }
  if (t == 0) {
    float sum = 0.f;
    for (int w = 0; w < k1dThreads / 32; ++w) sum += S.red[w];
    loss[b] = sum * s;
  }
}

static int sad1d_check(int32_t B, int32_t N, int32_t L, int32_t K, const char* name) {
  if (B < 1 || N < 1 || L < 1) return einval("%s: need B, N, L >= 1", name);
  if (N > k1dMaxN) return einval("%s: at most %d sites per signal", name, k1dMaxN);
  if (static_cast<int64_t>(B) * N > 0x7fffffff || static_cast<int64_t>(B) * L > (int64_t(1) << 40))
    return einval("%s: batch too large", name);
  if (K < 1) return einval("%s: K must be >= 1", name);
  if (K < N && K > k1dMaxKSel) return einval("%s: K < N needs K <= %d", name, k1dMaxKSel);
  return SAD_OK;
}

static void launch1d(float* params, float* m, float* v, const float* target, float* values, float* loss,
                     float* grads_out, int B, int N, int L, int K, const Sad1dAdam& A, bool train,
                     cudaStream_t st) {
  TraceScope tr_(st, train ? "k_sad1d_step" : "k_sad1d_render");
  if (K >= N) {
    k_sad1d<true, 1><<<B, k1dThreads, 0, st>>>(params, m, v, target, values, loss, grads_out, B, N, L, K, A, train);
  } else if (K <= 4) {
    k_sad1d<false, 4><<<B, k1dThreads, 0, st>>>(params, m, v, target, values, loss, grads_out, B, N, L, K, A, train);
  } else if (K <= 8) {
    k_sad1d<false, 8><<<B, k1dThreads, 0, st>>>(params, m, v, target, values, loss, grads_out, B, N, L, K, A, train);
  } else {
    k_sad1d<false, 16><<<B, k1dThreads, 0, st>>>(params, m, v, target, values, loss, grads_out, B, N, L, K, A, train);
  }
}

}  // namespace sad

using namespace sad;

extern "C" {

int sad1d_render(const float* params, int32_t B, int32_t N, int32_t L, int32_t K, float* values,
                 void* stream) {
  if (int e = sad1d_check(B, N, L, K, "sad1d_render")) return e;
  if (!params || !values) return einval("sad1d_render: null pointer");
  Sad1dAdam A{};
  launch1d(const_cast<float*>(params), nullptr, nullptr, nullptr, values, nullptr, nullptr, B, N, L, K, A,
           false, as_stream(stream));
  return check_launch("k_sad1d_render");
}

int sad1d_train_step(float* params, float* m, float* v, int32_t B, int32_t N, int32_t L, int32_t K,
                     const float* target, float* loss, const sad1d_adam_hparams* hp, int32_t t,
                     float* grads_out, void* stream) {
  if (int e = sad1d_check(B, N, L, K, "sad1d_train_step")) return e;
  if (!params || !m || !v || !target || !loss || !hp) return einval("sad1d_train_step: null pointer");
  if (t < 1) return einval("sad1d_train_step: the Adam step t starts at 1");
  if (!(hp->log_tau_min <= hp->log_tau_max)) return einval("sad1d_train_step: bad log_tau range");
  Sad1dAdam A;
  for (int j = 0; j < 4; ++j) A.lr[j] = hp->lr[j];
  A.beta1 = hp->beta1;
  A.beta2 = hp->beta2;
  A.eps = hp->eps;
  A.log_tau_min = hp->log_tau_min;
  A.log_tau_max = hp->log_tau_max;
  A.bc1 = static_cast<float>(1.0 - std::pow(static_cast<double>(hp->beta1), t));
  A.bc2 = static_cast<float>(1.0 - std::pow(static_cast<double>(hp->beta2), t));
  launch1d(params, m, v, target, nullptr, loss, grads_out, B, N, L, K, A, true, as_stream(stream));
  return check_launch("k_sad1d_step");
}

}  // extern "C"
