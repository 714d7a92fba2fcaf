// Gradient-weighted site initialisation (Sec. 4.4, Eq. P_init).
//
// 1. |grad I| per pixel (central differences, fp32) and the exact sum of its
//    2^-32 fixed-point images (int64 atomics: order independent);
// 2. P_init(x) = (1-lam) g/S + lam/P and the Efraimidis-Spirakis key
//    E/P_init with E = -log U, U a 24-bit SplitMix64 draw at counter = pixel;
// 3. the n smallest keys (ties by pixel index) by a 4-pass, 8-bit radix
//    select on the key bits, then a stable compaction in pixel order;
// 4. sites at the selected pixel centres with a U[-0.25,0.25) jitter, the
//    target colour there and the fixed defaults; the rest inactive.
// Every step that decides which pixels are chosen is an explicitly rounded
// fp32 (or integer) operation, so the choice is reproducible.
#include "sad_device.cuh"
#include "sad_host.h"
#include "sad_select.cuh"

namespace sad {

// Reproducible fp32 natural log (positive normal inputs): x = 2^e m,
// m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1), log m = 2s + 2s(s^2/3 + s^4/5 +
// s^6/7 + s^8/9) (odd series of 2 atanh s, Horner in s^2), log x = e ln2_hi +
// (e ln2_lo + log m).  Method: Cody & Waite (1980).
__device__ __forceinline__ float log32_repro(float x) {
  const uint32_t bits = __float_as_uint(x);
  int e = static_cast<int>((bits >> 23) & 0xffu) - 127;
  float m = __uint_as_float((bits & 0x7fffffu) | (127u << 23));
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float ef = static_cast<float>(e);
  const float s = __fdiv_rn(__fsub_rn(m, 1.f), __fadd_rn(m, 1.f));
  const float s2 = __fmul_rn(s, s);
  float p = 0x1.c71c72p-4f;                       // 1/9
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.24924ap-3f);  // 1/7
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.99999ap-3f);  // 1/5
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.555556p-2f);  // 1/3
  p = __fmul_rn(p, s2);
  const float t = __fadd_rn(s, s);
  const float lm = __fadd_rn(t, __fmul_rn(t, p));
  return __fadd_rn(__fmul_rn(ef, 0x1.62e4p-1f), __fadd_rn(__fmul_rn(ef, 0x1.7f7d1cp-20f), lm));
}

struct InitState {
  unsigned long long gsum;  // sum of fixed-point |grad I|
  uint32_t pad[62];
  SelState sel;             // radix-select state
};

struct InitLayout {
  size_t state, g, keys, flag, scan, bsums, total;
  uint32_t nb;
};

static InitLayout init_layout(int H, int W) {
  InitLayout L{};
  const size_t P = static_cast<size_t>(H) * W;
  L.nb = static_cast<uint32_t>((P + 1023) / 1024);
  auto al = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
  size_t o = 0;
  L.state = o; o = al(o + sizeof(InitState));
  L.g = o;     o = al(o + 4 * P);
  L.keys = o;  o = al(o + 4 * P);
  L.flag = o;  o = al(o + 4 * P);
  L.scan = o;  o = al(o + 4 * P);
  L.bsums = o; o = al(o + 4 * (L.nb + 2));
  L.total = o;
  return L;
}

__global__ void k_init_state(InitState* __restrict__ st, uint32_t n) {
  uint32_t* w = reinterpret_cast<uint32_t*>(st);
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(InitState) / 4); i += blockDim.x) w[i] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) st->sel.need = n;
}

__global__ void k_init_grad(const float* __restrict__ img, int H, int W, float* __restrict__ g,
                            InitState* __restrict__ st) {
  __shared__ unsigned long long s_sum[8];
  const size_t P = static_cast<size_t>(H) * W;
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  unsigned long long fx = 0ull;
  if (i < P) {
    const int row = static_cast<int>(i / W), c = static_cast<int>(i % W);
    const int cR = min(c + 1, W - 1), cL = max(c - 1, 0);
    const int rD = min(row + 1, H - 1), rU = max(row - 1, 0);
    const float ix = cR - cL == 2 ? 0.5f : (cR - cL == 1 ? 1.f : 0.f);
    const float iy = rD - rU == 2 ? 0.5f : (rD - rU == 1 ? 1.f : 0.f);
    float g2 = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float dx = __fmul_rn(__fsub_rn(img[(static_cast<size_t>(row) * W + cR) * 3 + ch],
                                           img[(static_cast<size_t>(row) * W + cL) * 3 + ch]), ix);
      const float dy = __fmul_rn(__fsub_rn(img[(static_cast<size_t>(rD) * W + c) * 3 + ch],
                                           img[(static_cast<size_t>(rU) * W + c) * 3 + ch]), iy);
      g2 = __fadd_rn(g2, __fmul_rn(dx, dx));
      g2 = __fadd_rn(g2, __fmul_rn(dy, dy));
    }
    const float gv = __fsqrt_rn(g2);
    g[i] = gv;
    fx = static_cast<unsigned long long>(__float2ll_rn(__fmul_rn(gv, 4294967296.f)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fx += __shfl_down_sync(0xffffffffu, fx, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = fx;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) t += s_sum[w];
    atomicAdd(&st->gsum, t);
  }
}

__global__ void k_init_keys(const float* __restrict__ g, size_t P, float lam, uint64_t seed,
                            const InitState* __restrict__ st, uint32_t* __restrict__ keys) {
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float S = __double2float_rn(__ll2double_rn(static_cast<long long>(st->gsum)) *
                                    2.3283064365386963e-10);
  const float a = __fsub_rn(1.f, lam);
  const float b = __fdiv_rn(lam, static_cast<float>(P));
  const float t = S > 0.f ? __fdiv_rn(g[i], S) : 0.f;
  const float w = __fadd_rn(__fmul_rn(a, t), b);
  const uint64_t h = splitmix64_at(seed, static_cast<uint64_t>(i));
  const float u = __fadd_rn(static_cast<float>(h >> 40) * 0x1p-24f, 0x1p-24f);
  const float E = u == 1.f ? 0.f : -log32_repro(u);
  const float key = w > 0.f ? __fdiv_rn(E, w) : INFINITY;
  keys[i] = __float_as_uint(key);
}

__global__ void k_init_write(const float* __restrict__ img, int W, size_t P, uint64_t seed,
                             float log_tau0, const uint32_t* __restrict__ take,
                             const uint32_t* __restrict__ pos, float* __restrict__ params,
                             int cap) {
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= P || !take[i]) return;
  const size_t c = static_cast<size_t>(cap);
  const uint32_t s = pos[i];
  const int row = static_cast<int>(i / W), col = static_cast<int>(i % W);
  const uint64_t ctr = (1ull << 40) + 2ull * i;
  const float jx = __fmul_rn(__fsub_rn(static_cast<float>(splitmix64_at(seed, ctr) >> 40) * 0x1p-24f, 0.5f), 0.5f);
  const float jy = __fmul_rn(__fsub_rn(static_cast<float>(splitmix64_at(seed, ctr + 1) >> 40) * 0x1p-24f, 0.5f), 0.5f);
  params[PX * c + s] = __fadd_rn(__fadd_rn(static_cast<float>(col), 0.5f), jx);
  params[PY * c + s] = __fadd_rn(__fadd_rn(static_cast<float>(row), 0.5f), jy);
  params[PLOGTAU * c + s] = log_tau0;
  params[PR * c + s] = 0.f;
  params[PCR * c + s] = img[3 * i];
  params[PCG * c + s] = img[3 * i + 1];
  params[PCB * c + s] = img[3 * i + 2];
  params[PUX * c + s] = 1.f;
  params[PUY * c + s] = 0.f;
  params[PA * c + s] = 0.f;
  params[PB * c + s] = 0.f;
}

__global__ void k_init_inactive(float* __restrict__ params, int n, int cap) {
  const int s = n + blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  for (int j = 0; j < kNParams; ++j) params[j * c + s] = 0.f;
  params[PX * c + s] = -1.f;
  params[PY * c + s] = -1.f;
  params[PUX * c + s] = 1.f;
}

}  // namespace sad

using namespace sad;

extern "C" {

size_t sad_init_workspace_bytes(int32_t H, int32_t W) {
  if (H <= 0 || W <= 0) return 0;
  return init_layout(H, W).total;
}

int sad_init_sites(const float* img, int32_t H, int32_t W, int32_t n, int32_t capacity,
                   float lambda_init, uint64_t seed, float log_tau0, float* params,
                   void* workspace, size_t workspace_bytes, void* stream) {
  if (int e = check_problem(capacity, H, W, 4, false)) return e;
  const size_t P = static_cast<size_t>(H) * W;
  if (n < 0 || n > capacity || static_cast<size_t>(n) > P)
    return einval("sad_init_sites: need 0 <= n <= min(capacity, H*W) (n=%d)", n);
  if (!(lambda_init >= 0.f && lambda_init <= 1.f))
    return einval("sad_init_sites: lambda_init must be in [0,1]");
  if (P >= (1ull << 31)) return einval("sad_init_sites: image too large");
  if (!img || !params || !workspace) return einval("sad_init_sites: null pointer");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return einval("sad_init_sites: workspace must be 256-byte aligned");
  const InitLayout L = init_layout(H, W);
  if (workspace_bytes < L.total) {
    set_error("sad_init_sites: workspace has %zu bytes, needs %zu", workspace_bytes, L.total);
    return SAD_EWORKSPACE;
  }
  cudaStream_t st = as_stream(stream);
  char* base = static_cast<char*>(workspace);
  InitState* S = reinterpret_cast<InitState*>(base + L.state);
  float* g = reinterpret_cast<float*>(base + L.g);
  uint32_t* keys = reinterpret_cast<uint32_t*>(base + L.keys);
  uint32_t* flag = reinterpret_cast<uint32_t*>(base + L.flag);
  uint32_t* scan = reinterpret_cast<uint32_t*>(base + L.scan);
  uint32_t* bsums = reinterpret_cast<uint32_t*>(base + L.bsums);
  { TraceScope tr_(st, "k_init_state"); k_init_state<<<1, 256, 0, st>>>(S, static_cast<uint32_t>(n)); }
  const unsigned g256 = static_cast<unsigned>((P + 255) / 256);
  if (capacity > n)
    { TraceScope tr_(st, "k_init_inactive"); k_init_inactive<<<(capacity - n + 255) / 256, 256, 0, st>>>(params, n, capacity); }
  if (n == 0) return check_launch("k_init_inactive");
  { TraceScope tr_(st, "k_init_grad"); k_init_grad<<<g256, 256, 0, st>>>(img, H, W, g, S); }
  { TraceScope tr_(st, "k_init_keys"); k_init_keys<<<g256, 256, 0, st>>>(g, P, lambda_init, seed, S, keys); }
  run_select_smallest(keys, P, &S->sel, flag, scan, bsums, st);
  run_xscan(flag, scan, P, bsums, st);
  { TraceScope tr_(st, "k_init_write"); k_init_write<<<g256, 256, 0, st>>>(img, W, P, seed, log_tau0, flag, scan, params, capacity); }
  return check_launch("sad_init_sites");
}

}  // extern "C"
