// Site preparation ("pack") and the per-pixel top-K field: seed pass and one
// propagation pass (Sec. 4.3; App. "Data Layout and Packing", "Candidate Field and Jump Schedule").
#include "sad_device.cuh"
#include "sad_host.h"

namespace sad {

// ---------------------------------------------------------------------------
// prepare: raw planes -> {x,y,tau s,r}, {G00,G01,G11,active}, {cr,cg,cb,0}
// ---------------------------------------------------------------------------
__global__ void k_prepare(const float* __restrict__ params, int cap, float s,
                          float4* __restrict__ geo, float4* __restrict__ met,
                          float4* __restrict__ col) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  const float x = params[PX * c + i], y = params[PY * c + i];
  const float logtau = params[PLOGTAU * c + i], r = params[PR * c + i];
  const float ux = params[PUX * c + i], uy = params[PUY * c + i];
  const float a = params[PA * c + i], b = params[PB * c + i];
  const float nrm = __fsqrt_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)));
  float uxn = 1.f, uyn = 0.f;
  if (nrm > 0.f) {
    uxn = __fdiv_rn(ux, nrm);
    uyn = __fdiv_rn(uy, nrm);
  }
  const float ep = exp32_repro(__fadd_rn(b, a));
  const float em = exp32_repro(__fsub_rn(b, a));
  const float xx = __fmul_rn(uxn, uxn), yy = __fmul_rn(uyn, uyn), xy = __fmul_rn(uxn, uyn);
  const float G00 = __fadd_rn(__fmul_rn(ep, xx), __fmul_rn(em, yy));
  const float G01 = __fmul_rn(__fsub_rn(ep, em), xy);
  const float G11 = __fadd_rn(__fmul_rn(ep, yy), __fmul_rn(em, xx));
  const float ts = __fmul_rn(exp32_repro(logtau), s);
  geo[i] = make_float4(x, y, ts, r);
  met[i] = make_float4(G00, G01, G11, x >= 0.f ? 1.f : 0.f);
  col[i] = make_float4(params[PCR * c + i], params[PCG * c + i], params[PCB * c + i], 0.f);
}

// ---------------------------------------------------------------------------
// seed: slot 0 of the pixel holding each active site <- min id
// ---------------------------------------------------------------------------
__global__ void k_seed(const float4* __restrict__ geo, const float4* __restrict__ met, int cap,
                       int H, int W, uint32_t* __restrict__ plane0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  if (met[i].w == 0.f) return;
  const float4 g = geo[i];
  int col = static_cast<int>(floorf(g.x));
  int row = static_cast<int>(floorf(g.y));
  col = col < 0 ? 0 : (col >= W ? W - 1 : col);
  row = row < 0 ? 0 : (row >= H ? H - 1 : row);
  const size_t q = static_cast<size_t>(row) * W + col;
  atomicMin(&plane0[q * 4], static_cast<uint32_t>(i));
}

// ---------------------------------------------------------------------------
// one propagation pass.  One thread per pixel keeps the K best (logit, id)
// pairs sorted in registers; candidates already in the list are skipped
// before scoring (a duplicate has an identical key).
// ---------------------------------------------------------------------------
template <int K>
struct TopK {
  float l[K];
  uint32_t id[K];

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      l[k] = -INFINITY;
      id[k] = kInvalid;
    }
  }
  __device__ __forceinline__ bool contains(uint32_t c) const {
    bool hit = false;
#pragma unroll
    for (int k = 0; k < K; ++k) hit |= (id[k] == c);
    return hit;
  }
  // Insert (cl, cid) known to precede the last entry and not to be present.
  __device__ __forceinline__ void insert(float cl, uint32_t cid) {
#pragma unroll
    for (int k = K - 1; k > 0; --k) {
      const bool shift = key_before(cl, cid, l[k - 1], id[k - 1]);
      const bool here = !shift && key_before(cl, cid, l[k], id[k]);
      const float nl = shift ? l[k - 1] : (here ? cl : l[k]);
      const uint32_t ni = shift ? id[k - 1] : (here ? cid : id[k]);
      l[k] = nl;
      id[k] = ni;
    }
    if (key_before(cl, cid, l[0], id[0])) {
      l[0] = cl;
      id[0] = cid;
    }
  }
};

template <int K>
__device__ __forceinline__ void consider(TopK<K>& tk, uint32_t cid, uint32_t ucap, float px,
                                         float py, const float4* __restrict__ geo,
                                         const float4* __restrict__ met) {
  if (cid >= ucap) return;  // also rejects the sentinel
  if (tk.contains(cid)) return;
  const float4 m = ldg(&met[cid]);
  if (m.w == 0.f) return;
  const float4 g = ldg(&geo[cid]);
  const float l = score_exact(px, py, g, m);
  if (l != l) return;  // NaN
  if (!key_before(l, cid, tk.l[K - 1], tk.id[K - 1])) return;
  tk.insert(l, cid);
}

template <int K>
__device__ __forceinline__ void consider4(TopK<K>& tk, uint4 v, uint32_t ucap, float px, float py,
                                          const float4* __restrict__ geo,
                                          const float4* __restrict__ met) {
  consider<K>(tk, v.x, ucap, px, py, geo, met);
  consider<K>(tk, v.y, ucap, px, py, geo, met);
  consider<K>(tk, v.z, ucap, px, py, geo, met);
  consider<K>(tk, v.w, ucap, px, py, geo, met);
}

template <int K>
__global__ void __launch_bounds__(256) k_topk_update(const float4* __restrict__ geo,
                                                     const float4* __restrict__ met, int cap,
                                                     int H, int W,
                                                     const uint4* __restrict__ map_in,
                                                     uint4* __restrict__ map_out, uint32_t code,
                                                     int J, uint64_t seed) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y * blockDim.y + threadIdx.y;
  if (col >= W || row >= H) return;
  const size_t P = static_cast<size_t>(H) * W;
  const size_t q = static_cast<size_t>(row) * W + col;
  const uint32_t ucap = static_cast<uint32_t>(cap);
  const float px = __fadd_rn(static_cast<float>(col), 0.5f);
  const float py = __fadd_rn(static_cast<float>(row), 0.5f);
  TopK<K> tk;
  tk.init();
  constexpr int NP = K / 4;
#pragma unroll
  for (int j = 0; j < NP; ++j) consider4<K>(tk, ldg(&map_in[j * P + q]), ucap, px, py, geo, met);
  const int s = static_cast<int>(code >> 16);
  const int nc[4] = {col - s, col + s, col, col};
  const int nr[4] = {row, row, row - s, row + s};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (nc[d] < 0 || nc[d] >= W || nr[d] < 0 || nr[d] >= H) continue;
    const size_t nq = static_cast<size_t>(nr[d]) * W + nc[d];
#pragma unroll
    for (int j = 0; j < NP; ++j) consider4<K>(tk, ldg(&map_in[j * P + nq]), ucap, px, py, geo, met);
  }
  const uint64_t base = (static_cast<uint64_t>(code) << 32);
  for (int j = 0; j < J; ++j) {
    const uint64_t ctr = base | static_cast<uint32_t>(q * static_cast<uint32_t>(J) + j);
    const uint64_t h = splitmix64_at(seed, ctr);
    const uint32_t cid = static_cast<uint32_t>(((h >> 32) * static_cast<uint64_t>(ucap)) >> 32);
    consider<K>(tk, cid, ucap, px, py, geo, met);
  }
#pragma unroll
  for (int j = 0; j < NP; ++j)
    map_out[j * P + q] = make_uint4(tk.id[4 * j], tk.id[4 * j + 1], tk.id[4 * j + 2], tk.id[4 * j + 3]);
}

}  // namespace sad

using namespace sad;

extern "C" {

int sad_prepare_sites(const float* params, int32_t capacity, int32_t H, int32_t W, float* prep,
                      void* stream) {
  if (int st = check_problem(capacity, H, W, 4, false)) return st;
  if (capacity == 0) return SAD_OK;
  if (!params || !prep) return einval("sad_prepare_sites: null pointer");
  if (!aligned16(prep)) return einval("sad_prepare_sites: prep must be 16-byte aligned");
  const float s = 1.0f / static_cast<float>(H > W ? H : W);
  float4* p4 = reinterpret_cast<float4*>(prep);
  const int bs = 256;
  k_prepare<<<(capacity + bs - 1) / bs, bs, 0, as_stream(stream)>>>(params, capacity, s, p4,
                                                                     p4 + capacity,
                                                                     p4 + 2 * (size_t)capacity);
  return check_launch("k_prepare");
}

int sad_topk_seed(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                  uint32_t* map, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (!map || (!prep && capacity > 0)) return einval("sad_topk_seed: null pointer");
  if (!aligned16(map) || !aligned16(prep)) return einval("sad_topk_seed: pointers must be 16-byte aligned");
  const size_t P = static_cast<size_t>(H) * W;
  cudaError_t e = cudaMemsetAsync(map, 0xff, P * K * sizeof(uint32_t), as_stream(stream));
  if (e != cudaSuccess) {
    set_error("sad_topk_seed memset: %s", cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  if (capacity == 0) return SAD_OK;
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  const int bs = 256;
  k_seed<<<(capacity + bs - 1) / bs, bs, 0, as_stream(stream)>>>(p4, p4 + capacity, capacity, H,
                                                                  W, map);
  return check_launch("k_seed");
}

int sad_update_topk(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                    const uint32_t* map_in, uint32_t* map_out, uint32_t step_code,
                    int32_t n_inject, uint64_t seed, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (!map_in || !map_out || (!prep && capacity > 0)) return einval("sad_update_topk: null pointer");
  if (!aligned16(map_in) || !aligned16(map_out) || !aligned16(prep))
    return einval("sad_update_topk: pointers must be 16-byte aligned");
  if (n_inject < 0 || n_inject > 16) return einval("sad_update_topk: n_inject must be in [0,16]");
  const size_t P = static_cast<size_t>(H) * W;
  if (static_cast<uint64_t>(P) * static_cast<uint64_t>(n_inject > 0 ? n_inject : 1) >= (1ull << 32))
    return einval("sad_update_topk: H*W*n_inject must be below 2^32");
  const char* a = reinterpret_cast<const char*>(map_in);
  const char* b = reinterpret_cast<const char*>(map_out);
  const size_t bytes = P * K * sizeof(uint32_t);
  if (a < b + bytes && b < a + bytes) return einval("sad_update_topk: map_in and map_out overlap");
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  const dim3 block(32, 8);
  const dim3 grid((W + 31) / 32, (H + 7) / 8);
  const uint4* in = reinterpret_cast<const uint4*>(map_in);
  uint4* out = reinterpret_cast<uint4*>(map_out);
  cudaStream_t st = as_stream(stream);
  switch (K) {
    case 4:
      k_topk_update<4><<<grid, block, 0, st>>>(p4, p4 + capacity, capacity, H, W, in, out,
                                               step_code, n_inject, seed);
      break;
    case 8:
      k_topk_update<8><<<grid, block, 0, st>>>(p4, p4 + capacity, capacity, H, W, in, out,
                                               step_code, n_inject, seed);
      break;
    default:
      k_topk_update<16><<<grid, block, 0, st>>>(p4, p4 + capacity, capacity, H, W, in, out,
                                                step_code, n_inject, seed);
      break;
  }
  return check_launch("k_topk_update");
}

}  // extern "C"
