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
// one propagation pass.
//
// Candidate keys: (logit, id) packed into one 64-bit integer whose unsigned
// order is the list order (logit descending, then id ascending):
//   key = orderable(logit) << 32 | ~id,
// with orderable() the usual sign-flip map of IEEE floats (-0 is first turned
// into +0 so that the two zeros tie, as they do in float comparison).  The
// empty entry is key 0, below every real candidate.
//
// Per pixel (one thread):
//  A. score the pixel's own list (independent gathers) and sort it with a
//     bitonic network; drop duplicate ids (only possible in a damaged input);
//  B. filter the 4 neighbour lists and the J injected ids against the list
//     and queue the novel ids in shared memory (per-thread column);
//  C. each thread scores its own queue and inserts winners.
// Phase C runs per lane, so the insertion network is paid for the queued
// candidates only, not for every candidate of every lane in the warp.
// ---------------------------------------------------------------------------
constexpr int kUpdThreads = 256;
constexpr int kQueue = 24;

__device__ __forceinline__ uint64_t make_key(float l, uint32_t id) {
  uint32_t u = __float_as_uint(__fadd_rn(l, 0.0f));
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return (static_cast<uint64_t>(u) << 32) | static_cast<uint64_t>(~id);
}

__device__ __forceinline__ uint32_t key_id(uint64_t k) { return ~static_cast<uint32_t>(k); }

template <int K>
__device__ __forceinline__ void bitonic_sort_desc(uint64_t (&v)[K]) {
#pragma unroll
  for (int k = 2; k <= K; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const bool desc = (i & k) == 0;
          const uint64_t a = v[i], b = v[l];
          const bool sw = desc ? (a < b) : (a > b);
          v[i] = sw ? b : a;
          v[l] = sw ? a : b;
        }
      }
    }
  }
}

template <int K>
__device__ __forceinline__ bool list_has(const uint64_t (&v)[K], uint32_t id) {
  const uint32_t nid = ~id;
  bool hit = false;
#pragma unroll
  for (int k = 0; k < K; ++k) hit |= (static_cast<uint32_t>(v[k]) == nid);
  return hit;
}

// Insert key c (greater than v[K-1], id not present) keeping v sorted.
template <int K>
__device__ __forceinline__ void list_insert(uint64_t (&v)[K], uint64_t c) {
  bool gt[K];
#pragma unroll
  for (int k = 0; k < K; ++k) gt[k] = c > v[k];
#pragma unroll
  for (int k = K - 1; k > 0; --k) v[k] = gt[k - 1] ? v[k - 1] : (gt[k] ? c : v[k]);
  v[0] = gt[0] ? c : v[0];
}

// Logit key of candidate id at (px, py), or 0 if the id cannot enter.
__device__ __forceinline__ uint64_t cand_key(uint32_t id, uint32_t ucap, float px, float py,
                                             const float4* __restrict__ geo,
                                             const float4* __restrict__ met) {
  if (id >= ucap) return 0ull;
  const float4 m = ldg(&met[id]);
  if (m.w == 0.f) return 0ull;
  const float l = score_exact(px, py, ldg(&geo[id]), m);
  if (l != l) return 0ull;
  return make_key(l, id);
}

template <int K>
__global__ void __launch_bounds__(kUpdThreads) k_topk_update(const float4* __restrict__ geo,
                                                             const float4* __restrict__ met, int cap,
                                                             int H, int W,
                                                             const uint4* __restrict__ map_in,
                                                             uint4* __restrict__ map_out,
                                                             uint32_t code, int J, uint64_t seed) {
  __shared__ uint32_t s_q[kQueue][kUpdThreads];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y * blockDim.y + threadIdx.y;
  if (col >= W || row >= H) return;
  const size_t P = static_cast<size_t>(H) * W;
  const size_t q = static_cast<size_t>(row) * W + col;
  const uint32_t ucap = static_cast<uint32_t>(cap);
  const float px = __fadd_rn(static_cast<float>(col), 0.5f);
  const float py = __fadd_rn(static_cast<float>(row), 0.5f);
  constexpr int NP = K / 4;

  // A. own list
  uint64_t v[K];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const uint4 w = ldg(&map_in[j * P + q]);
    v[4 * j] = cand_key(w.x, ucap, px, py, geo, met);
    v[4 * j + 1] = cand_key(w.y, ucap, px, py, geo, met);
    v[4 * j + 2] = cand_key(w.z, ucap, px, py, geo, met);
    v[4 * j + 3] = cand_key(w.w, ucap, px, py, geo, met);
  }
  bitonic_sort_desc<K>(v);
  bool dup = false;
#pragma unroll
  for (int k = 1; k < K; ++k) {
    const bool d = v[k] != 0ull && v[k] == v[k - 1];
    dup |= d;
  }
  if (dup) {  // damaged input list: zero repeated keys, re-sort
#pragma unroll
    for (int k = K - 1; k > 0; --k)
      if (v[k] != 0ull && v[k] == v[k - 1]) v[k] = 0ull;
    bitonic_sort_desc<K>(v);
  }

  // B + C. queue novel candidates; drain the queue when full and at the end
  int qn = 0;
  auto drain = [&]() {
    for (int i = 0; i < qn; ++i) {
      const uint32_t id = s_q[i][tid];
      if (list_has<K>(v, id)) continue;
      const uint64_t c = cand_key(id, ucap, px, py, geo, met);
      if (c > v[K - 1]) list_insert<K>(v, c);
    }
    qn = 0;
  };
  auto offer = [&](uint32_t id) {
    if (id >= ucap || list_has<K>(v, id)) return;
    for (int i = 0; i < qn; ++i)
      if (s_q[i][tid] == id) return;
    if (qn == kQueue) drain();
    s_q[qn++][tid] = id;
  };
  const int s = static_cast<int>(code >> 16);
  const int nc[4] = {col - s, col + s, col, col};
  const int nr[4] = {row, row, row - s, row + s};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (nc[d] < 0 || nc[d] >= W || nr[d] < 0 || nr[d] >= H) continue;
    const size_t nq = static_cast<size_t>(nr[d]) * W + nc[d];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const uint4 w = ldg(&map_in[j * P + nq]);
      offer(w.x);
      offer(w.y);
      offer(w.z);
      offer(w.w);
    }
  }
  const uint64_t base = (static_cast<uint64_t>(code) << 32);
  for (int j = 0; j < J; ++j) {
    const uint64_t ctr = base | static_cast<uint32_t>(q * static_cast<uint32_t>(J) + j);
    const uint64_t h = splitmix64_at(seed, ctr);
    offer(static_cast<uint32_t>(((h >> 32) * static_cast<uint64_t>(ucap)) >> 32));
  }
  drain();
#pragma unroll
  for (int j = 0; j < NP; ++j)
    map_out[j * P + q] = make_uint4(key_id(v[4 * j]), key_id(v[4 * j + 1]), key_id(v[4 * j + 2]),
                                    key_id(v[4 * j + 3]));
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
