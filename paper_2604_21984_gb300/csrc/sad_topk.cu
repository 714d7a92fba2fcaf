// Site preparation ("pack") and the per-pixel top-K field: seed pass and one
// propagation pass (Sec. 4.3; App. "Data Layout and Packing", "Candidate Field and Jump Schedule").
#include "sad_device.cuh"
#include "sad_host.h"
#include "sad_topk.cuh"

namespace sad {

// ---------------------------------------------------------------------------
// prepare: raw planes -> {x,y,tau s,r}, {G00,G01,G11,active}, {cr,cg,cb,0}
// ---------------------------------------------------------------------------
__global__ void k_prepare(const float* __restrict__ params, int cap, float s,
                          float4* __restrict__ geo, float4* __restrict__ met,
                          float4* __restrict__ col, float4* __restrict__ ba,
                          float4* __restrict__ bb, float* __restrict__ cbd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  prepare_site(params[PX * c + i], params[PY * c + i], params[PLOGTAU * c + i], params[PR * c + i],
               params[PCR * c + i], params[PCG * c + i], params[PCB * c + i], params[PUX * c + i],
               params[PUY * c + i], params[PA * c + i], params[PB * c + i], s, geo[i], met[i],
               col[i], ba[i], bb[i], cbd[i]);
}

// ---------------------------------------------------------------------------
// seed: slot 0 of the pixel holding each active site <- min id
// ---------------------------------------------------------------------------
__global__ void k_seed(const float4* __restrict__ geo, const float4* __restrict__ met, int cap,
                       int H, int W, int cell, int Wc, uint32_t* __restrict__ plane0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  if (met[i].w == 0.f) return;
  const float4 g = geo[i];
  int col = static_cast<int>(floorf(g.x));
  int row = static_cast<int>(floorf(g.y));
  col = col < 0 ? 0 : (col >= W ? W - 1 : col);
  row = row < 0 ? 0 : (row >= H ? H - 1 : row);
  const size_t q = static_cast<size_t>(row / cell) * Wc + col / cell;  // cell of a candidate grid
  atomicMin(&plane0[q * 4], static_cast<uint32_t>(i));
}

// ---------------------------------------------------------------------------
// one propagation pass over the whole image (per-pixel work in sad_topk.cuh)
// ---------------------------------------------------------------------------
constexpr int kUpdThreads = 256;

template <int K, class Sites>
__global__ void __launch_bounds__(kUpdThreads, 4) k_topk_update(Sites sites, int cap, int H, int W,
                                                             const uint4* __restrict__ map_in,
                                                             uint4* __restrict__ map_out,
                                                             uint32_t code, int J, uint64_t seed,
                                                             float cell) {
  __shared__ uint32_t s_q[kQueue][kUpdThreads];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y * blockDim.y + threadIdx.y;
  if (col >= W || row >= H) return;
  const size_t P = static_cast<size_t>(H) * W;
  const size_t q = static_cast<size_t>(row) * W + col;
  uint64_t v[K];
  pixel_update<K, kUpdThreads, 2>(v, true, col, row, H, W, SiteRange{0u, static_cast<uint32_t>(cap)},
                               sites, map_in, P, 0, code, J, seed, s_q, tid, cell);
#pragma unroll
  for (int j = 0; j < K / 4; ++j)
    map_out[j * P + q] = make_uint4(key_id(v[4 * j]), key_id(v[4 * j + 1]), key_id(v[4 * j + 2]),
                                    key_id(v[4 * j + 3]));
}

// ---------------------------------------------------------------------------
// JFA prepass flood pass: the 3x3 neighbourhood's first four slots -> the
// best four in slot 0..3 (App. "Candidate Field and Jump Schedule", JFA
// prepass); the other slots are copied.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(kUpdThreads) k_jfa_flood(const float4* __restrict__ geo,
                                                           const float4* __restrict__ met, int cap,
                                                           int H, int W,
                                                           const uint4* __restrict__ map_in,
                                                           uint4* __restrict__ map_out, int s) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y * blockDim.y + threadIdx.y;
  if (col >= W || row >= H) return;
  const size_t P = static_cast<size_t>(H) * W;
  const size_t q = static_cast<size_t>(row) * W + col;
  const float px = __fadd_rn(static_cast<float>(col), 0.5f);
  const float py = __fadd_rn(static_cast<float>(row), 0.5f);
  const SiteRange sr{0u, static_cast<uint32_t>(cap)};
  uint64_t v[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll 1
  for (int d = 0; d < 9; ++d) {
    const int nc = col + (d % 3 - 1) * s, nr = row + (d / 3 - 1) * s;
    if (nc < 0 || nc >= W || nr < 0 || nr >= H) continue;
    const uint4 w = ldg(&map_in[static_cast<size_t>(nr) * W + nc]);
    const uint32_t id4[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (list_has<4>(v, id4[u])) continue;
      const uint64_t c = cand_key(id4[u], sr, px, py, F32Sites{geo, met});
      if (c > v[3]) list_insert<4>(v, c);
    }
  }
  map_out[q] = make_uint4(key_id(v[0]), key_id(v[1]), key_id(v[2]), key_id(v[3]));
#pragma unroll
  for (int j = 1; j < K / 4; ++j) map_out[j * P + q] = ldg(&map_in[j * P + q]);
}

// Candidate grid -> per-pixel lists: pixel (x, y) takes cell (x / s, y / s).
__global__ void k_grid_expand(const uint4* __restrict__ grid, int H, int W, int s, int NP,
                              uint4* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  const int Wc = (W + s - 1) / s, Hc = (H + s - 1) / s;
  const size_t P = static_cast<size_t>(H) * W, Pc = static_cast<size_t>(Hc) * Wc;
  const size_t qc = static_cast<size_t>(y / s) * Wc + x / s;
  const size_t q = static_cast<size_t>(y) * W + x;
  for (int j = 0; j < NP; ++j) out[j * P + q] = ldg(&grid[j * Pc + qc]);
}

// Half2 candidate table from the prepared table (App. "Data Layout and
// Packing", Packed candidate sites): each value rounded to the nearest
// half (ties to even) after saturation to +-65504, the largest finite half.
__device__ __forceinline__ uint32_t half2_bits(float lo, float hi) {
  const float m = 65504.f;
  const unsigned short a = __half_as_ushort(__float2half_rn(fminf(fmaxf(lo, -m), m)));
  const unsigned short b = __half_as_ushort(__float2half_rn(fminf(fmaxf(hi, -m), m)));
  return static_cast<uint32_t>(a) | (static_cast<uint32_t>(b) << 16);
}

__global__ void k_pack_candidates(const float4* __restrict__ geo, const float4* __restrict__ met,
                                  int cap, uint4* __restrict__ cand) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const float4 g = ldg(&geo[i]), m = ldg(&met[i]);
  cand[i] = make_uint4(half2_bits(g.x, g.y), half2_bits(g.z, g.w), half2_bits(m.x, m.y),
                       half2_bits(m.z, m.w));
}

template <class Sites>
static void launch_update(int K, dim3 grid, dim3 block, cudaStream_t st, Sites sites, int cap,
                          int H, int W, const uint4* in, uint4* out, uint32_t code, int J,
                          uint64_t seed, float cell) {
  switch (K) {
    case 4: k_topk_update<4><<<grid, block, 0, st>>>(sites, cap, H, W, in, out, code, J, seed, cell); break;
    case 8: k_topk_update<8><<<grid, block, 0, st>>>(sites, cap, H, W, in, out, code, J, seed, cell); break;
    default: k_topk_update<16><<<grid, block, 0, st>>>(sites, cap, H, W, in, out, code, J, seed, cell); break;
  }
}

// One propagation pass over an H x W grid of lists whose entries are scored
// at ((col + 0.5) cell, (row + 0.5) cell), from the prepared fp32 table or,
// with h2, from the half2 candidate table.
static int run_update(const void* table, bool h2, int32_t capacity, int32_t H, int32_t W, int32_t K,
                      const uint32_t* map_in, uint32_t* map_out, uint32_t step_code,
                      int32_t n_inject, uint64_t seed, float cell, void* stream, const char* name) {
  if (!map_in || !map_out || (!table && capacity > 0)) return einval("%s: null pointer", name);
  if (!aligned16(map_in) || !aligned16(map_out) || !aligned16(table))
    return einval("%s: pointers must be 16-byte aligned", name);
  if (n_inject < 0 || n_inject > 16) return einval("%s: n_inject must be in [0,16]", name);
  const size_t P = static_cast<size_t>(H) * W;
  if (static_cast<uint64_t>(P) * static_cast<uint64_t>(n_inject > 0 ? n_inject : 1) >= (1ull << 32))
    return einval("%s: H*W*n_inject must be below 2^32", name);
  const char* a = reinterpret_cast<const char*>(map_in);
  const char* b = reinterpret_cast<const char*>(map_out);
  const size_t bytes = P * K * sizeof(uint32_t);
  if (a < b + bytes && b < a + bytes) return einval("%s: map_in and map_out overlap", name);
  const dim3 block(32, 8);
  const dim3 grid((W + 31) / 32, (H + 7) / 8);
  const uint4* in = reinterpret_cast<const uint4*>(map_in);
  uint4* out = reinterpret_cast<uint4*>(map_out);
  cudaStream_t st = as_stream(stream);
  if (!h2) {
    const float4* p4 = reinterpret_cast<const float4*>(table);
    TraceScope tr_(st, "k_topk_update");
    launch_update(K, grid, block, st, F32Sites{p4, p4 + capacity}, capacity, H, W, in, out,
                  step_code, n_inject, seed, cell);
  } else {
    TraceScope tr_(st, "k_topk_update_h2");
    launch_update(K, grid, block, st, H2Sites{reinterpret_cast<const uint4*>(table)}, capacity, H,
                  W, in, out, step_code, n_inject, seed, cell);
  }
  return check_launch(name);
}

// ---------------------------------------------------------------------------
// exact top-K of sampled pixels by brute force over every site: the set the
// propagation approximates (Sec. 4.3), scored and ordered exactly as a pass
// does (fp32 score of fixed operation order, keys ordered by logit then id)
// ---------------------------------------------------------------------------
constexpr int kExactThreads = 256;

template <int K>
__global__ void __launch_bounds__(kExactThreads) k_exact_topk(const float4* __restrict__ geo,
                                                              const float4* __restrict__ met, int cap,
                                                              int W, const int64_t* __restrict__ pix,
                                                              uint32_t* __restrict__ out) {
  __shared__ uint64_t s_best[kExactThreads / 32];
  __shared__ uint64_t s_win;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t q = pix[blockIdx.x];
  const float px = static_cast<float>(q % W) + 0.5f, py = static_cast<float>(q / W) + 0.5f;
  uint64_t v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0ull;
  for (int i = t; i < cap; i += kExactThreads) {
    const float4 mt = ldg(&met[i]);
    if (mt.w == 0.f) continue;
    const float l = score_exact(px, py, ldg(&geo[i]), mt);
    if (l != l) continue;  // a NaN logit never enters
    const uint64_t c = make_key(l, static_cast<uint32_t>(i));
    if (c > v[K - 1]) list_insert<K>(v, c);
  }
  // K rounds: the best head over the block wins and its thread pops it (ids
  // are distinct, so exactly one thread holds the winning key)
  for (int r = 0; r < K; ++r) {
    uint64_t h = v[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t y = __shfl_xor_sync(0xffffffffu, h, o);
      h = y > h ? y : h;
    }
    if (lane == 0) s_best[warp] = h;
    __syncthreads();
    if (t == 0) {
      uint64_t b = 0ull;
      for (int w = 0; w < kExactThreads / 32; ++w) b = s_best[w] > b ? s_best[w] : b;
      s_win = b;
      out[static_cast<size_t>(blockIdx.x) * K + r] = b ? key_id(b) : kInvalid;
    }
    __syncthreads();
    const uint64_t win = s_win;
    if (win != 0ull && v[0] == win) {
#pragma unroll
      for (int k = 0; k < K - 1; ++k) v[k] = v[k + 1];
      v[K - 1] = 0ull;
    }
    __syncthreads();
  }
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
  { TraceScope tr_(as_stream(stream), "k_prepare"); k_prepare<<<(capacity + bs - 1) / bs, bs, 0, as_stream(stream)>>>(params, capacity, s, p4,
                                                                     p4 + capacity,
                                                                     p4 + 2 * (size_t)capacity,
                                                                     p4 + 3 * (size_t)capacity,
                                                                     p4 + 4 * (size_t)capacity,
                                                                     reinterpret_cast<float*>(p4 + 5 * (size_t)capacity)); }
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
  { TraceScope tr_(as_stream(stream), "k_seed"); k_seed<<<(capacity + bs - 1) / bs, bs, 0, as_stream(stream)>>>(p4, p4 + capacity, capacity, H,
                                                                  W, 1, W, map); }
  return check_launch("k_seed");
}

int sad_jfa_flood(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                  const uint32_t* map_in, uint32_t* map_out, uint32_t step_code, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (!map_in || !map_out || (!prep && capacity > 0)) return einval("sad_jfa_flood: null pointer");
  if (!aligned16(map_in) || !aligned16(map_out) || !aligned16(prep))
    return einval("sad_jfa_flood: pointers must be 16-byte aligned");
  const size_t P = static_cast<size_t>(H) * W;
  const char* a = reinterpret_cast<const char*>(map_in);
  const char* b = reinterpret_cast<const char*>(map_out);
  if (a < b + P * K * 4 && b < a + P * K * 4) return einval("sad_jfa_flood: maps overlap");
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  const dim3 block(32, 8);
  const dim3 grid((W + 31) / 32, (H + 7) / 8);
  const int s = static_cast<int>(step_code >> 16);
  cudaStream_t st = as_stream(stream);
  const uint4* in = reinterpret_cast<const uint4*>(map_in);
  uint4* out = reinterpret_cast<uint4*>(map_out);
  {
    TraceScope tr_(st, "k_jfa_flood");
    switch (K) {
      case 4: k_jfa_flood<4><<<grid, block, 0, st>>>(p4, p4 + capacity, capacity, H, W, in, out, s); break;
      case 8: k_jfa_flood<8><<<grid, block, 0, st>>>(p4, p4 + capacity, capacity, H, W, in, out, s); break;
      default: k_jfa_flood<16><<<grid, block, 0, st>>>(p4, p4 + capacity, capacity, H, W, in, out, s); break;
    }
  }
  return check_launch("k_jfa_flood");
}

int sad_update_topk(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                    const uint32_t* map_in, uint32_t* map_out, uint32_t step_code,
                    int32_t n_inject, uint64_t seed, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  return run_update(prep, false, capacity, H, W, K, map_in, map_out, step_code, n_inject, seed, 1.f,
                    stream, "sad_update_topk");
}

int sad_grid_seed(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t s_grid,
                  int32_t K, uint32_t* map, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (s_grid < 1 || s_grid > 64) return einval("sad_grid_seed: s_grid must be in [1, 64]");
  if (!map || (!prep && capacity > 0)) return einval("sad_grid_seed: null pointer");
  if (!aligned16(map) || !aligned16(prep)) return einval("sad_grid_seed: pointers must be 16-byte aligned");
  const int Hc = (H + s_grid - 1) / s_grid, Wc = (W + s_grid - 1) / s_grid;
  const size_t Pc = static_cast<size_t>(Hc) * Wc;
  cudaError_t e = cudaMemsetAsync(map, 0xff, Pc * K * sizeof(uint32_t), as_stream(stream));
  if (e != cudaSuccess) {
    set_error("sad_grid_seed memset: %s", cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  if (capacity == 0) return SAD_OK;
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  {
    TraceScope tr_(as_stream(stream), "k_seed");
    k_seed<<<(capacity + 255) / 256, 256, 0, as_stream(stream)>>>(p4, p4 + capacity, capacity, H, W,
                                                                  s_grid, Wc, map);
  }
  return check_launch("k_seed");
}

int sad_grid_update(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t s_grid,
                    int32_t K, const uint32_t* map_in, uint32_t* map_out, uint32_t step_code,
                    int32_t n_inject, uint64_t seed, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (s_grid < 1 || s_grid > 64) return einval("sad_grid_update: s_grid must be in [1, 64]");
  return run_update(prep, false, capacity, (H + s_grid - 1) / s_grid, (W + s_grid - 1) / s_grid, K,
                    map_in, map_out, step_code, n_inject, seed, static_cast<float>(s_grid), stream,
                    "sad_grid_update");
}

int sad_pack_candidates(const float* prep, int32_t capacity, uint32_t* cand, void* stream) {
  if (capacity < 0) return einval("sad_pack_candidates: capacity must be >= 0");
  if (capacity == 0) return SAD_OK;
  if (!prep || !cand) return einval("sad_pack_candidates: null pointer");
  if (!aligned16(prep) || !aligned16(cand))
    return einval("sad_pack_candidates: pointers must be 16-byte aligned");
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  cudaStream_t st = as_stream(stream);
  {
    TraceScope tr_(st, "k_pack_candidates");
    k_pack_candidates<<<(capacity + 255) / 256, 256, 0, st>>>(p4, p4 + capacity, capacity,
                                                             reinterpret_cast<uint4*>(cand));
  }
  return check_launch("k_pack_candidates");
}

int sad_update_topk_h2(const uint32_t* cand, int32_t capacity, int32_t H, int32_t W, int32_t K,
                       const uint32_t* map_in, uint32_t* map_out, uint32_t step_code,
                       int32_t n_inject, uint64_t seed, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  return run_update(cand, true, capacity, H, W, K, map_in, map_out, step_code, n_inject, seed,
                    1.f, stream, "sad_update_topk_h2");
}

int sad_grid_expand(const uint32_t* map_grid, int32_t H, int32_t W, int32_t s_grid, int32_t K,
                    uint32_t* map_pixels, void* stream) {
  if (int st = check_problem(0, H, W, K, true)) return st;
  if (s_grid < 1 || s_grid > 64) return einval("sad_grid_expand: s_grid must be in [1, 64]");
  if (!map_grid || !map_pixels) return einval("sad_grid_expand: null pointer");
  if (!aligned16(map_grid) || !aligned16(map_pixels))
    return einval("sad_grid_expand: pointers must be 16-byte aligned");
  const dim3 block(32, 8);
  const dim3 grid((W + 31) / 32, (H + 7) / 8);
  cudaStream_t st = as_stream(stream);
  {
    TraceScope tr_(st, "k_grid_expand");
    k_grid_expand<<<grid, block, 0, st>>>(reinterpret_cast<const uint4*>(map_grid), H, W, s_grid, K / 4,
                                         reinterpret_cast<uint4*>(map_pixels));
  }
  return check_launch("k_grid_expand");
}

int sad_exact_topk(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                   const int64_t* pixels, int64_t n, uint32_t* ids_out, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (n < 0 || n > 0x7fffffff) return einval("sad_exact_topk: n must be in [0, 2^31)");
  if (n == 0) return SAD_OK;
  if (!pixels || !ids_out || (!prep && capacity > 0)) return einval("sad_exact_topk: null pointer");
  if (!aligned16(prep) || (reinterpret_cast<uintptr_t>(pixels) & 7u))
    return einval("sad_exact_topk: misaligned pointer");
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  const float4 *geo = p4, *met = p4 + capacity;
  cudaStream_t st = as_stream(stream);
  const unsigned grid = static_cast<unsigned>(n);
  TraceScope tr_(st, "k_exact_topk");
  switch (K) {
    case 4: k_exact_topk<4><<<grid, kExactThreads, 0, st>>>(geo, met, capacity, W, pixels, ids_out); break;
    case 8: k_exact_topk<8><<<grid, kExactThreads, 0, st>>>(geo, met, capacity, W, pixels, ids_out); break;
    default: k_exact_topk<16><<<grid, kExactThreads, 0, st>>>(geo, met, capacity, W, pixels, ids_out); break;
  }
  return check_launch("k_exact_topk");
}

}  // extern "C"
