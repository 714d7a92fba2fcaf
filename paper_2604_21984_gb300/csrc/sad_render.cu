// Forward blend (Sec. 4.2) over the cached top-K lists: full-image render and
// random-access decode at float coordinates.
#include "sad_device.cuh"
#include "sad_host.h"

namespace sad {

// Blend of the K listed sites at point (px, py): max-subtracted softmax of the
// logits, colour = sum w_i c_i; black if no listed site is valid.  Loads use
// clamped ids so that each batch of gathers is issued before the dependent
// arithmetic (memory-level parallelism); invalid entries are masked after.
template <int K>
__device__ __forceinline__ float3 blend(const uint32_t (&ids)[K], float px, float py, uint32_t ucap,
                                        const float4* __restrict__ geo,
                                        const float4* __restrict__ met,
                                        const float4* __restrict__ col) {
  constexpr int B = 4;
  float l[K];
  float m = -INFINITY;
  uint32_t valid = 0;
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += B) {
    float4 gk[B], mk[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const uint32_t id = ids[k0 + j] < ucap ? ids[k0 + j] : 0u;
      gk[j] = ldg(&geo[id]);
      mk[j] = ldg(&met[id]);
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const bool ok = ids[k0 + j] < ucap && mk[j].w != 0.f;
      const float lk = score_fast(px, py, gk[j], mk[j]).l;
      l[k0 + j] = ok ? lk : -INFINITY;
      valid |= ok ? (1u << (k0 + j)) : 0u;
      m = ok ? fmaxf(m, lk) : m;
    }
  }
  float3 c = make_float3(0.f, 0.f, 0.f);
  if (!valid) return c;
  float z = 0.f;
  constexpr int BC = 8;
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += BC) {
    float4 ck[BC];
#pragma unroll
    for (int j = 0; j < BC && k0 + j < K; ++j)
      ck[j] = ldg(&col[ids[k0 + j] < ucap ? ids[k0 + j] : 0u]);
#pragma unroll
    for (int j = 0; j < BC && k0 + j < K; ++j) {
      const float e = (valid >> (k0 + j) & 1u) ? __expf(l[k0 + j] - m) : 0.f;
      z += e;
      c.x += e * ck[j].x;
      c.y += e * ck[j].y;
      c.z += e * ck[j].z;
    }
  }
  const float iz = 1.f / z;
  c.x *= iz;
  c.y *= iz;
  c.z *= iz;
  return c;
}

template <int K>
__device__ __forceinline__ void load_list(const uint4* __restrict__ map, size_t P, size_t q,
                                          uint32_t (&ids)[K]) {
#pragma unroll
  for (int j = 0; j < K / 4; ++j) {
    const uint4 v = ldg(&map[j * P + q]);
    ids[4 * j] = v.x;
    ids[4 * j + 1] = v.y;
    ids[4 * j + 2] = v.z;
    ids[4 * j + 3] = v.w;
  }
}

template <int K>
__global__ void __launch_bounds__(256) k_render(const float4* __restrict__ geo,
                                                const float4* __restrict__ met,
                                                const float4* __restrict__ col, int cap, int H,
                                                int W, const uint4* __restrict__ map,
                                                float* __restrict__ rgb) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  const size_t P = static_cast<size_t>(H) * W;
  const size_t q = static_cast<size_t>(y) * W + x;
  uint32_t ids[K];
  load_list<K>(map, P, q, ids);
  const float3 c = blend<K>(ids, x + 0.5f, y + 0.5f, static_cast<uint32_t>(cap), geo, met, col);
  rgb[3 * q] = c.x;
  rgb[3 * q + 1] = c.y;
  rgb[3 * q + 2] = c.z;
}

template <int K>
__global__ void __launch_bounds__(256) k_decode(const float4* __restrict__ geo,
                                                const float4* __restrict__ met,
                                                const float4* __restrict__ col, int cap, int H,
                                                int W, const uint4* __restrict__ map,
                                                const float2* __restrict__ xy, int64_t n,
                                                float* __restrict__ rgb) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 p = ldg(&xy[i]);
  int cx = static_cast<int>(floorf(p.x));
  int cy = static_cast<int>(floorf(p.y));
  cx = cx < 0 ? 0 : (cx >= W ? W - 1 : cx);
  cy = cy < 0 ? 0 : (cy >= H ? H - 1 : cy);
  const size_t P = static_cast<size_t>(H) * W;
  uint32_t ids[K];
  load_list<K>(map, P, static_cast<size_t>(cy) * W + cx, ids);
  const float3 c = blend<K>(ids, p.x, p.y, static_cast<uint32_t>(cap), geo, met, col);
  rgb[3 * i] = c.x;
  rgb[3 * i + 1] = c.y;
  rgb[3 * i + 2] = c.z;
}

}  // namespace sad

using namespace sad;

extern "C" {

int sad_render(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
               const uint32_t* map, float* rgb, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (!map || !rgb || (!prep && capacity > 0)) return einval("sad_render: null pointer");
  if (!aligned16(map) || !aligned16(prep)) return einval("sad_render: pointers must be 16-byte aligned");
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  const float4 *geo = p4, *met = p4 + capacity, *col = p4 + 2 * (size_t)capacity;
  const uint4* m4 = reinterpret_cast<const uint4*>(map);
  const dim3 block(32, 8);
  const dim3 grid((W + 31) / 32, (H + 7) / 8);
  cudaStream_t st = as_stream(stream);
  switch (K) {
    case 4: k_render<4><<<grid, block, 0, st>>>(geo, met, col, capacity, H, W, m4, rgb); break;
    case 8: k_render<8><<<grid, block, 0, st>>>(geo, met, col, capacity, H, W, m4, rgb); break;
    default: k_render<16><<<grid, block, 0, st>>>(geo, met, col, capacity, H, W, m4, rgb); break;
  }
  return check_launch("k_render");
}

int sad_decode_points(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                      const uint32_t* map, const float* xy, int64_t n, float* rgb,
                      void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (n < 0) return einval("sad_decode_points: n must be >= 0");
  if (n == 0) return SAD_OK;
  if (!map || !rgb || !xy || (!prep && capacity > 0)) return einval("sad_decode_points: null pointer");
  if (!aligned16(map) || !aligned16(prep) || (reinterpret_cast<uintptr_t>(xy) & 7u))
    return einval("sad_decode_points: misaligned pointer");
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  const float4 *geo = p4, *met = p4 + capacity, *col = p4 + 2 * (size_t)capacity;
  const uint4* m4 = reinterpret_cast<const uint4*>(map);
  const float2* q = reinterpret_cast<const float2*>(xy);
  const int bs = 256;
  const unsigned grid = static_cast<unsigned>((n + bs - 1) / bs);
  cudaStream_t st = as_stream(stream);
  switch (K) {
    case 4: k_decode<4><<<grid, bs, 0, st>>>(geo, met, col, capacity, H, W, m4, q, n, rgb); break;
    case 8: k_decode<8><<<grid, bs, 0, st>>>(geo, met, col, capacity, H, W, m4, q, n, rgb); break;
    default: k_decode<16><<<grid, bs, 0, st>>>(geo, met, col, capacity, H, W, m4, q, n, rgb); break;
  }
  return check_launch("k_decode");
}

}  // extern "C"
