// Forward blend (Sec. 4.2) over the cached top-K lists: full-image render and
// random-access decode at float coordinates.
#include "sad_blend.cuh"
#include "sad_device.cuh"
#include "sad_host.h"

namespace sad {

// fwd (optional): float32[2][H*W] planes {max logit m, 1/Z} of every pixel.
template <int K, bool SAVE>
__global__ void __launch_bounds__(256, 5) k_render(const float4* __restrict__ geo,
                                                const float4* __restrict__ met,
                                                const float4* __restrict__ col, int cap, int H,
                                                int W, const uint4* __restrict__ map,
                                                float* __restrict__ rgb, float* __restrict__ fwd) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  const size_t P = static_cast<size_t>(H) * W;
  const size_t q = static_cast<size_t>(y) * W + x;
  float m, iz;
  const float3 c = blend_planes<K / 4>(map, P, q, x + 0.5f, y + 0.5f,
                                      SiteRange{0u, static_cast<uint32_t>(cap)}, geo + 3 * static_cast<size_t>(cap),
                                      geo + 4 * static_cast<size_t>(cap),
                                      reinterpret_cast<const float*>(geo + 5 * static_cast<size_t>(cap)),
                                      SAVE ? &m : nullptr, SAVE ? &iz : nullptr);
  rgb[3 * q] = c.x;
  rgb[3 * q + 1] = c.y;
  rgb[3 * q + 2] = c.z;
  if (SAVE) {
    fwd[q] = m;
    fwd[P + q] = iz;
  }
}

template <int K>
__global__ void __launch_bounds__(256, 5) k_decode(const float4* __restrict__ geo,
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
  const float3 c = blend_planes<K / 4>(map, P, static_cast<size_t>(cy) * W + cx, p.x, p.y,
                                       SiteRange{0u, static_cast<uint32_t>(cap)}, geo + 3 * static_cast<size_t>(cap),
                                       geo + 4 * static_cast<size_t>(cap),
                                       reinterpret_cast<const float*>(geo + 5 * static_cast<size_t>(cap)));
  rgb[3 * i] = c.x;
  rgb[3 * i + 1] = c.y;
  rgb[3 * i + 2] = c.z;
}

}  // namespace sad

using namespace sad;

extern "C" {

static int run_render(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                      const uint32_t* map, float* rgb, float* fwd, void* stream, const char* name) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (!map || !rgb || (!prep && capacity > 0)) return einval("%s: null pointer", name);
  if (!aligned16(map) || !aligned16(prep)) return einval("%s: pointers must be 16-byte aligned", name);
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  const float4 *geo = p4, *met = p4 + capacity, *col = p4 + 2 * (size_t)capacity;
  const uint4* m4 = reinterpret_cast<const uint4*>(map);
  const dim3 block(32, 8);
  const dim3 grid((W + 31) / 32, (H + 7) / 8);
  cudaStream_t st = as_stream(stream);
  TraceScope tr_(st, "k_render");
#define SAD_RENDER(KK) \
  (fwd ? k_render<KK, true><<<grid, block, 0, st>>>(geo, met, col, capacity, H, W, m4, rgb, fwd) \
       : k_render<KK, false><<<grid, block, 0, st>>>(geo, met, col, capacity, H, W, m4, rgb, nullptr))
  switch (K) {
    case 4: SAD_RENDER(4); break;
    case 8: SAD_RENDER(8); break;
    default: SAD_RENDER(16); break;
  }
#undef SAD_RENDER
  return check_launch("k_render");
}

int sad_render(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
               const uint32_t* map, float* rgb, void* stream) {
  return run_render(prep, capacity, H, W, K, map, rgb, nullptr, stream, "sad_render");
}

int sad_render_save(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                    const uint32_t* map, float* rgb, float* fwd, void* stream) {
  if (!fwd) return einval("sad_render_save: null fwd");
  return run_render(prep, capacity, H, W, K, map, rgb, fwd, stream, "sad_render_save");
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
    case 4: { TraceScope tr_(st, "k_decode"); k_decode<4><<<grid, bs, 0, st>>>(geo, met, col, capacity, H, W, m4, q, n, rgb); } break;
    case 8: { TraceScope tr_(st, "k_decode"); k_decode<8><<<grid, bs, 0, st>>>(geo, met, col, capacity, H, W, m4, q, n, rgb); } break;
    default: { TraceScope tr_(st, "k_decode"); k_decode<16><<<grid, bs, 0, st>>>(geo, met, col, capacity, H, W, m4, q, n, rgb); } break;
  }
  return check_launch("k_decode");
}

}  // extern "C"
