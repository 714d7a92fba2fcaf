// Packed 16-byte evaluation sites (App. "Data Layout and Packing", Packed
// storage for evaluation): pack, unpack and a random-access decode that
// reads the 16-byte records directly.
//
// Words per site: w0 = x, y as 15-bit UNORM of x/W, y/H, active flag in bit
// 31; w1 = colour as 11/11/10-bit UNORM over per-image ranges; w2 = (log tau,
// r) as 16/16-bit UNORM over per-image ranges; w3 = 16-bit angle code of u
// over [-pi, pi] and a as float16.  The sites' b is folded into (log tau, r):
// tau s (r - e^{b/2} n0) = (tau e^{b/2}) s (r e^{-b/2} - n0).  Quantisation is
// computed in double from the float32 parameters, so pack and unpack are
// reproducible bit for bit; the decode unpacks in float32.
#include <cuda_fp16.h>

#include <cmath>

#include "sad_blend.cuh"
#include "sad_device.cuh"
#include "sad_host.h"

namespace sad {

constexpr int kPackQ = 10;  // (lo, hi) of log tau', r', colour r, g, b

__device__ __forceinline__ uint32_t ord_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ord(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ void fold_b(float lt, float r, float b, float& lt2, float& r2) {
  lt2 = static_cast<float>(static_cast<double>(lt) + static_cast<double>(b) / 2.0);
  r2 = static_cast<float>(static_cast<double>(r) * exp(-static_cast<double>(b) / 2.0));
}

__device__ __forceinline__ uint32_t unorm_code(float v, float lo, float hi, int bits) {
  const double top = static_cast<double>((1u << bits) - 1u);
  const double d = static_cast<double>(hi) - static_cast<double>(lo);
  if (!(d > 0.0)) return 0u;
  double t = (static_cast<double>(v) - static_cast<double>(lo)) / d * top;
  t = t < 0.0 ? 0.0 : (t > top ? top : t);
  return static_cast<uint32_t>(rint(t));
}

__device__ __forceinline__ float unorm_value(uint32_t c, float lo, float hi, int bits) {
  const double top = static_cast<double>((1u << bits) - 1u);
  return static_cast<float>(static_cast<double>(lo) +
                            static_cast<double>(c) / top * (static_cast<double>(hi) - static_cast<double>(lo)));
}

__global__ void k_pack_init(uint32_t* qb) {
  const int i = threadIdx.x;
  if (i < kPackQ) qb[i] = (i & 1) ? 0u : 0xffffffffu;  // lo: +max, hi: -max (orderable)
}

__global__ void k_pack_range(const float* __restrict__ params, int cap, uint32_t* qb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  if (!(params[PX * c + i] >= 0.f)) return;
  float lt, r;
  fold_b(params[PLOGTAU * c + i], params[PR * c + i], params[PB * c + i], lt, r);
  const float v[5] = {lt, r, params[PCR * c + i], params[PCG * c + i], params[PCB * c + i]};
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    atomicMin(&qb[2 * j], ord_bits(v[j]));
    atomicMax(&qb[2 * j + 1], ord_bits(v[j]));
  }
}

__global__ void k_pack_finish(uint32_t* qb) {
  const int i = threadIdx.x;
  if (i >= kPackQ / 2) return;
  const uint32_t lo = qb[2 * i], hi = qb[2 * i + 1];
  const bool none = lo == 0xffffffffu && hi == 0u;  // no active site
  float* q = reinterpret_cast<float*>(qb);
  q[2 * i] = none ? 0.f : from_ord(lo);
  q[2 * i + 1] = none ? 0.f : from_ord(hi);
}

__global__ void k_pack_words(const float* __restrict__ params, int cap, float H, float W,
                             const float* __restrict__ q, uint4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  const float x = params[PX * c + i];
  if (!(x >= 0.f)) {
    out[i] = make_uint4(0u, 0u, 0u, 0u);
    return;
  }
  float lt, r;
  fold_b(params[PLOGTAU * c + i], params[PR * c + i], params[PB * c + i], lt, r);
  auto pos = [](float v, float ext) {
    double t = static_cast<double>(v) / static_cast<double>(ext);
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    return static_cast<uint32_t>(rint(t * 32767.0));
  };
  const uint32_t xq = pos(x, W), yq = pos(params[PY * c + i], H);
  const double th = atan2(static_cast<double>(params[PUY * c + i]), static_cast<double>(params[PUX * c + i]));
  double ta = (th + M_PI) / (2.0 * M_PI);
  ta = ta < 0.0 ? 0.0 : (ta > 1.0 ? 1.0 : ta);
  const uint32_t aq = static_cast<uint32_t>(rint(ta * 65535.0));
  const uint32_t ah = __half_as_ushort(__float2half_rn(params[PA * c + i]));
  uint4 w;
  w.x = xq | (yq << 15) | (1u << 31);
  w.y = unorm_code(params[PCR * c + i], q[4], q[5], 11) | (unorm_code(params[PCG * c + i], q[6], q[7], 11) << 11) |
        (unorm_code(params[PCB * c + i], q[8], q[9], 10) << 22);
  w.z = unorm_code(lt, q[0], q[1], 16) | (unorm_code(r, q[2], q[3], 16) << 16);
  w.w = aq | (ah << 16);
  out[i] = w;
}

__global__ void k_unpack(const uint4* __restrict__ words, const float* __restrict__ q, int cap,
                         float H, float W, float* __restrict__ params) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  const uint4 w = words[i];
  const bool act = (w.x >> 31) & 1u;
  params[PX * c + i] = act ? static_cast<float>(static_cast<double>(w.x & 0x7fffu) / 32767.0 * W) : -1.f;
  params[PY * c + i] =
      act ? static_cast<float>(static_cast<double>((w.x >> 15) & 0x7fffu) / 32767.0 * H) : -1.f;
  params[PLOGTAU * c + i] = unorm_value(w.z & 0xffffu, q[0], q[1], 16);
  params[PR * c + i] = unorm_value(w.z >> 16, q[2], q[3], 16);
  params[PCR * c + i] = unorm_value(w.y & 0x7ffu, q[4], q[5], 11);
  params[PCG * c + i] = unorm_value((w.y >> 11) & 0x7ffu, q[6], q[7], 11);
  params[PCB * c + i] = unorm_value(w.y >> 22, q[8], q[9], 10);
  const double th = static_cast<double>(w.w & 0xffffu) / 65535.0 * (2.0 * M_PI) - M_PI;
  params[PUX * c + i] = static_cast<float>(cos(th));
  params[PUY * c + i] = static_cast<float>(sin(th));
  params[PA * c + i] = __half2float(__ushort_as_half(static_cast<unsigned short>(w.w >> 16)));
  params[PB * c + i] = 0.f;
}

// Per-call constants of the float32 unpacking in the decode.
struct PackDecode {
  float sx, sy;                 // W / 32767, H / 32767
  float lo[5], step[5];         // range start and code step of log tau', r', cr, cg, cb
  float s;                      // 1 / max(H, W)
};

// One listed site unpacked and prepared in float32: geo {x,y,tau s,r},
// metric {G00,G01,G11,active}, colour.
__device__ __forceinline__ void unpack_prepared(uint4 w, const PackDecode& D, float4& g, float4& m,
                                                float4& col) {
  const float act = (w.x >> 31) ? 1.f : 0.f;
  const float x = static_cast<float>(w.x & 0x7fffu) * D.sx;
  const float y = static_cast<float>((w.x >> 15) & 0x7fffu) * D.sy;
  const float lt = fmaf(static_cast<float>(w.z & 0xffffu), D.step[0], D.lo[0]);
  const float r = fmaf(static_cast<float>(w.z >> 16), D.step[1], D.lo[1]);
  col = make_float4(fmaf(static_cast<float>(w.y & 0x7ffu), D.step[2], D.lo[2]),
                    fmaf(static_cast<float>((w.y >> 11) & 0x7ffu), D.step[3], D.lo[3]),
                    fmaf(static_cast<float>(w.y >> 22), D.step[4], D.lo[4]), 0.f);
  float su, cu;
  sincospif(static_cast<float>(w.w & 0xffffu) * (2.f / 65535.f) - 1.f, &su, &cu);
  const float a = __half2float(__ushort_as_half(static_cast<unsigned short>(w.w >> 16)));
  const float ep = __expf(a), em = __expf(-a);
  g = make_float4(x, y, __expf(lt) * D.s, r);
  m = make_float4(ep * cu * cu + em * su * su, (ep - em) * cu * su, ep * su * su + em * cu * cu, act);
}

template <int K>
__global__ void __launch_bounds__(256) k_decode_packed(const uint4* __restrict__ words, int cap,
                                                       PackDecode D, int H, int W,
                                                       const uint4* __restrict__ map,
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
  const size_t q = static_cast<size_t>(cy) * W + cx;
  float m = -INFINITY, z = 0.f;
  float3 c = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 0; j < K / 4; ++j) {
    const uint4 v = ldg(&map[j * P + q]);
    const uint32_t id4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t id = id4[u];
      const bool in = id < static_cast<uint32_t>(cap);
      const uint4 w = ldg(&words[in ? id : 0u]);
      float4 g, mt, ck;
      unpack_prepared(w, D, g, mt, ck);
      blend_step(score_fast(p.x, p.y, g, mt).l, in && mt.w != 0.f, ck, m, z, c);
    }
  }
  if (z > 0.f) {
    const float iz = 1.f / z;
    c.x *= iz;
    c.y *= iz;
    c.z *= iz;
  }
  rgb[3 * i] = c.x;
  rgb[3 * i + 1] = c.y;
  rgb[3 * i + 2] = c.z;
}

// Full-image render from the packed records (the paper's evaluation render).
template <int K>
__global__ void __launch_bounds__(256) k_render_packed(const uint4* __restrict__ words, int cap,
                                                       PackDecode D, int H, int W,
                                                       const uint4* __restrict__ map,
                                                       float* __restrict__ rgb) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  const size_t P = static_cast<size_t>(H) * W;
  const size_t q = static_cast<size_t>(y) * W + x;
  const float px = x + 0.5f, py = y + 0.5f;
  float m = -INFINITY, z = 0.f;
  float3 c = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 0; j < K / 4; ++j) {
    const uint4 v = ldg(&map[j * P + q]);
    const uint32_t id4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t id = id4[u];
      const bool in = id < static_cast<uint32_t>(cap);
      const uint4 w = ldg(&words[in ? id : 0u]);
      float4 g, mt, ck;
      unpack_prepared(w, D, g, mt, ck);
      blend_step(score_fast(px, py, g, mt).l, in && mt.w != 0.f, ck, m, z, c);
    }
  }
  if (z > 0.f) {
    const float iz = 1.f / z;
    c.x *= iz;
    c.y *= iz;
    c.z *= iz;
  }
  rgb[3 * q] = c.x;
  rgb[3 * q + 1] = c.y;
  rgb[3 * q + 2] = c.z;
}

static PackDecode pack_decode(const float* q_host, int H, int W) {
  PackDecode D;
  D.sx = static_cast<float>(W) / 32767.f;
  D.sy = static_cast<float>(H) / 32767.f;
  const int bits[5] = {16, 16, 11, 11, 10};
  for (int j = 0; j < 5; ++j) {
    D.lo[j] = q_host[2 * j];
    D.step[j] = (q_host[2 * j + 1] - q_host[2 * j]) / static_cast<float>((1u << bits[j]) - 1u);
  }
  D.s = 1.0f / static_cast<float>(H > W ? H : W);
  return D;
}

}  // namespace sad

using namespace sad;

extern "C" {

int sad_pack_sites(const float* params, int32_t capacity, int32_t H, int32_t W, uint32_t* packed,
                   float* q, void* stream) {
  if (int st = check_problem(capacity, H, W, 4, false)) return st;
  if (!q || (capacity > 0 && (!params || !packed))) return einval("sad_pack_sites: null pointer");
  if (!aligned16(packed)) return einval("sad_pack_sites: packed must be 16-byte aligned");
  cudaStream_t st = as_stream(stream);
  uint32_t* qb = reinterpret_cast<uint32_t*>(q);
  { TraceScope tr_(st, "k_pack_init"); k_pack_init<<<1, 32, 0, st>>>(qb); }
  if (capacity > 0) {
    TraceScope tr_(st, "k_pack_range");
    k_pack_range<<<(capacity + 255) / 256, 256, 0, st>>>(params, capacity, qb);
  }
  { TraceScope tr_(st, "k_pack_finish"); k_pack_finish<<<1, 32, 0, st>>>(qb); }
  if (capacity > 0) {
    TraceScope tr_(st, "k_pack_words");
    k_pack_words<<<(capacity + 255) / 256, 256, 0, st>>>(params, capacity, static_cast<float>(H),
                                                          static_cast<float>(W), q,
                                                          reinterpret_cast<uint4*>(packed));
  }
  return check_launch("sad_pack_sites");
}

int sad_unpack_sites(const uint32_t* packed, const float* q, int32_t capacity, int32_t H, int32_t W,
                     float* params, void* stream) {
  if (int st = check_problem(capacity, H, W, 4, false)) return st;
  if (capacity == 0) return SAD_OK;
  if (!packed || !q || !params) return einval("sad_unpack_sites: null pointer");
  if (!aligned16(packed)) return einval("sad_unpack_sites: packed must be 16-byte aligned");
  cudaStream_t st = as_stream(stream);
  {
    TraceScope tr_(st, "k_unpack");
    k_unpack<<<(capacity + 255) / 256, 256, 0, st>>>(reinterpret_cast<const uint4*>(packed), q, capacity,
                                                     static_cast<float>(H), static_cast<float>(W), params);
  }
  return check_launch("k_unpack");
}

int sad_decode_packed(const uint32_t* packed, const float* q_host, int32_t capacity, int32_t H,
                      int32_t W, int32_t K, const uint32_t* map, const float* xy, int64_t n,
                      float* rgb, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (n < 0) return einval("sad_decode_packed: n must be >= 0");
  if (n == 0) return SAD_OK;
  if (!q_host || !map || !xy || !rgb || (capacity > 0 && !packed))
    return einval("sad_decode_packed: null pointer");
  if (!aligned16(map) || !aligned16(packed) || (reinterpret_cast<uintptr_t>(xy) & 7u))
    return einval("sad_decode_packed: misaligned pointer");
  const PackDecode D = pack_decode(q_host, H, W);
  const unsigned grid = static_cast<unsigned>((n + 255) / 256);
  cudaStream_t st = as_stream(stream);
  const uint4* w4 = reinterpret_cast<const uint4*>(packed);
  const uint4* m4 = reinterpret_cast<const uint4*>(map);
  const float2* q2 = reinterpret_cast<const float2*>(xy);
  {
    TraceScope tr_(st, "k_decode_packed");
    switch (K) {
      case 4: k_decode_packed<4><<<grid, 256, 0, st>>>(w4, capacity, D, H, W, m4, q2, n, rgb); break;
      case 8: k_decode_packed<8><<<grid, 256, 0, st>>>(w4, capacity, D, H, W, m4, q2, n, rgb); break;
      default: k_decode_packed<16><<<grid, 256, 0, st>>>(w4, capacity, D, H, W, m4, q2, n, rgb); break;
    }
  }
  return check_launch("k_decode_packed");
}

int sad_render_packed(const uint32_t* packed, const float* q_host, int32_t capacity, int32_t H,
                      int32_t W, int32_t K, const uint32_t* map, float* rgb, void* stream) {
  if (int st = check_problem(capacity, H, W, K, true)) return st;
  if (!q_host || !map || !rgb || (capacity > 0 && !packed)) return einval("sad_render_packed: null pointer");
  if (!aligned16(map) || !aligned16(packed)) return einval("sad_render_packed: misaligned pointer");
  const PackDecode D = pack_decode(q_host, H, W);
  const dim3 block(32, 8);
  const dim3 grid((W + 31) / 32, (H + 7) / 8);
  cudaStream_t st = as_stream(stream);
  const uint4* w4 = reinterpret_cast<const uint4*>(packed);
  const uint4* m4 = reinterpret_cast<const uint4*>(map);
  {
    TraceScope tr_(st, "k_render_packed");
    switch (K) {
      case 4: k_render_packed<4><<<grid, block, 0, st>>>(w4, capacity, D, H, W, m4, rgb); break;
      case 8: k_render_packed<8><<<grid, block, 0, st>>>(w4, capacity, D, H, W, m4, rgb); break;
      default: k_render_packed<16><<<grid, block, 0, st>>>(w4, capacity, D, H, W, m4, rgb); break;
    }
  }
  return check_launch("k_render_packed");
}

}  // extern "C"
