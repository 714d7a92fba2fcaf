// The soft blend of Sec. 4.2 over a pixel's listed sites, shared by the
// render, decode and batched decode kernels.
#pragma once

#include "sad_device.cuh"
#include "sad_topk.cuh"

namespace sad {

// Blend of the listed sites at point (px, py), streamed two entries at a time
// with an online max-subtracted softmax: m = running max of the logits,
// z = sum exp(l - m), c = sum exp(l - m) c_i, rescaled by exp(m_old - m_new)
// when the max grows (the same w_i = exp(l_i - m)/z in exact arithmetic, no
// per-entry state kept).  Lists are sorted by logit, so the rescale is a
// rare branch rather than a second exponential per entry.  Black if no
// listed site is valid.
__device__ __forceinline__ void blend_step(float l, bool ok, float4 ck, float& m, float& z, float3& c) {
  if (!ok) return;
  if (l > m) {  // a new maximum: rare after the first entry (lists are sorted by logit)
    const float a = __expf(m - l);
    z *= a;
    c.x *= a;
    c.y *= a;
    c.z *= a;
    m = l;
  }
  const float b = l == m ? 1.f : __expf(l - m);
  z += b;
  c.x += b * ck.x;
  c.y += b * ck.y;
  c.z += b * ck.z;
}

// The blend reads each listed site's blend record (two 16-byte gathers,
// {x, y, tau s r, G'00} and {G'01, G'11, cr, cg}, plus cb from the dense
// blue plane: 36 bytes per (pixel, site)), with l = tau s r - sqrt(dx G' dx).
// m_out / iz_out (optional): the max logit and 1/Z of the blend (0 if no
// listed site is valid), the per-pixel state the saved-forward adjoint reads.
template <int NP>
__device__ __forceinline__ float3 blend_planes(const uint4* __restrict__ map, size_t P, size_t q,
                                               float px, float py, SiteRange sr,
                                               const float4* __restrict__ ba,
                                               const float4* __restrict__ bb,
                                               const float* __restrict__ cbd,
                                               float* m_out = nullptr, float* iz_out = nullptr) {
  float m = -INFINITY, z = 0.f;
  float3 c = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const uint4 v = ldg(&map[j * P + q]);
    const uint32_t id4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int u0 = 0; u0 < 4; u0 += 2) {
      float4 A[2], B[2];
      float cb[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint32_t id = sr.has(id4[u0 + u]) ? id4[u0 + u] : sr.lo;  // clamped: loads issue early
        A[u] = ldg(&ba[id]);
        B[u] = ldg(&bb[id]);
        cb[u] = ldg(&cbd[id]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const bool ok = sr.has(id4[u0 + u]) && A[u].z > -INFINITY;  // an inactive site has -inf
        const float dx = px - A[u].x, dy = py - A[u].y;
        const float qq = A[u].w * dx * dx + 2.f * B[u].x * dx * dy + B[u].y * dy * dy;
        const float l = A[u].z - sqrtf(fmaxf(qq, 0.f));
        blend_step(l, ok, make_float4(B[u].z, B[u].w, cb[u], 0.f), m, z, c);
      }
    }
  }
  float iz = 0.f;
  if (z > 0.f) {
    iz = 1.f / z;
    c.x *= iz;
    c.y *= iz;
    c.z *= iz;
  }
  if (m_out) *m_out = z > 0.f ? m : 0.f;
  if (iz_out) *iz_out = iz;
  return c;
}

}  // namespace sad
