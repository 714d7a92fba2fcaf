// Device-side building blocks shared by the SAD kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sad {

constexpr uint32_t kInvalid = 0xffffffffu;
constexpr int kNParams = 11;
enum Plane { PX = 0, PY, PLOGTAU, PR, PCR, PCG, PCB, PUX, PUY, PA, PB };

// ---------------------------------------------------------------------------
// Reproducible float32 exponential.  Published method: Cody & Waite (1980)
// two-constant argument reduction x = k ln2 + r (ln 2 split into a 16-bit head,
// so k*head is exact), degree-7 Taylor polynomial of e^r (coefficients 1/k!,
// each the float nearest the rational) by Horner's rule, scaling by 2^k.  Every
// operation is an explicitly rounded fp32 op, so the result is identical on any
// IEEE machine that follows the same steps.  Input clamped to [-80, 80].
// ---------------------------------------------------------------------------
__device__ __forceinline__ float exp32_repro(float x) {
  x = x < -80.f ? -80.f : (x > 80.f ? 80.f : x);
  const float log2e = 0x1.715476p+0f;
  const float ln2_hi = 0x1.62e4p-1f;      // 45426 / 65536
  const float ln2_lo = 0x1.7f7d1cp-20f;   // ln 2 - ln2_hi, rounded
  const float k = rintf(__fmul_rn(x, log2e));
  float r = __fsub_rn(x, __fmul_rn(k, ln2_hi));
  r = __fsub_rn(r, __fmul_rn(k, ln2_lo));
  float p = 0x1.a01a02p-13f;                        // 1/7!
  p = __fadd_rn(__fmul_rn(p, r), 0x1.6c16c2p-10f);  // 1/6!
  p = __fadd_rn(__fmul_rn(p, r), 0x1.111112p-7f);   // 1/5!
  p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-5f);   // 1/4!
  p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-3f);   // 1/3!
  p = __fadd_rn(__fmul_rn(p, r), 0.5f);             // 1/2!
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  const int ki = static_cast<int>(k);
  const float scale = __int_as_float((ki + 127) << 23);  // 2^k, exact for |k| <= 116
  return __fmul_rn(p, scale);
}

// SplitMix64 (Steele, Lea & Flood 2014): output number ctr+1 of the generator
// whose state starts at `seed` (state advances by the golden-ratio increment).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Logit l = (tau s)(r - |x - p|_G) in a fixed fp32 operation order with no
// contraction (decides top-K membership, so it must be reproducible).
// geo = {x, y, tau*s, r}, met = {G00, G01, G11, active}.
__device__ __forceinline__ float score_exact(float px, float py, float4 geo, float4 met) {
  const float dx = __fsub_rn(px, geo.x);
  const float dy = __fsub_rn(py, geo.y);
  const float t0 = __fmul_rn(__fmul_rn(met.x, dx), dx);
  float t1 = __fmul_rn(__fmul_rn(met.y, dx), dy);
  t1 = __fadd_rn(t1, t1);
  const float t2 = __fmul_rn(__fmul_rn(met.z, dy), dy);
  const float q = __fadd_rn(__fadd_rn(t0, t1), t2);
  const float n = __fsqrt_rn(fmaxf(q, 0.f));
  return __fmul_rn(geo.z, __fsub_rn(geo.w, n));
}

// Same logit with free contraction, for the blend and its adjoint (tolerance
// based).  Also returns the pieces the adjoint needs.
struct ScoreParts {
  float l, n, dx, dy;
};
__device__ __forceinline__ ScoreParts score_fast(float px, float py, float4 geo, float4 met) {
  ScoreParts s;
  s.dx = px - geo.x;
  s.dy = py - geo.y;
  const float q = met.x * s.dx * s.dx + 2.f * met.y * s.dx * s.dy + met.z * s.dy * s.dy;
  s.n = sqrtf(fmaxf(q, 0.f));
  s.l = geo.z * (geo.w - s.n);
  return s;
}

// Top-K ordering: a precedes b iff la > lb, or la == lb and ida < idb.
__device__ __forceinline__ bool key_before(float la, uint32_t ia, float lb, uint32_t ib) {
  return la > lb || (la == lb && ia < ib);
}

// Derived table of one site (the "pack" of App. "Data Layout and Packing";
// metric G of Sec. 4.1), each fp32 operation explicitly rounded so that the
// result is reproducible: u = (ux,uy)/|(ux,uy)| (or (1,0)), e+ = exp(b+a),
// e- = exp(b-a), G00 = e+ ux^2 + e- uy^2, G01 = (e+ - e-) ux uy,
// G11 = e+ uy^2 + e- ux^2, tau s = exp(log_tau) s, active = (x >= 0).
// The blend record (ba, bb) is the same site folded for the softmax blend
// and its 36 bytes per (pixel, site) gather: with G' = (tau s)^2 G the logit
// is l = tau s r - sqrt(dx G' dx), so ba = {x, y, tau s r, G'00} (tau s r =
// -inf for an inactive site) and bb = {G'01, G'11, cr, cg}; cb goes to a
// dense plane (cbd: one float per site), whose 4-byte gathers spread over
// all 32 shared-memory banks of the L1 (cb inside the 16-byte colour record
// falls on 8 of them).
__device__ __forceinline__ void prepare_site(float x, float y, float logtau, float r, float cr,
                                             float cg, float cb, float ux, float uy, float a,
                                             float b, float s, float4& geo, float4& met,
                                             float4& col, float4& ba, float4& bb, float& cbd) {
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
  const bool act = x >= 0.f;
  geo = make_float4(x, y, ts, r);
  met = make_float4(G00, G01, G11, act ? 1.f : 0.f);
  col = make_float4(cr, cg, cb, 0.f);
  const float t2 = ts * ts;
  ba = make_float4(x, y, act ? ts * r : -INFINITY, t2 * G00);
  bb = make_float4(t2 * G01, t2 * G11, cr, cg);
  cbd = cb;
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}

}  // namespace sad
