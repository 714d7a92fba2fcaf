// Adjoint of the blend (App. "Gradient Computation and Reduction", Per-pixel gradients) with an atomic-free,
// deterministic gradient reduction that replaces the per-tile hash table plus
// global float atomics of Sec. 4.8, Alg. 1 (threadgroup hash reduction).
//
// Per 16x16 pixel tile (one CTA, one pixel per thread):
//  1. forward: every pixel recomputes its max-subtracted softmax over its K
//     listed sites (nothing from the forward pass is stored), forms its
//     upstream gradient g (given, or 2(c - I)/P for the fused MSE loss) and
//     parks {m, 1/Z, cbar, g} in shared memory;
//  2. the tile's distinct sites get slots in a shared hash table (the paper's
//     multiplicative hash, linear probing); each warp records, per slot, the
//     bitmask of its 32 pixels that list the site (__match_any_sync, no
//     atomics: a warp owns its mask word);
//  3. the masks give each slot a stable, pixel-ordered pair list; one warp
//     walks a slot's list 32 pairs at a time with the site's parameters in
//     registers (lane i takes pairs i, i+32, ...) and a fixed butterfly sums
//     the lane partials, giving ten sufficient statistics per (site, tile):
//       sum w g (3),  sum d,  sum d n,  sum d dx/n,  sum d dy/n,
//       sum d dx^2/n, sum d dx dy/n, sum d dy^2/n,   d = dL/dl = w g.(c_k - cbar)
//     written as one partial record per (site, tile).  If the table fills,
//     the remaining sites are handled in further rounds.
// Then every record's statistics are added into per-site sums in exact
// 64-bit fixed point (integer atomics, per-statistic scale from the largest
// record value), which makes each site's total independent of the order of
// the additions; the eleven parameter gradients follow from the statistics by
// the chain rule through G(a, b, u) of Sec. 4.1.
#include "sad_device.cuh"
#include "sad_host.h"

#include <mutex>

namespace sad {

constexpr int kTileSide = 16;
constexpr int kTileThreads = kTileSide * kTileSide;
constexpr int kSlots = 128;  // shared hash table size per round (power of 2)
constexpr int kLog2Slots = 7;
constexpr uint32_t kNone = 0xffffffffu;
constexpr int kModeGrad = 0;
constexpr int kModeStats = 1;

struct alignas(16) Record {
  uint32_t site;
  uint32_t tile;
  float acc[10];
};
static_assert(sizeof(Record) == 48, "record layout");

struct WsHeader {
  uint32_t cursor;     // records written
  uint32_t overflow;   // records that did not fit
  uint32_t pmax[10];   // per statistic: bits of the largest |value| of any record
  uint32_t pad[52];
};
static_assert(sizeof(WsHeader) == 256, "header layout");

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
struct WsLayout {
  size_t hdr, tile_loss, records, acc, total;
  uint32_t max_records, n_tiles;
};

static inline size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

// records: 48 B per (site, tile); acc: 10 int64 fixed-point sums per site
static WsLayout ws_layout(int H, int W, int K, int cap, int64_t max_records) {
  WsLayout L{};
  const uint64_t tiles_x = (W + kTileSide - 1) / kTileSide;
  const uint64_t tiles_y = (H + kTileSide - 1) / kTileSide;
  L.n_tiles = static_cast<uint32_t>(tiles_x * tiles_y);
  uint64_t mr = max_records > 0 ? static_cast<uint64_t>(max_records)
                                : static_cast<uint64_t>(H) * W * K / 8;
  if (max_records <= 0 && mr < 128ull * L.n_tiles) mr = 128ull * L.n_tiles;
  if (mr > 0xfffffff0ull) mr = 0xfffffff0ull;
  L.max_records = static_cast<uint32_t>(mr);
  size_t o = 0;
  L.hdr = o;        o = align256(o + sizeof(WsHeader));
  L.tile_loss = o;  o = align256(o + sizeof(float) * L.n_tiles);
  L.acc = o;        o = align256(o + sizeof(unsigned long long) * 10 * static_cast<size_t>(cap));
  L.records = o;    o = align256(o + sizeof(Record) * L.max_records);
  L.total = o;
  return L;
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan of a 64-bit value over 256 threads (fixed order)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t block_excl_scan256(uint64_t v, uint64_t* warp_tot,
                                                       uint64_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t run = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) {
      run += warp_tot[w];
      warp_tot[w] = run;
    }
  }
  __syncthreads();
  const uint64_t pre = warp ? warp_tot[warp - 1] : 0ull;
  total = warp_tot[kTileThreads / 32 - 1];
  __syncthreads();
  return pre + x - v;
}

__device__ __forceinline__ uint32_t probe_slot(uint32_t id, uint32_t* keys) {
  const uint32_t h = (id * 2654435761u) >> (32 - kLog2Slots);
  volatile uint32_t* vk = keys;
  for (int i = 0; i < kSlots; ++i) {
    const uint32_t s = (h + i) & (kSlots - 1);
    const uint32_t k = vk[s];
    if (k == id) return s;
    if (k == kInvalid) {
      const uint32_t old = atomicCAS(&keys[s], kInvalid, id);
      if (old == kInvalid || old == id) return s;
    }
  }
  return kNone;
}

// Sum 10 per-lane values over a warp by recursive halving (padded to 16):
// each stage sends half of the values to the partner lane and keeps the other
// half, so 8+4+2+1+1 shuffles replace the 5x10 of a butterfly.  The order of
// every addition is fixed.  Returns, on lane l, the total of value l/2
// (values 10..15 are padding).
__device__ __forceinline__ float warp_sum10_halving(const float (&in)[10], int lane) {
  float a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = j < 10 ? in[j] : 0.f;
#pragma unroll
  for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float keep = up ? a[h + j] : a[j];
      const float give = up ? a[j] : a[h + j];
      a[j] = keep + __shfl_xor_sync(0xffffffffu, give, o);
    }
  }
  return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// ---------------------------------------------------------------------------
// per-tile kernel
// ---------------------------------------------------------------------------
template <int K, int MODE>
__global__ void __launch_bounds__(kTileThreads, MODE == kModeStats ? 2 : 4) k_bwd_tile(
    const float4* __restrict__ geo, const float4* __restrict__ met,
    const float4* __restrict__ col, int cap, int H, int W, const uint4* __restrict__ map,
    const float* __restrict__ grad_rgb, const float* __restrict__ target, float two_over_P,
    float* __restrict__ rgb_out, float* __restrict__ tile_loss, Record* __restrict__ records,
    uint32_t max_records, WsHeader* __restrict__ hdr) {
  constexpr int kWarps = kTileThreads / 32;
  __shared__ uint32_t s_keys[kSlots];
  __shared__ uint32_t s_mask[kWarps][kSlots];   // [warp word][slot]: conflict-free per-slot reads
  __shared__ uint16_t s_wpre[kWarps][kSlots];
  __shared__ uint32_t s_cnt[kSlots];
  __shared__ uint32_t s_off[kSlots];
  __shared__ uint32_t s_rix[kSlots];
  __shared__ uint8_t s_list[kTileThreads * K];
  // per pixel.  gradient mode: {m, 1/Z, g.cbar, gx}, {gy, gz, -, -};
  // statistics mode: {m, 1/Z, cbar.x, cbar.y}, {cbar.z, I}, {c' of the
  // dominant site (blend without it), dominant id}
  __shared__ float4 s_pa[kTileThreads];
  __shared__ float2 s_pg[MODE == kModeStats ? 1 : kTileThreads];
  __shared__ float4 s_pb[MODE == kModeStats ? kTileThreads : 1];
  __shared__ float4 s_pc[MODE == kModeStats ? kTileThreads : 1];
  __shared__ uint64_t s_scan[kWarps];
  __shared__ float s_red[kWarps];
  __shared__ uint32_t s_base;
  __shared__ uint32_t s_pmax[10];

  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const uint32_t tiles_x = (W + kTileSide - 1) / kTileSide;
  const uint32_t tile = blockIdx.x;
  const int x0 = (tile % tiles_x) * kTileSide;
  const int y0 = (tile / tiles_x) * kTileSide;
  const int x = x0 + (t & (kTileSide - 1));
  const int y = y0 + (t >> 4);
  const bool inimg = x < W && y < H;
  const size_t P = static_cast<size_t>(H) * W;
  const size_t q = inimg ? static_cast<size_t>(y) * W + x : 0;
  const uint32_t ucap = static_cast<uint32_t>(cap);
  const float px = x + 0.5f, py = y + 0.5f;
  if (t < 10) s_pmax[t] = 0u;

  // ---- 1. per-pixel forward --------------------------------------------
  uint32_t ids[K];
#pragma unroll
  for (int j = 0; j < K / 4; ++j) {
    uint4 v = make_uint4(kInvalid, kInvalid, kInvalid, kInvalid);
    if (inimg) v = ldg(&map[j * P + q]);
    ids[4 * j] = v.x;
    ids[4 * j + 1] = v.y;
    ids[4 * j + 2] = v.z;
    ids[4 * j + 3] = v.w;
  }
  float m = -INFINITY;
  float z = 0.f;
  float3 cb = make_float3(0.f, 0.f, 0.f);
  uint32_t vm = 0;
  float l[MODE == kModeStats ? K : 1];
  if (MODE == kModeStats) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      l[k] = -INFINITY;
      if (ids[k] < ucap) {
        const float4 mt = ldg(&met[ids[k]]);
        if (mt.w != 0.f) {
          l[k] = score_fast(px, py, ldg(&geo[ids[k]]), mt).l;
          vm |= 1u << k;
          m = fmaxf(m, l[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (vm >> k & 1u) {
        const float e = __expf(l[k] - m);
        const float4 ck = ldg(&col[ids[k]]);
        z += e;
        cb.x += e * ck.x;
        cb.y += e * ck.y;
        cb.z += e * ck.z;
      }
    }
  } else {
    // online max-subtracted softmax over the list, kB entries at a time
    constexpr int kB = 1;
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += kB) {
      float4 g[kB], mt[kB], ck[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const uint32_t id = ids[k0 + u] < ucap ? ids[k0 + u] : 0u;
        g[u] = ldg(&geo[id]);
        mt[u] = ldg(&met[id]);
        ck[u] = ldg(&col[id]);
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const bool ok = ids[k0 + u] < ucap && mt[u].w != 0.f;
        vm |= ok ? (1u << (k0 + u)) : 0u;
        const float lk = score_fast(px, py, g[u], mt[u]).l;
        const float mn = ok ? fmaxf(m, lk) : m;
        const float a = m == mn ? 1.f : __expf(m - mn);   // unchanged max (or still -inf): 1
        const float b = ok ? (lk == mn ? 1.f : __expf(lk - mn)) : 0.f;
        z = z * a + b;
        cb.x = cb.x * a + b * ck[u].x;
        cb.y = cb.y * a + b * ck[u].y;
        cb.z = cb.z * a + b * ck[u].z;
        m = mn;
      }
    }
  }
  const float iz = vm ? 1.f / z : 0.f;
  cb.x *= iz;
  cb.y *= iz;
  cb.z *= iz;
  float3 g = make_float3(0.f, 0.f, 0.f);
  float lpx = 0.f;
  float3 I = make_float3(0.f, 0.f, 0.f);
  if (inimg) {
    if (grad_rgb) {
      g = make_float3(grad_rgb[3 * q], grad_rgb[3 * q + 1], grad_rgb[3 * q + 2]);
    } else {
      I = make_float3(target[3 * q], target[3 * q + 1], target[3 * q + 2]);
      const float rx = cb.x - I.x, ry = cb.y - I.y, rz = cb.z - I.z;
      lpx = rx * rx + ry * ry + rz * rz;
      g = make_float3(two_over_P * rx, two_over_P * ry, two_over_P * rz);
    }
    if (rgb_out) {
      rgb_out[3 * q] = cb.x;
      rgb_out[3 * q + 1] = cb.y;
      rgb_out[3 * q + 2] = cb.z;
    }
  }
  if (MODE == kModeStats) {
    // dominant site (first largest logit) and the blend of the others with
    // their own max subtracted
    int dk = -1;
    float ld = -INFINITY;
    uint32_t did = kInvalid;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool better = (vm >> k & 1u) && (dk < 0 || l[k] > ld);
      dk = better ? k : dk;
      ld = better ? l[k] : ld;
      did = better ? ids[k] : did;
    }
    float m2 = -INFINITY;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if ((vm >> k & 1u) && k != dk) m2 = fmaxf(m2, l[k]);
    float z2 = 0.f;
    float3 c2 = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if ((vm >> k & 1u) && k != dk) {
        const float e = __expf(l[k] - m2);
        const float4 ck = ldg(&col[ids[k]]);
        z2 += e;
        c2.x += e * ck.x;
        c2.y += e * ck.y;
        c2.z += e * ck.z;
      }
    }
    if (z2 > 0.f) {
      const float i2 = 1.f / z2;
      c2.x *= i2;
      c2.y *= i2;
      c2.z *= i2;
    }
    s_pa[t] = make_float4(m, iz, cb.x, cb.y);
    s_pb[t] = make_float4(cb.z, I.x, I.y, I.z);
    s_pc[t] = make_float4(c2.x, c2.y, c2.z, __uint_as_float(did));
  } else {
    s_pa[t] = make_float4(m, iz, g.x * cb.x + g.y * cb.y + g.z * cb.z, g.x);
    s_pg[t] = make_float2(g.y, g.z);
  }
  if (tile_loss) {  // deterministic tile sum of the per-pixel squared error
    float v = lpx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (t == 0) {
      float sum = 0.f;
      for (int w = 0; w < kWarps; ++w) sum += s_red[w];
      tile_loss[tile] = sum;
    }
  }

  // ---- 2..3. rounds: slot assignment, stable pair lists, warp per slot ---
  uint32_t pending = vm;
  uint32_t slot[K];
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (;;) {
    for (int i = t; i < kSlots; i += kTileThreads) {
      s_keys[i] = kInvalid;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s_mask[w][i] = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
      uint32_t sl = kNone;
      if (pending >> k & 1u) {
        sl = probe_slot(ids[k], s_keys);
        if (sl != kNone) pending &= ~(1u << k);
      }
      slot[k] = sl;
      // the warp's own mask word: OR is order independent, so the masks (and
      // the pair lists built from them) are deterministic
      if (sl != kNone) atomicOr(&s_mask[warp][sl], 1u << lane);
    }
    __syncthreads();
    uint64_t packed = 0;
    if (t < kSlots && s_keys[t] != kInvalid) {
      uint32_t c = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        s_wpre[w][t] = static_cast<uint16_t>(c);
        c += __popc(s_mask[w][t]);
      }
      packed = static_cast<uint64_t>(c) | (1ull << 32);
    }
    uint64_t total;
    const uint64_t ex = block_excl_scan256(packed, s_scan, total);
    if (t < kSlots) {
      s_cnt[t] = static_cast<uint32_t>(packed & 0xffffffffu);
      s_off[t] = static_cast<uint32_t>(ex & 0xffffffffu);
      s_rix[t] = static_cast<uint32_t>(ex >> 32);
    }
    if (t == 0) s_base = atomicAdd(&hdr->cursor, static_cast<uint32_t>(total >> 32));
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t sl = slot[k];
      if (sl != kNone) {
        const uint32_t pos = s_off[sl] + s_wpre[warp][sl] + __popc(s_mask[warp][sl] & lt_mask);
        s_list[pos] = static_cast<uint8_t>(t);
      }
    }
    __syncthreads();
    // one warp per slot: lanes walk the slot's pixel-ordered pairs, then a
    // fixed butterfly sums the 32 lane partials (deterministic order)
    for (int sl = warp; sl < kSlots; sl += kWarps) {
      const uint32_t cnt = s_cnt[sl];
      if (cnt == 0) continue;
      const uint32_t id = s_keys[sl];
      const uint32_t off = s_off[sl];
      const float4 gs = ldg(&geo[id]), ms = ldg(&met[id]), cs = ldg(&col[id]);
      float acc[10];
#pragma unroll
      for (int j = 0; j < 10; ++j) acc[j] = 0.f;
      for (uint32_t i = lane; i < cnt; i += 32) {
        const uint32_t p = s_list[off + i];
        const float4 A = s_pa[p];
        const float dx = (x0 + static_cast<int>(p & (kTileSide - 1)) + 0.5f) - gs.x;
        const float dy = (y0 + static_cast<int>(p >> 4) + 0.5f) - gs.y;
        const float qq = ms.x * dx * dx + 2.f * ms.y * dx * dy + ms.z * dy * dy;
        const float n = sqrtf(fmaxf(qq, 0.f));
        const float w = __expf(gs.z * (gs.w - n) - A.x) * A.y;
        if (MODE == kModeStats) {
          // A = {m, 1/Z, cbar.x, cbar.y}, B = {cbar.z, I}
          const float4 B = s_pb[p];
          const float ex = A.z - B.y, ey = A.w - B.z, ez = B.x - B.w;
          const float e = ex * ex + ey * ey + ez * ez;
          const float om = w * e;
          acc[0] += w;
          acc[1] += om;
          acc[2] += om * dx;
          acc[3] += om * dy;
          acc[4] += om * dx * dx;
          acc[5] += om * dx * dy;
          acc[6] += om * dy * dy;
          float3 cp;
          const float4 C = s_pc[p];
          if (__float_as_uint(C.w) == id) {
            cp = make_float3(C.x, C.y, C.z);
          } else {
            const float inv = 1.f / (1.f - w);
            cp = make_float3((A.z - w * cs.x) * inv, (A.w - w * cs.y) * inv, (B.x - w * cs.z) * inv);
          }
          const float fx = cp.x - B.y, fy = cp.y - B.z, fz = cp.z - B.w;
          acc[7] += fx * fx + fy * fy + fz * fz - e;
        } else {
          // A = {m, 1/Z, g.cbar, gx}, B = {gy, gz}
          const float2 B = s_pg[p];
          const float d = w * (A.w * cs.x + B.x * cs.y + B.y * cs.z - A.z);
          acc[0] += w * A.w;
          acc[1] += w * B.x;
          acc[2] += w * B.y;
          acc[3] += d;
          acc[4] += d * n;
          if (n > 0.f) {
            const float a = d / n;
            acc[5] += a * dx;
            acc[6] += a * dy;
            acc[7] += a * dx * dx;
            acc[8] += a * dx * dy;
            acc[9] += a * dy * dy;
          }
        }
      }
      // sum the 10 lane partials over the warp by recursive halving (fixed
      // order): afterwards lanes 2i and 2i+1 hold the total of statistic i
      const float tot = warp_sum10_halving(acc, lane);
      const uint32_t ridx = s_base + s_rix[sl];
      const int stat = lane >> 1;
      if (ridx < max_records) {
        float* dst = reinterpret_cast<float*>(&records[ridx]);
        if (lane == 0) {
          dst[0] = __uint_as_float(id);
          dst[1] = __uint_as_float(tile);
        }
        if ((lane & 1) == 0 && stat < 10) {
          const float v = isfinite(tot) ? tot : 0.f;  // non-finite contributions are dropped
          dst[2 + stat] = v;
          if (v != 0.f) atomicMax(&s_pmax[stat], __float_as_uint(fabsf(v)));
        }
      } else if (lane == 0) {
        hdr->overflow = 1u;
      }
    }
    if (!__syncthreads_or(pending != 0u)) break;
  }
  if (t < 10 && s_pmax[t]) atomicMax(&hdr->pmax[t], s_pmax[t]);
}

// ---------------------------------------------------------------------------
// per-site sums of the per-tile records in exact fixed point
//
// Statistic j of every record is scaled by 2^S_j, S_j = 61 - e_j - L with
// max_j |value| < 2^e_j and 2^L > number of records, rounded to an int64 and
// added with integer atomics: no sum can overflow, integer addition is
// associative, so each site's total is the same bit pattern whatever the order
// of the additions, and its rounding error is below 2^-(61-L) of the largest
// record value of that statistic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fixed_shift(uint32_t pmax_bits, uint32_t n_records) {
  if (pmax_bits == 0u) return 0;
  int e;
  frexpf(__uint_as_float(pmax_bits), &e);       // pmax < 2^e
  int L = 1;
  while (L < 32 && (1ull << L) <= n_records) ++L;  // 2^L > n_records
  return 61 - e - L;
}

template <int NV>
__global__ void k_seg_accum(const Record* __restrict__ rec, const WsHeader* __restrict__ hdr,
                            uint32_t max_records, int cap, unsigned long long* __restrict__ acc) {
  const uint32_t n = min(hdr->cursor, max_records);
  double scale[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) scale[j] = ldexp(1.0, fixed_shift(hdr->pmax[j], n));
  const size_t c = static_cast<size_t>(cap);
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const float4* src = reinterpret_cast<const float4*>(&rec[r]);
    const float4 r0 = src[0], r1 = src[1], r2 = src[2];
    const uint32_t site = __float_as_uint(r0.x);
    const float v[10] = {r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w};
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      if (v[j] != 0.f) {
        const long long q = __double2ll_rn(static_cast<double>(v[j]) * scale[j]);
        atomicAdd(&acc[j * c + site], static_cast<unsigned long long>(q));
      }
    }
  }
}

// Per site: the exact sums back to float, then the chain rule to 11 grads.
__global__ void k_site_grads(const float* __restrict__ params, const float4* __restrict__ geo,
                             const float4* __restrict__ met, int cap,
                             const WsHeader* __restrict__ hdr, uint32_t max_records,
                             const unsigned long long* __restrict__ accq,
                             float* __restrict__ grads) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  const uint32_t n = min(hdr->cursor, max_records);
  float acc[10];
  bool any = false;
#pragma unroll
  for (int j = 0; j < 10; ++j) {
    const long long q = static_cast<long long>(accq[j * c + i]);
    acc[j] = static_cast<float>(static_cast<double>(q) * ldexp(1.0, -fixed_shift(hdr->pmax[j], n)));
    any |= q != 0;
  }
  float out[kNParams];
#pragma unroll
  for (int j = 0; j < kNParams; ++j) out[j] = 0.f;
  if (any) {
    const float4 gs = geo[i], ms = met[i];
    const float ts = gs.z, r = gs.w;
    const float G00 = ms.x, G01 = ms.y, G11 = ms.z;
    const float rawx = params[PUX * c + i], rawy = params[PUY * c + i];
    const float a = params[PA * c + i], b = params[PB * c + i];
    const float nrm2 = rawx * rawx + rawy * rawy;
    float ux = 1.f, uy = 0.f;
    if (nrm2 > 0.f) {
      const float inv = rsqrtf(nrm2);
      ux = rawx * inv;
      uy = rawy * inv;
    }
    const float ep = expf(b + a), em = expf(b - a);
    const float gG00 = -0.5f * ts * acc[7];
    const float gG01 = -ts * acc[8];
    const float gG11 = -0.5f * ts * acc[9];
    out[PX] = ts * (G00 * acc[5] + G01 * acc[6]);
    out[PY] = ts * (G01 * acc[5] + G11 * acc[6]);
    out[PLOGTAU] = ts * (r * acc[3] - acc[4]);
    out[PR] = ts * acc[3];
    out[PCR] = acc[0];
    out[PCG] = acc[1];
    out[PCB] = acc[2];
    const float xx = ux * ux, yy = uy * uy, xy = ux * uy;
    out[PA] = gG00 * (ep * xx - em * yy) + gG01 * (ep + em) * xy + gG11 * (ep * yy - em * xx);
    out[PB] = gG00 * G00 + gG01 * G01 + gG11 * G11;
    const float gth = (ep - em) * (-2.f * xy * gG00 + (xx - yy) * gG01 + 2.f * xy * gG11);
    if (nrm2 > 0.f) {
      out[PUX] = -gth * rawy / nrm2;
      out[PUY] = gth * rawx / nrm2;
    }
  }
#pragma unroll
  for (int j = 0; j < kNParams; ++j) grads[j * c + i] = out[j];
}

// Per site: the exact statistic sums back to float (statistics mode).
__global__ void k_site_stats(int cap, const WsHeader* __restrict__ hdr, uint32_t max_records,
                             const unsigned long long* __restrict__ accq,
                             float* __restrict__ stats) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  const uint32_t n = min(hdr->cursor, max_records);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const long long q = static_cast<long long>(accq[j * c + i]);
    stats[j * c + i] =
        static_cast<float>(static_cast<double>(q) * ldexp(1.0, -fixed_shift(hdr->pmax[j], n)));
  }
}

__global__ void k_loss_final(const float* __restrict__ tile_loss, uint32_t n_tiles, float inv_P,
                             float* __restrict__ loss) {
  __shared__ float s_w[8];
  float v = 0.f;
  for (uint32_t i = threadIdx.x; i < n_tiles; i += 256) v += tile_loss[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += s_w[w];
    loss[0] = s * inv_P;
  }
}

// ---------------------------------------------------------------------------
static int run_backward(const float* params, const float* prep, int cap, int H, int W, int K,
                        const uint32_t* map, const float* grad_rgb, const float* target,
                        float* grads, float* loss, float* rgb_out, void* ws, size_t ws_bytes,
                        cudaStream_t st, const char* name, float* stats = nullptr) {
  if (int e = check_problem(cap, H, W, K, true)) return e;
  const bool stats_mode = stats != nullptr;
  if (!map || (!grads && !stats_mode) || !ws || (!prep && cap > 0) ||
      (!params && cap > 0 && !stats_mode))
    return einval("%s: null pointer", name);
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return einval("%s: workspace must be 256-byte aligned", name);
  if (!aligned16(map) || !aligned16(prep)) return einval("%s: pointers must be 16-byte aligned", name);
  // Minimum: room for one record; any larger workspace holds as many
  // records as fit (the default size holds H*W*K/4).
  const WsLayout L1 = ws_layout(H, W, K, cap, 1);
  if (ws_bytes < L1.total) {
    set_error("%s: workspace has %zu bytes, needs at least %zu", name, ws_bytes, L1.total);
    return SAD_EWORKSPACE;
  }
  WsLayout LL = L1;
  {
    const uint64_t per = sizeof(Record) + sizeof(uint64_t);
    uint64_t mr = 1 + (ws_bytes - L1.total) / per;
    if (mr > 0xfffffff0ull) mr = 0xfffffff0ull;
    for (int it = 0; it < 64 && mr > 1; ++it, --mr) {
      const WsLayout T = ws_layout(H, W, K, cap, static_cast<int64_t>(mr));
      if (T.total <= ws_bytes) {
        LL = T;
        break;
      }
    }
  }
  char* base = static_cast<char*>(ws);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + LL.hdr);
  float* tile_loss = reinterpret_cast<float*>(base + LL.tile_loss);
  Record* rec = reinterpret_cast<Record*>(base + LL.records);
  unsigned long long* accq = reinterpret_cast<unsigned long long*>(base + LL.acc);

  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
  if (e == cudaSuccess && cap > 0)
    e = cudaMemsetAsync(accq, 0, sizeof(unsigned long long) * 10 * static_cast<size_t>(cap), st);
  if (e != cudaSuccess) {
    set_error("%s memset: %s", name, cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  const float4 *geo = p4, *met = p4 + cap, *col = p4 + 2 * static_cast<size_t>(cap);
  const uint4* m4 = reinterpret_cast<const uint4*>(map);
  const float two_over_P = 2.0f / static_cast<float>(static_cast<double>(H) * W);
  float* tl = (target && loss) ? tile_loss : nullptr;
#define SAD_TILE_LAUNCH(KK, MM)                                                           \
  k_bwd_tile<KK, MM><<<LL.n_tiles, kTileThreads, 0, st>>>(geo, met, col, cap, H, W, m4, grad_rgb, \
                                                          target, two_over_P, rgb_out, tl, rec,  \
                                                          LL.max_records, hdr)
  if (stats_mode) {
    switch (K) {
      case 4: SAD_TILE_LAUNCH(4, kModeStats); break;
      case 8: SAD_TILE_LAUNCH(8, kModeStats); break;
      default: SAD_TILE_LAUNCH(16, kModeStats); break;
    }
  } else {
    switch (K) {
      case 4: SAD_TILE_LAUNCH(4, kModeGrad); break;
      case 8: SAD_TILE_LAUNCH(8, kModeGrad); break;
      default: SAD_TILE_LAUNCH(16, kModeGrad); break;
    }
  }
#undef SAD_TILE_LAUNCH
  if (int r = check_launch("k_bwd_tile")) return r;
  if (target && loss) {
    k_loss_final<<<1, 256, 0, st>>>(tile_loss, LL.n_tiles, 1.0f / static_cast<float>(static_cast<double>(H) * W), loss);
    if (int r = check_launch("k_loss_final")) return r;
  }
  if (cap == 0) return SAD_OK;
  const int sgrid = 152 * 8;
  if (stats_mode) {
    k_seg_accum<8><<<sgrid, 256, 0, st>>>(rec, hdr, LL.max_records, cap, accq);
    if (int r = check_launch("k_seg_accum")) return r;
    k_site_stats<<<(cap + 255) / 256, 256, 0, st>>>(cap, hdr, LL.max_records, accq, stats);
    return check_launch("k_site_stats");
  }
  k_seg_accum<10><<<sgrid, 256, 0, st>>>(rec, hdr, LL.max_records, cap, accq);
  if (int r = check_launch("k_seg_accum")) return r;
  k_site_grads<<<(cap + 255) / 256, 256, 0, st>>>(params, geo, met, cap, hdr, LL.max_records, accq, grads);
  return check_launch("k_site_grads");
}

}  // namespace sad

using namespace sad;

extern "C" {

size_t sad_backward_workspace_bytes(int32_t H, int32_t W, int32_t K, int32_t capacity,
                                    int64_t max_records) {
  if (H <= 0 || W <= 0 || capacity < 0 || (K != 4 && K != 8 && K != 16)) return 0;
  return ws_layout(H, W, K, capacity, max_records).total;
}

int sad_render_backward(const float* params, const float* prep, int32_t capacity, int32_t H,
                        int32_t W, int32_t K, const uint32_t* map, const float* grad_rgb,
                        float* grads, void* workspace, size_t workspace_bytes, void* stream) {
  if (!grad_rgb) return einval("sad_render_backward: null grad_rgb");
  return run_backward(params, prep, capacity, H, W, K, map, grad_rgb, nullptr, grads, nullptr,
                      nullptr, workspace, workspace_bytes, as_stream(stream), "sad_render_backward");
}

int sad_train_grads(const float* params, const float* prep, int32_t capacity, int32_t H,
                    int32_t W, int32_t K, const uint32_t* map, const float* target,
                    float* grads, float* loss, float* rgb_out, void* workspace,
                    size_t workspace_bytes, void* stream) {
  if (!target || !loss) return einval("sad_train_grads: null target or loss");
  return run_backward(params, prep, capacity, H, W, K, map, nullptr, target, grads, loss, rgb_out,
                      workspace, workspace_bytes, as_stream(stream), "sad_train_grads");
}

int sad_site_stats(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                   const uint32_t* map, const float* target, float* stats, void* workspace,
                   size_t workspace_bytes, void* stream) {
  if (!target || !stats) return einval("sad_site_stats: null target or stats");
  return run_backward(nullptr, prep, capacity, H, W, K, map, nullptr, target, nullptr, nullptr,
                      nullptr, workspace, workspace_bytes, as_stream(stream), "sad_site_stats",
                      stats);
}

int sad_workspace_status(const void* workspace, int64_t* records_used, void* stream) {
  if (!workspace) return einval("sad_workspace_status: null workspace");
  WsHeader h;
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error("sad_workspace_status: %s", cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  if (records_used) *records_used = h.cursor;
  if (h.overflow) {
    set_error("partial records overflowed the workspace (%u produced)", h.cursor);
    return SAD_EWORKSPACE;
  }
  return SAD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Backward without a caller-provided workspace.
//
// Some callers cannot allocate device memory for the workspace: a host
// program that only receives device pointers from another component, code
// running where cudaMalloc is forbidden or would synchronise at the wrong
// moment, or an embedding whose allocator is owned by someone else.  For them
// the library keeps one fixed scratch buffer of kStaticScratchBytes in global
// memory, declared here at file scope.  Every GPU that loads this library
// holds that buffer until the process exits.
//
// The buffer's name is only a host-side stand-in in host code, so its device
// address is looked up with cudaGetSymbolAddress, once per device, with that
// device current; the first call on each device does this lookup (make that
// first call before any stream capture).  All calls share the one buffer and
// it keeps the previous call's contents: every call clears the parts that
// must start at zero, and calls whose executions overlap on the GPU (two
// streams, or two threads) race on it and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace sad {

constexpr size_t kStaticScratchBytes = 64ull << 20;       // 64 MiB
constexpr int64_t kStaticMaxPixels = 4194304;             // e.g. 2048 x 2048
constexpr int32_t kStaticMaxCapacity = 262144;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_ptr[kMaxDevices] = {nullptr};

static int static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("sad_render_backward_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sad_render_backward_noalloc: device %d beyond the supported %d", dev, kMaxDevices);
    return SAD_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      set_error("sad_render_backward_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return SAD_ECUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return SAD_OK;
}

__global__ void k_static_status(const WsHeader* __restrict__ hdr, int32_t* __restrict__ status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *status = hdr->overflow ? SAD_EWORKSPACE : SAD_OK;
}

}  // namespace sad

extern "C" int sad_render_backward_noalloc(const float* params, const float* prep, int32_t capacity,
                                           int32_t H, int32_t W, int32_t K, const uint32_t* map,
                                           const float* grad_rgb, float* grads,
                                           int32_t* status_out, void* stream) {
  if (!grad_rgb) return einval("sad_render_backward_noalloc: null grad_rgb");
  if (int e = check_problem(capacity, H, W, K, true)) return e;
  if (static_cast<int64_t>(H) * W > kStaticMaxPixels)
    return einval("sad_render_backward_noalloc: %d x %d pixels exceed the static limit of %lld",
                  H, W, static_cast<long long>(kStaticMaxPixels));
  if (capacity > kStaticMaxCapacity)
    return einval("sad_render_backward_noalloc: capacity %d exceeds the static limit of %d",
                  capacity, kStaticMaxCapacity);
  void* scratch = nullptr;
  if (int e = static_scratch(&scratch)) return e;
  const int st = run_backward(params, prep, capacity, H, W, K, map, grad_rgb, nullptr, grads,
                              nullptr, nullptr, scratch, kStaticScratchBytes, as_stream(stream),
                              "sad_render_backward_noalloc");
  if (st != SAD_OK || !status_out) return st;
  k_static_status<<<1, 32, 0, as_stream(stream)>>>(reinterpret_cast<const WsHeader*>(scratch),
                                                   status_out);
  return check_launch("k_static_status");
}
