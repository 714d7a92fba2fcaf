// Per-site sums of the per-tile partial records (the reduction of
// App. "Gradient Computation and Reduction", written without any atomic on
// the gradient values): a segmented reduce.
//
//  1. the tile kernels count each site's records (one integer increment per
//     record, in the site's compacted index j, whose old value is the
//     record's place among the site's records) and keep, per image and
//     statistic, the largest |record value| (an atomic max: order
//     independent);
//  2. an exclusive scan of the counts gives each site its segment
//     [start[j], start[j] + count[j]) of the record directory (a local scan
//     per block of 1024 sites; the last block to finish scans the block
//     totals) and clears the counts for the next call;
//  3. k_rec_scatter files every record index at its place in its site's
//     segment (no atomics: the place was taken in step 1);
//  4. each warp sums the segments of its 32 consecutive sites exactly: the
//     warp's records (one contiguous range of the directory) are cut into 32
//     equal chunks, one per lane, so a site with many records is spread over
//     several lanes and no lane walks a long segment alone; every statistic
//     of every record is scaled by 2^S, S = 62 - e - L, with max |value| <
//     2^e over the image's records of that statistic and 2^L above the
//     image's tile count (a site has at most one record per tile), rounded
//     to an int64 and added in integer arithmetic, which is associative; the
//     partial sums of a site split over lanes meet in a segmented scan over
//     the lanes.  The sum is the same bit pattern whatever order the scatter
//     left the segment in and however the chunks fall, its rounding is below
//     2^(L - 62) of the image's largest record value (2^-47 for 16384 tiles),
//     and it depends only on the site's records and the image's scale (so an
//     image's result does not depend on the rest of a batch).
#pragma once

#include "sad_host.h"
#include "sad_tile.cuh"

namespace sad {

// exact 2^a for -126 <= a <= 127, as a float
__device__ __forceinline__ float pow2f(int a) { return __int_as_float((127 + a) << 23); }

// The scale exponent of a statistic: S = 62 - e - L with |values| < 2^e
// (e from the bits of the largest |value|; 0 if all are zero).
__device__ __forceinline__ int fixed_scale_bits(uint32_t max_bits, int L) {
  if (max_bits == 0u) return 0;
  const int E = static_cast<int>(max_bits >> 23);
  return 62 - ((E > 0 ? E : 1) - 126) - L;
}

// v * 2^sh rounded to the nearest integer (halves away from zero), in integer
// arithmetic only (the 64-bit float <-> integer conversions run on the
// narrow double-precision pipe): v = mant 2^(be - 150) for a normal float
// (biased exponent be), mant 2^-149 for a subnormal one.  |v| 2^sh < 2^62 by
// the choice of sh, so the left shift is at most 38.
__device__ __forceinline__ long long fixed_of(float v, int sh) {
  const uint32_t u = __float_as_uint(v);
  const int be = static_cast<int>((u >> 23) & 0xffu);
  const uint32_t mant = (u & 0x7fffffu) | (be != 0 ? 0x800000u : 0u);
  const int ee = (be != 0 ? be : 1) - 150 + sh;  // |v| 2^sh = mant 2^ee
  uint64_t mag = 0;
  if (ee >= 0) {
    mag = static_cast<uint64_t>(mant) << ee;
  } else if (ee > -25) {
    const int r = -ee;  // 1..24: mant + 2^(r-1) < 2^25
    mag = (mant + (1u << (r - 1))) >> r;
  }
  return (u >> 31) != 0u ? -static_cast<long long>(mag) : static_cast<long long>(mag);
}

// q 2^-sh as the nearest float (ties to even; the power of two is applied
// afterwards in two exact factors, so only a result below the normal range
// rounds twice), again in integer arithmetic.
__device__ __forceinline__ float float_of(long long q, int sh) {
  if (q == 0) return 0.f;
  const uint64_t a = q < 0 ? 0ull - static_cast<uint64_t>(q) : static_cast<uint64_t>(q);
  const int lz = __clzll(static_cast<long long>(a));
  const uint64_t n = a << lz;                     // bit 63 set
  uint32_t m = static_cast<uint32_t>(n >> 40);    // the 24 leading bits
  const uint64_t rest = n << 24, half = 1ull << 63;  // the dropped bits
  if (rest > half || (rest == half && (m & 1u) != 0u)) ++m;
  uint32_t E = static_cast<uint32_t>(190 - lz);  // |q| = 1.f 2^(63 - lz)
  if (m == (1u << 24)) {
    m = 1u << 23;
    ++E;
  }
  const float f = __uint_as_float((E << 23) | (m & 0x7fffffu));
  const int a2 = sh >> 1, b2 = sh - (sh >> 1);
  const float r = f * pow2f(-a2) * pow2f(-b2);
  return q < 0 ? -r : r;
}

// Segment starts of the reduce: blocks of 4096 compacted sites (1024
// threads, four consecutive sites each) get a local exclusive scan of their
// counts (start_local) and their total (bsums); the last block to finish
// turns bsums into each block's offset and the grand total (bsums[nb]).
// Consumers add the block's offset to the local start.
constexpr int kSegThreads = 1024;
constexpr int kSegBlock = 4 * kSegThreads;

__host__ __device__ inline uint32_t seg_blocks(size_t n) { return static_cast<uint32_t>((n + kSegBlock - 1) / kSegBlock); }

__device__ __forceinline__ uint32_t block_excl_scan1024(uint32_t v, uint32_t* s_w, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_w[lane] = w;
  }
  __syncthreads();
  const uint32_t pre = warp ? s_w[warp - 1] : 0u;
  total = s_w[31];
  __syncthreads();
  return pre + x - v;
}

static __global__ void __launch_bounds__(kSegThreads) k_seg_scan(uint32_t* __restrict__ cnt, uint32_t n,
                                                                 uint32_t* __restrict__ start_local,
                                                                 uint32_t* __restrict__ bsums,
                                                                 WsHeader* __restrict__ hdr) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_last;
  const uint32_t nb = gridDim.x;
  const uint32_t i0 = blockIdx.x * kSegBlock + 4u * threadIdx.x;
  uint32_t c[4];
  const bool whole = i0 + 3u < n;  // cnt and start_local are 16-byte aligned, i0 a multiple of 4
  if (whole) {
    const uint4 v = *reinterpret_cast<const uint4*>(cnt + i0);
    c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
    *reinterpret_cast<uint4*>(cnt + i0) = make_uint4(0u, 0u, 0u, 0u);  // consumed: zero for the next call
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c[u] = i0 + u < n ? cnt[i0 + u] : 0u;
      if (i0 + u < n) cnt[i0 + u] = 0u;
    }
  }
  uint32_t total;
  const uint32_t ex = block_excl_scan1024(c[0] + c[1] + c[2] + c[3], s_w, total);
  const uint32_t e1 = ex + c[0], e2 = e1 + c[1], e3 = e2 + c[2];
  if (whole) {
    *reinterpret_cast<uint4*>(start_local + i0) = make_uint4(ex, e1, e2, e3);
  } else {
    const uint32_t e[4] = {ex, e1, e2, e3};
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u < n) start_local[i0 + u] = e[u];
  }
  if (threadIdx.x == 0) {
    bsums[blockIdx.x] = total;
    __threadfence();
    s_last = atomicAdd(&hdr->done, 1u) == nb - 1;  // a block count, not a value
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last block: exclusive scan of the block totals, chunk by chunk
  uint32_t carry = 0;
  for (uint32_t c0 = 0; c0 < nb; c0 += kSegThreads) {
    const uint32_t k = c0 + threadIdx.x;
    const uint32_t v = k < nb ? *reinterpret_cast<volatile uint32_t*>(&bsums[k]) : 0u;
    uint32_t tot;
    const uint32_t x = block_excl_scan1024(v, s_w, tot);
    if (k < nb) bsums[k] = carry + x;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    bsums[nb] = carry;
    hdr->done = 0u;  // ready for the next call
  }
}

// The segment starts of n compacted sites (start_local: n entries, bsums:
// seg_blocks(n) + 1 entries, the last one the number of records); the counts
// are left zero.  hdr->done must be zero (the header is cleared by every
// call).
static inline void run_seg_scan(uint32_t* cnt, uint32_t n, uint32_t* start_local, uint32_t* bsums,
                                WsHeader* hdr, cudaStream_t st) {
  const uint32_t nb = seg_blocks(n);
  if (nb == 0) return;
  TraceScope tr_(st, "k_seg_scan");
  k_seg_scan<<<nb, kSegThreads, 0, st>>>(cnt, n, start_local, bsums, hdr);
}

// bits for the record count of one site of an image of n_tiles tiles:
// 2^L > n_tiles (at most one record per tile)
static inline int count_bits(uint32_t n_tiles) {
  int L = 0;
  while (L < 32 && (1ull << L) <= n_tiles) ++L;
  return L;
}

__device__ __forceinline__ uint32_t seg_start(const uint32_t* __restrict__ start_local,
                                              const uint32_t* __restrict__ boff, uint32_t j) {
  return start_local[j] + boff[j / kSegBlock];
}

// Files record r at its place in its site's segment of the directory (place:
// the records' {place, site} pairs, contiguous).  Each thread takes four
// records a pass (all loads issued before the stores).
static __global__ void k_rec_scatter(const uint2* __restrict__ place, const WsHeader* __restrict__ hdr,
                                     uint32_t max_records, const uint32_t* __restrict__ start_local,
                                     const uint32_t* __restrict__ boff, uint32_t* __restrict__ dir) {
  const uint64_t n = min(hdr->cursor, max_records);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t r0 = blockIdx.x * blockDim.x + threadIdx.x; r0 < n; r0 += 4u * stride) {
    uint2 rc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint64_t r = r0 + u * stride;
      rc[u] = r < n ? ldg(place + r) : make_uint2(0u, 0u);  // {rank, cj}
    }
    uint32_t at[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) at[u] = r0 + u * stride < n ? seg_start(start_local, boff, rc[u].y) + rc[u].x : 0u;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (r0 + u * stride < n) dir[at[u]] = static_cast<uint32_t>(r0 + u * stride);
  }
}

// The warp's scratch of warp_site_sums.
template <int NV>
struct WarpSums {
  long long head[32][NV];     // per lane: its chunk's partial sum of its first site
  long long res[32][NV + 1];  // per local site: the finished integer sums
  int sh[32][NV];             // per local site: the scale exponents of its image
};
constexpr int kSumThreads = 128;  // block size of the kernels that call warp_site_sums

// The NV exact statistic sums of each lane's site (compacted index j, valid
// if `have`; the lanes' sites are the 32 consecutive indices from j - lane;
// boff[seg_blocks(n_sites)] records in all), at the scale of the site's image
// (pmax: that image's largest |record value| bits per statistic; L: count
// bits).  Every lane of the warp must call it (with the same j - lane).
// Each lane loads NB records of its chunk at a time.  Returns the lane's
// site's record count.
template <int NV, int NB = 4>
__device__ __forceinline__ uint32_t warp_site_sums(bool have, uint32_t j, uint32_t n_sites,
                                                   const uint32_t* __restrict__ start_local,
                                                   const uint32_t* __restrict__ boff,
                                                   const uint32_t* __restrict__ dir,
                                                   const Record* __restrict__ rec,
                                                   const uint32_t* __restrict__ pmax, int L,
                                                   WarpSums<NV>& ws, float (&out)[NV]) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const uint32_t j0 = j - static_cast<uint32_t>(lane);
  uint32_t b = 0u, e = 0u;
  if (have) {
    b = seg_start(start_local, boff, j);
    e = j + 1 < n_sites ? seg_start(start_local, boff, j + 1) : boff[seg_blocks(n_sites)];
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) ws.sh[lane][k] = have ? fixed_scale_bits(pmax[k], L) : 0;
  // the warp's records: one contiguous range (the segments follow the
  // sites); the valid lanes come first, so lane 0 holds its start
  const uint32_t lo = __shfl_sync(kFull, b, 0);
  const uint32_t hi = __reduce_max_sync(kFull, e);
  const uint32_t n = hi > lo ? hi - lo : 0u;
  const uint32_t per = (n + 31u) / 32u;
  const uint32_t qa = min(lo + per * static_cast<uint32_t>(lane), hi), qb = min(qa + per, hi);
  __syncwarp();
  // walk the chunk: runs of equal sites; a run that ends inside the chunk
  // and did not start it is a whole site (finished here), the first run may
  // continue a site of the lanes before, the last one may go on in the
  // lanes after
  uint32_t first = 32u + lane, cur = 32u + lane;  // an empty chunk's key: no site
  long long run[NV];
  int shc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    run[k] = 0;
    shc[k] = 0;
  }
  bool split = false;  // the chunk holds more than one site
  for (uint32_t q0 = qa; q0 < qb; q0 += NB) {
    uint32_t r[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) r[u] = q0 + u < qb ? ldg(&dir[q0 + u]) : 0u;
    float4 w[NB][3];
#pragma unroll
    for (int u = 0; u < NB; ++u)
      if (q0 + u < qb) {
        const float4* p = reinterpret_cast<const float4*>(rec + r[u]);
        w[u][0] = ldg(&p[0]);
        if (NV > 2) w[u][1] = ldg(&p[1]);
        if (NV > 6) w[u][2] = ldg(&p[2]);
      }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      if (q0 + u >= qb) break;
      const float a[12] = {w[u][0].x, w[u][0].y, w[u][0].z, w[u][0].w, w[u][1].x, w[u][1].y,
                           w[u][1].z, w[u][1].w, w[u][2].x, w[u][2].y, w[u][2].z, w[u][2].w};
      const uint32_t s = (__float_as_uint(a[1]) - j0) & 31u;
      if (s != cur) {
        if (cur < 32u) {
          if (!split) {
            first = cur;
#pragma unroll
            for (int k = 0; k < NV; ++k) ws.head[lane][k] = run[k];
            split = true;
          } else {
#pragma unroll
            for (int k = 0; k < NV; ++k) ws.res[cur][k] = run[k];
          }
        }
        cur = s;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          shc[k] = ws.sh[s][k];
          run[k] = 0;
        }
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) run[k] += fixed_of(a[2 + k], shc[k]);
    }
  }
  if (!split) first = cur;
  // segmented inclusive scan over the lanes of the last runs, keyed by site
  // (equal keys are adjacent lanes)
  const uint32_t key = cur;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t ko = __shfl_up_sync(kFull, key, o);
    const bool take = lane >= o && ko == key;
    // no run reaches o lanes back: no later offset adds anything either
    // (equal keys are adjacent), so the scan is complete
    if (!__any_sync(kFull, take)) break;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const long long t = __shfl_up_sync(kFull, run[k], o);
      if (take) run[k] += t;
    }
  }
  const uint32_t kprev = __shfl_up_sync(kFull, key, 1);
  const uint32_t knext = __shfl_down_sync(kFull, key, 1), fnext = __shfl_down_sync(kFull, first, 1);
  const bool join = split && lane > 0 && kprev == first;  // the first run continues the lanes before
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const long long t = __shfl_up_sync(kFull, run[k], 1);
    if (split) ws.res[first][k] = ws.head[lane][k] + (join ? t : 0ll);
  }
  // the last run's site ends here unless the next lane goes on with it
  if (key < 32u && (lane == 31 || (knext != key && fnext != key))) {
#pragma unroll
    for (int k = 0; k < NV; ++k) ws.res[key][k] = run[k];
  }
  __syncwarp();
  // each lane turns its own site's sums back into floats (no divergence)
  const uint32_t mine = e > b ? e - b : 0u;
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = mine ? float_of(ws.res[lane][k], ws.sh[lane][k]) : 0.f;
  __syncwarp();  // the scratch may be reused by the warp
  return mine;
}

}  // namespace sad
