// Per-site sums of the per-tile partial records (the reduction of
// App. "Gradient Computation and Reduction", written without any atomic on
// the gradient values): a segmented reduce.
//
//  1. the tile kernels count each site's records (one integer increment per
//     record, in the site's compacted index j);
//  2. an exclusive scan of the counts gives each site its segment
//     [start[j], start[j] + count[j]) of the record directory (a local scan
//     per block of 1024 sites plus each block's offset);
//  3. k_rec_scatter files every record index into its site's segment (the
//     counts are decremented back to zero, so the next call finds them
//     cleared);
//  4. each site sums its segment exactly (its own thread, or its warp for a
//     site with many records): every statistic of
//     every record is scaled by 2^S, S = 62 - e - ceil(log2(n + 1)) with
//     max |value| < 2^e over the site's n records, rounded to an int64 and
//     added in integer arithmetic, which is associative (the conversion
//     itself is integer work on the float's bits: no double precision).
//     The sum is the same bit pattern whatever order the scatter left the
//     segment in, its
//     rounding is below 2^(ceil(log2(n+1)) - 62) of the site's largest record
//     value, and it depends on the site's own records only (so an image's
//     result does not depend on the rest of a batch).
#pragma once

#include "sad_host.h"
#include "sad_tile.cuh"

namespace sad {

// v * 2^sh rounded to the nearest integer (halves away from zero), in
// integer arithmetic: v = m 2^(e - 150) with the 24-bit significand m.
// Requires |v| 2^sh < 2^62.
__device__ __forceinline__ long long fixed_of(float v, int sh) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint64_t m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
  const int s = static_cast<int>(e ? e : 1u) - 150 + sh;
  uint64_t q;
  if (s >= 0) q = m << s;
  else if (s > -64) q = (m + (1ull << (-s - 1))) >> (-s);
  else q = 0ull;
  return (b >> 31) ? -static_cast<long long>(q) : static_cast<long long>(q);
}

// Segment starts of the reduce: blocks of 1024 compacted sites get a local
// exclusive scan of their counts (start_local) and their total (bsums);
// k_seg_scan_blocks turns bsums into each block's offset and the grand total
// (bsums[nb]).  Consumers add the block's offset to the local start.
constexpr int kSegBlock = 1024;

static __global__ void __launch_bounds__(kSegBlock) k_seg_scan_local(const uint32_t* __restrict__ cnt,
                                                                     uint32_t n, uint32_t* __restrict__ start_local,
                                                                     uint32_t* __restrict__ bsums) {
  __shared__ uint32_t s_w[32];
  const uint32_t i = blockIdx.x * kSegBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t v = i < n ? cnt[i] : 0u;
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
  if (i < n) start_local[i] = pre + x - v;
  if (threadIdx.x == kSegBlock - 1) bsums[blockIdx.x] = pre + x;
}

// exclusive scan of the nb block totals in place, one block of 1024 threads
// (chunks of 1024 with a running carry); bsums[nb] receives the total
static __global__ void __launch_bounds__(kSegBlock) k_seg_scan_blocks(uint32_t* __restrict__ bsums, uint32_t nb) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0u;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < nb; c0 += kSegBlock) {
    const uint32_t i = c0 + threadIdx.x;
    const uint32_t v = i < nb ? bsums[i] : 0u;
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
    const uint32_t carry = s_carry;
    const uint32_t pre = warp ? s_w[warp - 1] : 0u;
    if (i < nb) bsums[i] = carry + pre + x - v;
    __syncthreads();
    if (threadIdx.x == kSegBlock - 1) s_carry = carry + pre + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsums[nb] = s_carry;
}

__host__ __device__ inline uint32_t seg_blocks(size_t n) { return static_cast<uint32_t>((n + kSegBlock - 1) / kSegBlock); }

// The segment starts of n compacted sites (start_local: n entries, bsums:
// seg_blocks(n) + 1 entries, the last one the number of records).
static inline void run_seg_scan(const uint32_t* cnt, uint32_t n, uint32_t* start_local, uint32_t* bsums,
                                cudaStream_t st) {
  const uint32_t nb = seg_blocks(n);
  if (nb == 0) return;
  { TraceScope tr_(st, "k_seg_scan_local"); k_seg_scan_local<<<nb, kSegBlock, 0, st>>>(cnt, n, start_local, bsums); }
  { TraceScope tr_(st, "k_seg_scan_blocks"); k_seg_scan_blocks<<<1, kSegBlock, 0, st>>>(bsums, nb); }
}

__device__ __forceinline__ uint32_t seg_start(const uint32_t* __restrict__ start_local,
                                              const uint32_t* __restrict__ boff, uint32_t j) {
  return start_local[j] + boff[j / kSegBlock];
}

// Files record r into its site's segment of the directory; counts go back to
// zero.
static __global__ void k_rec_scatter(const Record* __restrict__ rec, const WsHeader* __restrict__ hdr,
                                     uint32_t max_records, const uint32_t* __restrict__ start_local,
                                     const uint32_t* __restrict__ boff, uint32_t* __restrict__ cnt,
                                     uint32_t* __restrict__ dir) {
  const uint32_t n = min(hdr->cursor, max_records);
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const uint32_t j = rec[r].cj;
    dir[seg_start(start_local, boff, j) + atomicSub(&cnt[j], 1u) - 1u] = r;
  }
}

// A record is three aligned 16-byte words {site, cj, acc0, acc1},
// {acc2..acc5}, {acc6..acc9}: read whole.
__device__ __forceinline__ void load_record(const Record* __restrict__ rec, uint32_t r, float (&a)[10]) {
  const float4* w = reinterpret_cast<const float4*>(rec + r);
  const float4 w0 = ldg(&w[0]), w1 = ldg(&w[1]), w2 = ldg(&w[2]);
  a[0] = w0.z; a[1] = w0.w; a[2] = w1.x; a[3] = w1.y; a[4] = w1.z;
  a[5] = w1.w; a[6] = w2.x; a[7] = w2.y; a[8] = w2.z; a[9] = w2.w;
}

// the scale of a statistic: 2^sh with n * max 2^sh < 2^62
__device__ __forceinline__ int fixed_scale(float mx, uint32_t n) {
  int ex = 0;
  frexpf(mx, &ex);  // mx < 2^ex
  return mx > 0.f ? 62 - ex - (32 - __clz(n)) : 0;
}

constexpr uint32_t kHeavySite = 16;  // records above which a site is summed by its warp
constexpr int kBatch = 4;            // records whose loads a thread issues together

// The NV exact statistic sums of each lane's site (compacted index j, valid
// if `have`; the counts of the n_sites sites are segments of the directory,
// boff[seg_blocks(n_sites)] records in all).  Every lane of the warp must call
// it.  A site with at most kHeavySite records is summed by its own lane; a
// heavier site by the whole warp (lanes take its records in turn, then exact
// warp-wide max and integer sums), so one heavy site does not hold its warp
// for a serial walk.  Returns the lane's site's record count.
template <int NV>
__device__ __forceinline__ uint32_t site_exact_sums(bool have, uint32_t j, uint32_t n_sites,
                                                    const uint32_t* __restrict__ start_local,
                                                    const uint32_t* __restrict__ boff,
                                                    const uint32_t* __restrict__ dir,
                                                    const Record* __restrict__ rec, float (&out)[NV]) {
  const int lane = threadIdx.x & 31;
  uint32_t b = 0u, e = 0u;
  if (have) {
    b = seg_start(start_local, boff, j);
    e = j + 1 < n_sites ? seg_start(start_local, boff, j + 1) : boff[seg_blocks(n_sites)];
  }
  const uint32_t n = e > b ? e - b : 0u;
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = 0.f;
  const bool heavy = n > kHeavySite;
  if (n > 0u && !heavy) {
    float mx[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) mx[k] = 0.f;
    for (uint32_t q0 = b; q0 < e; q0 += kBatch) {
      float a[kBatch][10];
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (q0 + u < e) load_record(rec, dir[q0 + u], a[u]);
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (q0 + u < e)
#pragma unroll
          for (int k = 0; k < NV; ++k) mx[k] = fmaxf(mx[k], fabsf(a[u][k]));
    }
    int sh[NV];
    long long sum[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      sh[k] = fixed_scale(mx[k], n);
      sum[k] = 0;
    }
    for (uint32_t q0 = b; q0 < e; q0 += kBatch) {
      float a[kBatch][10];
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (q0 + u < e) load_record(rec, dir[q0 + u], a[u]);
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (q0 + u < e)
#pragma unroll
          for (int k = 0; k < NV; ++k) sum[k] += fixed_of(a[u][k], sh[k]);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = ldexpf(static_cast<float>(sum[k]), -sh[k]);
  }
  unsigned hm = __ballot_sync(0xffffffffu, heavy);
  while (hm) {
    const int src = __ffs(hm) - 1;
    hm &= hm - 1;
    const uint32_t hb = __shfl_sync(0xffffffffu, b, src), he = __shfl_sync(0xffffffffu, e, src);
    float mx[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) mx[k] = 0.f;
    for (uint32_t q = hb + lane; q < he; q += 32) {
      float a[10];
      load_record(rec, dir[q], a);
#pragma unroll
      for (int k = 0; k < NV; ++k) mx[k] = fmaxf(mx[k], fabsf(a[k]));
    }
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
    int sh[NV];
    long long sum[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      sh[k] = fixed_scale(mx[k], he - hb);
      sum[k] = 0;
    }
    for (uint32_t q = hb + lane; q < he; q += 32) {
      float a[10];
      load_record(rec, dir[q], a);
#pragma unroll
      for (int k = 0; k < NV; ++k) sum[k] += fixed_of(a[k], sh[k]);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum[k] += __shfl_xor_sync(0xffffffffu, sum[k], o);
    if (lane == src)
#pragma unroll
      for (int k = 0; k < NV; ++k) out[k] = ldexpf(static_cast<float>(sum[k]), -sh[k]);
  }
  return n;
}

}  // namespace sad
