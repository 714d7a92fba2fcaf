// Deterministic selection of the `need` smallest 32-bit keys (ties to the
// smaller index) and exclusive scans, shared by the initialisation and the
// densify/prune passes.  Internal linkage: every translation unit that
// includes this header gets its own copies of the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sad {

// Device-resident selection state.  `need` must be set (device side) before
// run_select_smallest; the rest must be zero.
struct SelState {
  uint32_t prefix;     // key bits fixed so far
  uint32_t need;       // keys still to take at or below the prefix
  uint32_t hist[256];  // digit histogram of the current pass
  uint32_t pad[62];
};

// radix pass: histogram of the digit at `shift` among keys whose bits above
// shift+8 equal the prefix
static __global__ void k_sel_hist(const uint32_t* __restrict__ keys, size_t n, int shift,
                                  SelState* __restrict__ st) {
  __shared__ uint32_t s_h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_h[i] = 0;
  __syncthreads();
  const uint32_t prefix = st->prefix;
  const int hi = shift + 8;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const uint32_t k = keys[i];
    if (hi >= 32 || (k >> hi) == prefix) atomicAdd(&s_h[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (s_h[i]) atomicAdd(&st->hist[i], s_h[i]);
}

static __global__ void k_sel_pick(SelState* __restrict__ st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint32_t need = st->need;
  uint32_t run = 0;
  int d = 255;
  for (int i = 0; i < 256; ++i) {
    if (run + st->hist[i] >= need) {
      d = i;
      break;
    }
    run += st->hist[i];
  }
  st->prefix = (st->prefix << 8) | static_cast<uint32_t>(d);
  st->need = need - run;
  for (int i = 0; i < 256; ++i) st->hist[i] = 0;
}

static __global__ void k_sel_flag_eq(const uint32_t* __restrict__ keys, size_t n,
                                     const SelState* __restrict__ st, uint32_t* __restrict__ flag) {
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = keys[i] == st->prefix ? 1u : 0u;
}

static __global__ void k_sel_flag_take(const uint32_t* __restrict__ keys, size_t n,
                                       const SelState* __restrict__ st,
                                       const uint32_t* __restrict__ eqrank,
                                       uint32_t* __restrict__ flag) {
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys[i], T = st->prefix;
  flag[i] = (k < T || (k == T && eqrank[i] < st->need)) ? 1u : 0u;
}

// exclusive scan in blocks of 1024, then a serial pass over the block sums
static __global__ void k_xscan_blocks(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                      size_t n, uint32_t* __restrict__ bsums) {
  __shared__ uint32_t s_w[32];
  const size_t i = static_cast<size_t>(blockIdx.x) * 1024 + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t v = i < n ? in[i] : 0u;
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
  if (i < n) out[i] = pre + x - v;
  if (threadIdx.x == 1023) bsums[blockIdx.x] = pre + x;
}

// exclusive scan of the block sums; bsums[nb] receives the grand total
static __global__ void k_xscan_sums(uint32_t* __restrict__ bsums, uint32_t nb) {
  if (threadIdx.x || blockIdx.x) return;
  uint32_t run = 0;
  for (uint32_t b = 0; b < nb; ++b) {
    const uint32_t v = bsums[b];
    bsums[b] = run;
    run += v;
  }
  bsums[nb] = run;
}

static __global__ void k_xscan_add(uint32_t* __restrict__ out, size_t n,
                                   const uint32_t* __restrict__ bsums) {
  const size_t i = static_cast<size_t>(blockIdx.x) * 1024 + threadIdx.x;
  if (i < n) out[i] += bsums[blockIdx.x];
}

static inline uint32_t scan_blocks(size_t n) { return static_cast<uint32_t>((n + 1023) / 1024); }

// out = exclusive scan of in[n]; bsums needs scan_blocks(n) + 1 entries and
// holds the total at bsums[scan_blocks(n)] afterwards.
static inline void run_xscan(const uint32_t* in, uint32_t* out, size_t n, uint32_t* bsums,
                             cudaStream_t st) {
  const uint32_t nb = scan_blocks(n);
  if (nb == 0) return;
  { TraceScope tr_(st, "k_xscan_blocks"); k_xscan_blocks<<<nb, 1024, 0, st>>>(in, out, n, bsums); }
  { TraceScope tr_(st, "k_xscan_sums"); k_xscan_sums<<<1, 32, 0, st>>>(bsums, nb); }
  { TraceScope tr_(st, "k_xscan_add"); k_xscan_add<<<nb, 1024, 0, st>>>(out, n, bsums); }
}

// flag[i] = 1 for the `need` smallest keys (ties to the smaller index),
// need <= n.  scan and bsums are scratch of n and scan_blocks(n)+1 entries.
static inline void run_select_smallest(const uint32_t* keys, size_t n, SelState* sel,
                                       uint32_t* flag, uint32_t* scan, uint32_t* bsums,
                                       cudaStream_t st) {
  const unsigned g256 = static_cast<unsigned>((n + 255) / 256);
  for (int shift = 24; shift >= 0; shift -= 8) {
    { TraceScope tr_(st, "k_sel_hist"); k_sel_hist<<<152 * 4, 256, 0, st>>>(keys, n, shift, sel); }
    { TraceScope tr_(st, "k_sel_pick"); k_sel_pick<<<1, 32, 0, st>>>(sel); }
  }
  { TraceScope tr_(st, "k_sel_flag_eq"); k_sel_flag_eq<<<g256, 256, 0, st>>>(keys, n, sel, flag); }
  run_xscan(flag, scan, n, bsums, st);
  { TraceScope tr_(st, "k_sel_flag_take"); k_sel_flag_take<<<g256, 256, 0, st>>>(keys, n, sel, scan, flag); }
}

}  // namespace sad
