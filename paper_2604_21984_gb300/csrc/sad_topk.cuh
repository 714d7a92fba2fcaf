// One propagation pass of the per-pixel top-K field for a single pixel
// (Sec. 4.3, update C_t = topK(C_{t-1} U P_t U G_t)), shared by the
// stand-alone pass kernel and the fused training-step kernel.
//
// Candidate keys: (logit, id) packed into one 64-bit integer whose unsigned
// order is the list order (logit descending, then id ascending):
//   key = orderable(logit) << 32 | ~id,
// with orderable() the usual sign-flip map of IEEE floats (-0 is first turned
// into +0 so that the two zeros tie, as they do in float comparison).  The
// empty entry is key 0, below every real candidate.
//
// Per pixel (one thread):
//  A. score the pixel's own list (independent gathers) and sort it with a
//     bitonic network; drop duplicate ids (only possible in a damaged input);
//  B. filter the 4 neighbour lists and the J injected ids against the list
//     and queue the novel ids in shared memory (per-thread column);
//  C. each thread scores its own queue and inserts winners.
// Phase C runs per lane, so the insertion network is paid for the queued
// candidates only, not for every candidate of every lane in the warp.
#pragma once

#include "sad_device.cuh"

namespace sad {

constexpr int kQueue = 24;

__device__ __forceinline__ uint64_t make_key(float l, uint32_t id) {
  uint32_t u = __float_as_uint(__fadd_rn(l, 0.0f));
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return (static_cast<uint64_t>(u) << 32) | static_cast<uint64_t>(~id);
}

__device__ __forceinline__ uint32_t key_id(uint64_t k) { return ~static_cast<uint32_t>(k); }

template <int K>
__device__ __forceinline__ void bitonic_sort_desc(uint64_t (&v)[K]) {
#pragma unroll
  for (int k = 2; k <= K; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const bool desc = (i & k) == 0;
          const uint64_t a = v[i], b = v[l];
          const bool sw = desc ? (a < b) : (a > b);
          v[i] = sw ? b : a;
          v[l] = sw ? a : b;
        }
      }
    }
  }
}

template <int K>
__device__ __forceinline__ bool list_has(const uint64_t (&v)[K], uint32_t id) {
  const uint32_t nid = ~id;
  bool hit = false;
#pragma unroll
  for (int k = 0; k < K; ++k) hit |= (static_cast<uint32_t>(v[k]) == nid);
  return hit;
}

// Insert key c (greater than v[K-1], id not present) keeping v sorted.
template <int K>
__device__ __forceinline__ void list_insert(uint64_t (&v)[K], uint64_t c) {
  bool gt[K];
#pragma unroll
  for (int k = 0; k < K; ++k) gt[k] = c > v[k];
#pragma unroll
  for (int k = K - 1; k > 0; --k) v[k] = gt[k - 1] ? v[k - 1] : (gt[k] ? c : v[k]);
  v[0] = gt[0] ? c : v[0];
}

// Site ids of one image: [lo, lo + n).
struct SiteRange {
  uint32_t lo, n;
  __device__ __forceinline__ bool has(uint32_t id) const { return id - lo < n; }
};

// Logit key of candidate id at (px, py), or 0 if the id cannot enter.
__device__ __forceinline__ uint64_t cand_key(uint32_t id, SiteRange sr, float px, float py,
                                             const float4* __restrict__ geo,
                                             const float4* __restrict__ met) {
  if (!sr.has(id)) return 0ull;
  const float4 m = ldg(&met[id]);
  if (m.w == 0.f) return 0ull;
  const float l = score_exact(px, py, ldg(&geo[id]), m);
  if (l != l) return 0ull;
  return make_key(l, id);
}

// The K best keys of pixel (col, row) of an H x W image after one pass.
// map_in: K/4 planes of uint4 with plane stride P; the image's pixels start
// at plane index pix_off.  q_local = row*W + col (injection counter).  Threads
// outside the image pass inimg = false and get an empty list; the queue
// column `tid` of s_q must be private to the thread.
template <int K, int NT>
__device__ __forceinline__ void pixel_update(uint64_t (&v)[K], bool inimg, int col, int row, int H,
                                             int W, SiteRange sr, const float4* __restrict__ geo,
                                             const float4* __restrict__ met,
                                             const uint4* __restrict__ map_in, size_t P,
                                             size_t pix_off, uint32_t code, int J, uint64_t seed,
                                             uint32_t (*s_q)[NT], int tid) {
  constexpr int NP = K / 4;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0ull;
  if (!inimg) return;
  const uint32_t q = static_cast<uint32_t>(row) * static_cast<uint32_t>(W) + col;
  const float px = __fadd_rn(static_cast<float>(col), 0.5f);
  const float py = __fadd_rn(static_cast<float>(row), 0.5f);

  // A. own list
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const uint4 w = ldg(&map_in[j * P + pix_off + q]);
    v[4 * j] = cand_key(w.x, sr, px, py, geo, met);
    v[4 * j + 1] = cand_key(w.y, sr, px, py, geo, met);
    v[4 * j + 2] = cand_key(w.z, sr, px, py, geo, met);
    v[4 * j + 3] = cand_key(w.w, sr, px, py, geo, met);
  }
  bitonic_sort_desc<K>(v);
  bool dup = false;
#pragma unroll
  for (int k = 1; k < K; ++k) dup |= v[k] != 0ull && v[k] == v[k - 1];
  if (dup) {  // damaged input list: zero repeated keys, re-sort
#pragma unroll
    for (int k = K - 1; k > 0; --k)
      if (v[k] != 0ull && v[k] == v[k - 1]) v[k] = 0ull;
    bitonic_sort_desc<K>(v);
  }

  // B + C. queue novel candidates; drain the queue when full and at the end
  int qn = 0;
  auto drain = [&]() {
    for (int i = 0; i < qn; ++i) {
      const uint32_t id = s_q[i][tid];
      if (list_has<K>(v, id)) continue;
      const uint64_t c = cand_key(id, sr, px, py, geo, met);
      if (c > v[K - 1]) list_insert<K>(v, c);
    }
    qn = 0;
  };
  auto offer = [&](uint32_t id) {
    if (!sr.has(id) || list_has<K>(v, id)) return;
    for (int i = 0; i < qn; ++i)
      if (s_q[i][tid] == id) return;
    if (qn == kQueue) drain();
    s_q[qn++][tid] = id;
  };
  const int s = static_cast<int>(code >> 16);
  const int nc[4] = {col - s, col + s, col, col};
  const int nr[4] = {row, row, row - s, row + s};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (nc[d] < 0 || nc[d] >= W || nr[d] < 0 || nr[d] >= H) continue;
    const size_t nq = pix_off + static_cast<size_t>(nr[d]) * W + nc[d];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const uint4 w = ldg(&map_in[j * P + nq]);
      offer(w.x);
      offer(w.y);
      offer(w.z);
      offer(w.w);
    }
  }
  const uint64_t base = (static_cast<uint64_t>(code) << 32);
  for (int j = 0; j < J; ++j) {
    const uint64_t ctr = base | static_cast<uint32_t>(q * static_cast<uint32_t>(J) + j);
    const uint64_t h = splitmix64_at(seed, ctr);
    offer(sr.lo + static_cast<uint32_t>(((h >> 32) * static_cast<uint64_t>(sr.n)) >> 32));
  }
  drain();
}

}  // namespace sad
