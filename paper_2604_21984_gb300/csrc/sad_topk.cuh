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
//  A. score the pixel's own list (independent gathers) and sort it
//     (odd-even transposition passes until one swaps nothing); drop
//     duplicate ids (only possible in a damaged input);
//  B. filter each neighbour list and the J injected ids against the list
//     and queue the novel ids in shared memory (per-thread column);
//  C. the thread scores its queue and inserts the winners, after each
//     neighbour whose ids could overflow the queue, and at the end.
// Phase C runs per lane, so the insertion network is paid for the queued
// candidates only, not for every candidate of every lane in the warp.
#pragma once

#include <cuda_fp16.h>

#include "sad_device.cuh"

namespace sad {

// per-thread queues of novel candidate ids: the stand-alone pass's, and the
// fused step's (longer: with room for two neighbours' offers the step
// drains once, at the end, in most pixels)
constexpr int kQueue = 24;
constexpr int kQueueStep = 32;

__device__ __forceinline__ uint64_t make_key(float l, uint32_t id) {
  uint32_t u = __float_as_uint(__fadd_rn(l, 0.0f));
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return (static_cast<uint64_t>(u) << 32) | static_cast<uint64_t>(~id);
}

__device__ __forceinline__ uint32_t key_id(uint64_t k) { return ~static_cast<uint32_t>(k); }

// The logit a (non-empty) key was made from.
__device__ __forceinline__ float key_logit(uint64_t k) {
  const uint32_t u = static_cast<uint32_t>(k >> 32);
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Sorts keys descending by odd-even transposition: each pass compares the
// even pairs (0,1), (2,3), ... then the odd pairs (1,2), (3,4), ..., and the
// passes stop once one swaps nothing (then every adjacent pair is in order).
// A pixel's own list arrives sorted by its previous logits, so one pass
// (K - 1 compare-exchanges) confirms an unchanged order and a few fix a
// slightly changed one; K passes sort any input.  Keys that compare equal
// are equal values (the empty key, or a repeated id in a damaged list), so
// the result is the same whatever the sorting network.
template <int K>
__device__ __forceinline__ void sort_desc(uint64_t (&v)[K]) {
#pragma unroll 1
  for (int pass = 0; pass < K; ++pass) {
    bool sw = false;
#pragma unroll
    for (int i = 0; i + 1 < K; i += 2) {
      const uint64_t a = v[i], b = v[i + 1];
      const bool s = a < b;
      v[i] = s ? b : a;
      v[i + 1] = s ? a : b;
      sw |= s;
    }
#pragma unroll
    for (int i = 1; i + 1 < K; i += 2) {
      const uint64_t a = v[i], b = v[i + 1];
      const bool s = a < b;
      v[i] = s ? b : a;
      v[i + 1] = s ? a : b;
      sw |= s;
    }
    if (!sw) break;
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

// Where a pass reads a candidate's scoring record g = {x, y, tau s, r},
// m = {G00, G01, G11, active}: the prepared fp32 table (two 16-byte gathers
// per candidate) ...
struct F32Sites {
  const float4* geo;
  const float4* met;
  __device__ __forceinline__ void load(uint32_t id, float4& g, float4& m) const {
    m = ldg(&met[id]);
    g = ldg(&geo[id]);
  }
};

__device__ __forceinline__ float2 half2_bits_to_float2(uint32_t u) {
  __half2_raw r;
  r.x = static_cast<unsigned short>(u & 0xffffu);
  r.y = static_cast<unsigned short>(u >> 16);
  return __half22float2(__half2(r));
}

// ... or the 16-byte half2 candidate table (App. "Data Layout and Packing",
// Packed candidate sites): words {x, y}, {tau s, r}, {G00, G01},
// {G11, active}, each a half2 with the first value in the low half (one
// gather per candidate; halves widen to fp32 exactly).
struct H2Sites {
  const uint4* cand;
  __device__ __forceinline__ void load(uint32_t id, float4& g, float4& m) const {
    const uint4 w = ldg(&cand[id]);
    const float2 a = half2_bits_to_float2(w.x), b = half2_bits_to_float2(w.y);
    const float2 c = half2_bits_to_float2(w.z), d = half2_bits_to_float2(w.w);
    g = make_float4(a.x, a.y, b.x, b.y);
    m = make_float4(c.x, c.y, d.x, d.y);
  }
};

// Logit key of candidate id at (px, py), or 0 if the id cannot enter.
template <class Sites>
__device__ __forceinline__ uint64_t cand_key(uint32_t id, SiteRange sr, float px, float py,
                                             const Sites& sites) {
  if (!sr.has(id)) return 0ull;
  float4 g, m;
  sites.load(id, g, m);
  if (m.w == 0.f) return 0ull;
  const float l = score_exact(px, py, g, m);
  if (l != l) return 0ull;
  return make_key(l, id);
}

// The K best keys of pixel (col, row) of an H x W image after one pass
// (with a candidate grid: of cell (col, row) of an H x W grid).
// map_in: K/4 planes of uint4 with plane stride P; the image's pixels start
// at plane index pix_off.  q_local = row*W + col (injection counter).  Threads
// outside the image pass inimg = false and get an empty list; the queue
// column `tid` of s_q (QL rows) must be private to the thread.
// STORE_ALL: every offer writes its id at the queue's end and only a novel
// id advances the count (no branch per offer; the unused slot is
// overwritten by the next offer).  Faster inside the fused step's tile
// kernel, slower in the stand-alone pass (measured), the same result.
template <int K, int NT, int NG = 4, bool STORE_ALL = false, int QL = kQueue, class Sites>
__device__ __forceinline__ void pixel_update(uint64_t (&v)[K], bool inimg, int col, int row, int H,
                                             int W, SiteRange sr, const Sites& sites,
                                             const uint4* __restrict__ map_in, size_t P,
                                             size_t pix_off, uint32_t code, int J, uint64_t seed,
                                             uint32_t (*s_q)[NT], int tid, float cell = 1.f) {
  constexpr int NP = K / 4;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0ull;
  if (!inimg) return;
  const uint32_t q = static_cast<uint32_t>(row) * static_cast<uint32_t>(W) + col;
  // the evaluation point: the pixel centre, or the cell centre of a
  // candidate grid (col, row index cells of `cell` pixels)
  const float px = __fmul_rn(__fadd_rn(static_cast<float>(col), 0.5f), cell);
  const float py = __fmul_rn(__fadd_rn(static_cast<float>(row), 0.5f), cell);

  // A. own list
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const uint4 w = ldg(&map_in[j * P + pix_off + q]);
    v[4 * j] = cand_key(w.x, sr, px, py, sites);
    v[4 * j + 1] = cand_key(w.y, sr, px, py, sites);
    v[4 * j + 2] = cand_key(w.z, sr, px, py, sites);
    v[4 * j + 3] = cand_key(w.w, sr, px, py, sites);
  }
  sort_desc<K>(v);
  bool dup = false;
#pragma unroll
  for (int k = 1; k < K; ++k) dup |= v[k] != 0ull && v[k] == v[k - 1];
  if (dup) {  // damaged input list: zero repeated keys, re-sort
#pragma unroll
    for (int k = K - 1; k > 0; --k)
      if (v[k] != 0ull && v[k] == v[k - 1]) v[k] = 0ull;
    sort_desc<K>(v);
  }

  // B + C. Novel ids (valid, not in the list) go to the thread's queue
  // column without a scan of the queue: an id that two neighbours offer is
  // queued twice and scored twice, and the insertion test drops the second
  // copy.  (Scanning the queue for every offer was a chain of dependent
  // shared loads, the slowest part of the pass at long jumps.)  The queue
  // is scored in groups of NG (2 NG independent gathers in flight) and
  // merged; the result is the top K of the union, whatever the order.  The
  // drain body has one call site and the offer body a few: fully unrolling
  // them over all candidates made the kernel too large for the instruction
  // cache.
  int qn = 0;
  auto drain = [&]() {
    // Score the queue in groups of NG; only ids whose key beats the list's
    // last key at the start of the drain are kept (compacted to the front
    // of the queue: a kept id never overwrites an unread one).  Few are
    // kept (about 0.2 insertions per pixel and pass once the field has
    // settled), so the insertion network below runs for those alone
    // instead of for every scored candidate of every lane in the warp.
    const uint64_t thr = v[K - 1];
    int nw = 0;
#pragma unroll 1
    for (int i = 0; i < qn; i += NG) {
      uint32_t id[NG];
      float4 g[NG], m[NG];
#pragma unroll
      for (int u = 0; u < NG; ++u) id[u] = s_q[i + u < qn ? i + u : i][tid];
#pragma unroll
      for (int u = 0; u < NG; ++u) sites.load(id[u], g[u], m[u]);
#pragma unroll
      for (int u = 0; u < NG; ++u) {
        uint64_t c = 0ull;
        if (i + u < qn && m[u].w != 0.f) {
          const float l = score_exact(px, py, g[u], m[u]);
          if (l == l) c = make_key(l, id[u]);
        }
        if (c > thr) s_q[nw++][tid] = id[u];
      }
    }
    // Insert the kept ids, re-scored: an id queued twice (offered by two
    // neighbours) finds itself in the list the second time, and a key that
    // an earlier insertion pushed below the list's last one is dropped.
#pragma unroll 1
    for (int i = 0; i < nw; ++i) {
      const uint32_t id = s_q[i][tid];
      float4 g, m;
      sites.load(id, g, m);
      const uint64_t c = make_key(score_exact(px, py, g, m), id);
      if (c > v[K - 1] && !list_has<K>(v, id)) list_insert<K>(v, c);
    }
    qn = 0;
  };
  auto offer = [&](uint32_t id) {
    if (STORE_ALL) {
      // qn <= QL - 1 here: a stage starts with room for all its offers
      const bool in_range = sr.has(id);
      const bool listed = list_has<K>(v, id);
      s_q[qn][tid] = id;
      qn += (in_range && !listed) ? 1 : 0;
    } else {
      if (!sr.has(id) || list_has<K>(v, id)) return;
      s_q[qn++][tid] = id;
    }
  };
  // One drain call site (the drain body is large; more copies cost
  // instruction-cache misses): stages 0..3 offer the four neighbours'
  // lists, stage 4 the injected ids.  After a stage the queue is drained
  // unless it has room for the next one: K ids before a neighbour, J
  // (at most 16, checked by every entry point) before the injections.
  static_assert(QL >= K && QL >= 16, "queue must hold a neighbour list or the injections");
  const int s = static_cast<int>(code >> 16);
  const uint64_t base = (static_cast<uint64_t>(code) << 32);
#pragma unroll 1
  for (int d = 0; d < 5; ++d) {
    if (d < 4) {
      const int nc = d == 0 ? col - s : (d == 1 ? col + s : col);
      const int nr = d == 2 ? row - s : (d == 3 ? row + s : row);
      if (nc >= 0 && nc < W && nr >= 0 && nr < H) {
        const size_t nq = pix_off + static_cast<size_t>(nr) * W + nc;
        uint4 w[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) w[j] = ldg(&map_in[j * P + nq]);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          offer(w[j].x);
          offer(w[j].y);
          offer(w[j].z);
          offer(w[j].w);
        }
      }
    } else {
#pragma unroll 1
      for (int j = 0; j < J; ++j) {
        const uint64_t ctr = base | static_cast<uint32_t>(q * static_cast<uint32_t>(J) + j);
        const uint64_t h = splitmix64_at(seed, ctr);
        offer(sr.lo + static_cast<uint32_t>(((h >> 32) * static_cast<uint64_t>(sr.n)) >> 32));
      }
    }
    if (d == 4 || qn > QL - (d == 3 ? (J > K ? J : K) : K)) drain();
  }
}

}  // namespace sad
