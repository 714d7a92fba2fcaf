// Per-tile adjoint / statistics of the SAD blend (App. "Gradient Computation
// and Reduction"), shared by the stand-alone backward and the fused training
// step.  Per pixel tile of 256 pixels (16x16, or 32x8 in the batched step;
// one 256-thread block, one pixel per thread):
//  1. forward: every pixel forms its max-subtracted softmax over its K
//     listed sites (no per-entry weights are stored): recomputed from the
//     site table; or, in the fused step, from the exact sorted logits its
//     propagation pass just produced, its list ending at the first entry
//     below 1e-7 of the running sum; or, in the saved-forward form, from
//     the render's max logit, 1/Z and blend.  It then forms its upstream
//     gradient g (given, or 2(c - I)/P for the fused MSE loss);
//  2. the tile's distinct sites get slots in a shared hash table (the paper's
//     multiplicative hash, linear probing), every lane probing for each of
//     its entries; each lane ORs its bit into its warp's word of a per-slot
//     pixel mask (order independent);
//  3. the masks give each slot a stable, pixel-ordered pair list; one warp
//     walks a slot's list 32 pairs at a time with the site's parameters in
//     registers and a fixed-order recursive-halving reduction sums the lane
//     partials into ten statistics per (site, tile), written as one record,
//     and counts the record for its site (the per-site sums are the
//     segmented reduce of sad_reduce.cuh).
//     If the table fills, the remaining sites are handled in further rounds.
#pragma once

#include "sad_device.cuh"
#include "sad_topk.cuh"

namespace sad {


constexpr int kTileSide = 16;
constexpr int kTileThreads = kTileSide * kTileSide;
constexpr int kSlots = 256;  // shared hash table size per round (power of 2)
constexpr int kLog2Slots = 8;
constexpr uint32_t kNone = 0xffffffffu;
constexpr int kModeGrad = 0;
constexpr int kModeStats = 1;

struct alignas(16) Record {
  uint32_t rank;  // place among its site's records (from the site's record count)
  uint32_t cj;    // compacted site index of the launch (its segment of the reduction)
  float acc[10];
};
static_assert(sizeof(Record) == 48, "record layout");

constexpr int kMaxImages = 64;

struct WsHeader {
  uint32_t cursor;    // records written
  uint32_t overflow;  // records that did not fit
  uint32_t done;      // blocks of the segment scan that have finished
  uint32_t pad[61];
  uint32_t pmax[kMaxImages][16];  // per image and statistic: bits of the largest |record value|
};
static_assert(sizeof(WsHeader) == 256 + 4 * 16 * kMaxImages, "header layout");

// ---------------------------------------------------------------------------
// block-wide exclusive scan of the packed slot counts over 256 threads (fixed order)
// ---------------------------------------------------------------------------
// 32-bit form for the slot scan: each value packs a pair count (at most 256
// per slot, 4096 per tile) in its low 16 bits and a record count (at most
// 256) in its high 16 bits, so the sums never carry across.  warp_tot must
// not be written again before a barrier that follows the call.
__device__ __forceinline__ uint32_t block_excl_scan256_u32(uint32_t v, uint32_t* warp_tot,
                                                           uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  uint32_t pre = 0u, run = 0u;
#pragma unroll
  for (int w = 0; w < kTileThreads / 32; ++w) {  // every thread adds the eight warp totals itself
    const uint32_t tw = warp_tot[w];
    pre += w < warp ? tw : 0u;
    run += tw;
  }
  total = run;
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

constexpr float kLog2e = 1.4426950408889634f;

// 2^x by the hardware's approximate base-2 exponential (the instruction the
// fast exponential uses; subnormal results flush to zero)
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The same over each quarter-warp (8 lanes, offsets 4, 2, 1; the quarters
// sum their own values): returns, on lane l, the totals of values 2 (l % 8)
// and 2 (l % 8) + 1 of its quarter (values 10..15 are padding).
__device__ __forceinline__ float2 quarter_sum10_halving(const float (&in)[10], int lane) {
  float a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = j < 10 ? in[j] : 0.f;
#pragma unroll
  for (int h = 8, o = 4; o >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float keep = up ? a[h + j] : a[j];
      const float give = up ? a[j] : a[h + j];
      a[j] = keep + __shfl_xor_sync(0xffffffffu, give, o);
    }
  }
  return make_float2(a[0], a[1]);
}

// The same over each half-warp (16 lanes, offsets 8, 4, 2, 1; the halves sum
// their own values): returns, on lane l, the total of value l % 16 of its
// half (values 10..15 are padding).
__device__ __forceinline__ float half_sum10_halving(const float (&in)[10], int lane) {
  float a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = j < 10 ? in[j] : 0.f;
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float keep = up ? a[h + j] : a[j];
      const float give = up ? a[j] : a[h + j];
      a[j] = keep + __shfl_xor_sync(0xffffffffu, give, h);
    }
  }
  return a[0];
}

// ---------------------------------------------------------------------------
// per-tile kernel
// ---------------------------------------------------------------------------
// Geometry of one tile of one image of a (possibly single-image) batch.
struct TileCtx {
  int H, W;          // image size
  int x0, y0;        // tile origin inside the image
  size_t pix_off;    // first pixel of the image in the packed per-pixel arrays
  SiteRange sr;      // the image's site ids
  uint32_t site_cum; // compacted index of the image's first site (sites of the images before it)
  uint32_t tile;     // global tile index (slot of the tile loss)
  uint32_t img;      // image index (< kMaxImages)
  float two_over_P;  // 2 / (H W): gradient of the mean loss
};

struct TileIO {
  const float4 *geo, *met, *col;  // prepared sites (global ids)
  const float* grad_rgb;          // dL/dc per pixel, or NULL (fused MSE with target)
  const float* target;            // target image(s), packed pixels
  float* rgb_out;                 // optional render
  float* tile_loss;               // optional per-tile squared-error sums
  Record* records;
  uint2* place;  // per record {place among its site's records, compacted site index}, for the scatter
  uint32_t max_records;
  WsHeader* hdr;
  uint32_t* site_cnt;  // records per compacted site index (incremented per stored record)
  float2* bias = nullptr;  // training step: per image {1 - beta1^t, 1 - beta2^t} for the site step
  float beta1 = 0.f, beta2 = 0.f;
  const float* fwd = nullptr;     // saved forward: float32[2][P] {max logit, 1/Z} per pixel
  const float* rgb_in = nullptr;  // saved forward: the blend c per pixel, float32[P][3]
  // the tile's lists in global memory (K/4 uint4 planes of lists_P entries,
  // indexed by the packed pixel index), re-read by the slot rounds instead of
  // keeping the ids in registers through the tile body
  const uint4* lists = nullptr;
  size_t lists_P = 0;
};

// Adjoint (MODE = kModeGrad) or budget statistics (kModeStats) of one tile
// of TW x (256 / TW) pixels whose pixels' lists are ids[] (thread t = pixel
// (t % TW, t / TW) of the tile).
// With HAVE_L (gradient mode), lk[] holds the logits of the listed sites in
// descending order (the propagation pass just computed them exactly; invalid
// entries are the empty tail), so the forward takes them instead of
// re-gathering and re-scoring, and the first entry is the maximum.
// Every thread of the 256-thread block must call it.
// The tile body's shared memory, as one object so that a kernel can overlay
// it on other shared data it no longer needs (the fused step: the
// propagation's candidate queue).
template <int K, int MODE>
struct TileShared {
  static constexpr int kW = kTileThreads / 32;
  uint32_t keys[kSlots];
  uint32_t mask[kW][kSlots];  // [warp word][slot]: conflict-free per-slot reads
  uint16_t wpre[kW][kSlots];
  uint32_t cnt[kSlots];
  uint32_t off[kSlots];
  uint32_t rix[kSlots];
  uint8_t order[kSlots];           // this round's slots with a record, largest pair counts first
  uint32_t hist[32];               // slots per 8-wide pair-count bucket (largest first)
  uint32_t hoff[32];               // their exclusive prefix
  uint8_t list[kTileThreads * K];
  // per pixel.  gradient mode: {m log2 e - log2(1/Z), 1/Z, g.cbar, gx},
  // {gy, gz, px, py};
  // statistics mode: {m, 1/Z, cbar.x, cbar.y}, {cbar.z, I}, {c' of the
  // dominant site (blend without it), dominant id}
  float4 pa[kTileThreads];
  float4 pg[MODE == kModeStats ? 1 : kTileThreads];
  float4 pb[MODE == kModeStats ? kTileThreads : 1];
  float4 pc[MODE == kModeStats ? kTileThreads : 1];
  uint32_t scan[kW];
  float red[kW];
  uint32_t base;
  uint32_t next;      // the walk's next record index (slots are taken in turn by the warps)
  uint32_t pmax[10];  // the tile's largest |record value| per statistic (float bits)
};

template <int K, int MODE, bool HAVE_L = false, int TW = kTileSide, bool SAVED = false>
__device__ __forceinline__ void tile_body(const TileCtx& c, const TileIO& io, uint32_t (&ids)[K],
                                          const float (&lk)[K], TileShared<K, MODE>& sm) {
  const float4* __restrict__ geo = io.geo;
  const float4* __restrict__ met = io.met;
  const float4* __restrict__ col = io.col;
  const float* __restrict__ grad_rgb = io.grad_rgb;
  const float* __restrict__ target = io.target;
  float* __restrict__ rgb_out = io.rgb_out;
  float* __restrict__ tile_loss = io.tile_loss;
  Record* __restrict__ records = io.records;
  const uint32_t max_records = io.max_records;
  WsHeader* __restrict__ hdr = io.hdr;
  const float two_over_P = c.two_over_P;
  constexpr int kWarps = kTileThreads / 32;
  auto& s_keys = sm.keys;
  auto& s_mask = sm.mask;
  auto& s_wpre = sm.wpre;
  auto& s_cnt = sm.cnt;
  auto& s_off = sm.off;
  auto& s_rix = sm.rix;
  auto& s_list = sm.list;
  auto& s_pa = sm.pa;
  auto& s_pg = sm.pg;
  auto& s_pb = sm.pb;
  auto& s_pc = sm.pc;
  auto& s_scan = sm.scan;
  auto& s_red = sm.red;
  auto& s_base = sm.base;
  auto& s_pmax = sm.pmax;

  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const int H = c.H, W = c.W, x0 = c.x0, y0 = c.y0;
  const uint32_t tile = c.tile;
  static_assert(TW == 16 || TW == 32, "tile width 16 (16x16 tiles) or 32 (32x8 tiles)");
  constexpr int kLog2TW = TW == 16 ? 4 : 5;
  const int x = x0 + (t & (TW - 1));
  const int y = y0 + (t >> kLog2TW);
  const bool inimg = x < W && y < H;
  const size_t q = inimg ? c.pix_off + static_cast<size_t>(y) * W + x : 0;
  const SiteRange sr = c.sr;
  const float px = x + 0.5f, py = y + 0.5f;
  if (t < 10) s_pmax[t] = 0u;

  // ---- 1. per-pixel forward (entries outside the image's sites are invalid)
#pragma unroll
  for (int k = 0; k < K; ++k) ids[k] = (inimg && sr.has(ids[k])) ? ids[k] : kInvalid;
  float m = -INFINITY;
  float z = 0.f;
  float3 cb = make_float3(0.f, 0.f, 0.f);
  uint32_t vm = 0;
  float l[MODE == kModeStats ? K : 1];
  if (SAVED) {
    // the render's max logit, 1/Z and blend (io.fwd, io.rgb_in): no
    // gathers; listed inactive sites contribute zero in the pair loop
#pragma unroll
    for (int k = 0; k < K; ++k) vm |= ids[k] != kInvalid ? (1u << k) : 0u;
    if (inimg) {
      const size_t P = static_cast<size_t>(c.H) * c.W;  // stand-alone: one image
      m = io.fwd[q];
      z = io.fwd[P + q];  // holds 1/Z here
      cb = make_float3(io.rgb_in[3 * q], io.rgb_in[3 * q + 1], io.rgb_in[3 * q + 2]);
    }
  } else if (MODE == kModeStats) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      l[k] = -INFINITY;
      if (ids[k] != kInvalid) {
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
  } else if (HAVE_L) {
    // sorted logits: the first valid entry is the maximum
    m = ids[0] != kInvalid ? lk[0] : -INFINITY;
    // entries whose weight is below 1e-7 of the running sum are left out of
    // the blend and of the pair lists (the rest of the list is smaller
    // still: it is sorted): at most 16e-7 of the pixel's weight, far
    // inside the loss and gradient tolerances, and no colour gathers or
    // pairs for them once the field has sharpened
    bool cut = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (ids[k] != kInvalid && !cut) {
        const float e = __expf(lk[k] - m);
        cut = e < 1e-7f * z;
        if (!cut) {
          vm |= 1u << k;
          const float4 ck = ldg(&col[ids[k]]);
          z += e;
          cb.x += e * ck.x;
          cb.y += e * ck.y;
          cb.z += e * ck.z;
        }
      }
    }
  } else {
    // online max-subtracted softmax over the list, kB entries at a time
    // (a new maximum is rare: lists are sorted by logit, so the rescale
    // is a branch, not a second exponential per entry)
    constexpr int kB = 1;
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += kB) {
      float4 g[kB], mt[kB], ck[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const uint32_t id = ids[k0 + u] != kInvalid ? ids[k0 + u] : sr.lo;
        g[u] = ldg(&geo[id]);
        mt[u] = ldg(&met[id]);
        ck[u] = ldg(&col[id]);
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const bool ok = ids[k0 + u] != kInvalid && mt[u].w != 0.f;
        vm |= ok ? (1u << (k0 + u)) : 0u;
        const float lk = score_fast(px, py, g[u], mt[u]).l;
        if (ok) {
          if (lk > m) {  // a new maximum: rare after the first entry (lists are sorted by logit)
            const float a = __expf(m - lk);
            z *= a;
            cb.x *= a;
            cb.y *= a;
            cb.z *= a;
            m = lk;
          }
          const float b = lk == m ? 1.f : __expf(lk - m);
          z += b;
          cb.x += b * ck[u].x;
          cb.y += b * ck[u].y;
          cb.z += b * ck[u].z;
        }
      }
    }
  }
  const float iz = SAVED ? z : (vm ? 1.f / z : 0.f);
  if (!SAVED) {
    cb.x *= iz;
    cb.y *= iz;
    cb.z *= iz;
  }
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
    // the pair weight is exp2(tau s log2 e (r - n) - M2) with M2 = m log2 e -
    // log2(1/Z): the max logit and the normaliser folded into one offset
    const float m2 = vm ? m * kLog2e - __log2f(iz) : 0.f;
    s_pa[t] = make_float4(m2, iz, g.x * cb.x + g.y * cb.y + g.z * cb.z, g.x);
    s_pg[t] = make_float4(g.y, g.z, px, py);
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
  // lanes i, 8 + i, 16 + i, 24 + i (i < 5): the largest |value| of statistics
  // 2i (pm) and 2i + 1 (pm1) in this warp's records (float bits)
  uint32_t pm = 0u, pm1 = 0u;
  uint32_t got = 0u;      // entries that got a slot this round (their slots replace the ids in idr[])
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (;;) {
    // this round's ids from the lists in memory (the same entries as ids[],
    // validated the same way; ids[] is dead after the forward)
    uint32_t idr[K];
#pragma unroll
    for (int j = 0; j < K / 4; ++j) {
      uint4 w = make_uint4(kInvalid, kInvalid, kInvalid, kInvalid);
      if (inimg) w = ldg(&io.lists[j * io.lists_P + q]);
      idr[4 * j] = w.x;
      idr[4 * j + 1] = w.y;
      idr[4 * j + 2] = w.z;
      idr[4 * j + 3] = w.w;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) idr[k] = sr.has(idr[k]) ? idr[k] : kInvalid;
    if (t < 32) sm.hist[t] = 0u;
    for (int i = t; i < kSlots; i += kTileThreads) {
      s_keys[i] = kInvalid;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s_mask[w][i] = 0u;
    }
    __syncthreads();
    // Every lane probes the table for each of its pending entries.  Lanes
    // next to each other that got the same slot form a run; the run's first
    // lane ORs the run's bits into its warp's mask word of the slot (one
    // shared atomic per run instead of one per lane: lanes of a warp that
    // list the same site at the same rank would otherwise serialise on one
    // word).  OR is order independent, so the masks (and the pair lists
    // built from them) are deterministic.  Slot numbers are kept as bytes.
    got = 0u;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      uint32_t sl = kNone;
      if ((pending >> k & 1u) != 0u) sl = probe_slot(idr[k], s_keys);
      const uint32_t left = __shfl_up_sync(0xffffffffu, sl, 1);
      const bool lead = sl != kNone && (lane == 0 || left != sl);
      const unsigned breaks = __ballot_sync(0xffffffffu, lead || sl == kNone);
      if (lead) {
        const unsigned above = breaks & ~((2u << lane) - 1u);  // run breaks after this lane
        const unsigned upto = above ? (above & (0u - above)) - 1u : 0xffffffffu;
        atomicOr(&s_mask[warp][sl], upto & ~((1u << lane) - 1u));
      }
      if (sl != kNone) {
        pending &= ~(1u << k);
        got |= 1u << k;
        idr[k] = sl;  // the id is not needed again this round
      }
    }
    __syncthreads();
    uint32_t packed = 0;
    uint32_t b_id = 0u, b_pos = 0u;  // the slot's pair-count bucket and its place there
    if (t < kSlots && s_keys[t] != kInvalid) {
      uint32_t c = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        s_wpre[w][t] = static_cast<uint16_t>(c);
        c += __popc(s_mask[w][t]);
      }
      packed = c | (1u << 16);
      b_id = 31u - min(31u, (c - 1u) >> 3);
      b_pos = atomicAdd(&sm.hist[b_id], 1u);  // a place in the walk order, not a value
    }
    uint32_t total;
    const uint32_t ex = block_excl_scan256_u32(packed, s_scan, total);
    if (t < kSlots) {
      s_cnt[t] = packed & 0xffffu;
      s_off[t] = ex & 0xffffu;
      s_rix[t] = ex >> 16;
    }
    if (t < 32) {  // bucket offsets (the histogram is complete: the scan synchronised)
      const uint32_t h = sm.hist[t];
      uint32_t x = h;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      sm.hoff[t] = x - h;
    }
    if (t == 0) {
      s_base = atomicAdd(&hdr->cursor, total >> 16);
      sm.next = 0u;
    }
    __syncthreads();
    // thread t files slot t's record: its index, its site's compacted index
    // and its place among the site's records (the count's old value), taken
    // here so that the atomic's round trip overlaps the list build
    uint32_t r_idx = kNone, r_cj = 0u, r_rank = 0u;
    if (t < kSlots && s_keys[t] != kInvalid) {
      r_idx = s_base + s_rix[t];
      r_cj = c.site_cum + (s_keys[t] - sr.lo);
      if (r_idx < max_records) r_rank = atomicAdd(&io.site_cnt[r_cj], 1u);  // a count, not a value
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if ((got >> k & 1u) != 0u) {
        const uint32_t sl = idr[k];
        const uint32_t pos = s_off[sl] + s_wpre[warp][sl] + __popc(s_mask[warp][sl] & lt_mask);
        s_list[pos] = static_cast<uint8_t>(t);
      }
    }
    if (r_idx < max_records) {
      const uint2 rc = make_uint2(r_rank, r_cj);
      *reinterpret_cast<uint2*>(&records[r_idx]) = rc;
      io.place[r_idx] = rc;  // the scatter reads these 8 bytes contiguously
    }
    if (packed != 0u) sm.order[sm.hoff[b_id] + b_pos] = static_cast<uint8_t>(t);
    __syncthreads();
    // Four slots at a time, one per quarter-warp: the 8 lanes walk the slot's
    // pixel-ordered pairs, then a fixed-order reduction sums their partials.
    // The warps take groups of four slots in turn from a shared counter, in
    // the order of the slots' pair counts (8-wide buckets, largest first),
    // so the quarters of a warp walk similar counts; a slot's record is the
    // same whichever quarter-warp computes it.
    const uint32_t n_rec = total >> 16;
    const int quarter = lane >> 3, ql = lane & 7;
    for (;;) {
      uint32_t j = 0u;
      if (lane == 0) j = atomicAdd(&sm.next, 4u);
      j = __shfl_sync(0xffffffffu, j, 0);
      if (j >= n_rec) break;
      {
        const bool live = j + quarter < n_rec;  // the last group may leave quarters idle
        const int sl = sm.order[live ? j + quarter : j];
        const uint32_t cnt = live ? s_cnt[sl] : 0u;
        const uint32_t id = s_keys[sl];
        const uint32_t off = s_off[sl];
        const uint32_t ridx = s_base + s_rix[sl];
        const float4 gs = ldg(&geo[id]), ms = ldg(&met[id]), cs = ldg(&col[id]);
        float acc[10];
#pragma unroll
        for (int j = 0; j < 10; ++j) acc[j] = 0.f;
        // (ms.w = 0 only for a listed inactive site in the saved-forward
        // mode: its weights are zero, so its pairs are skipped)
        const uint32_t n_pairs = (SAVED && ms.w == 0.f) ? 0u : cnt;
        if (MODE == kModeStats) {
          for (uint32_t i = ql; i < n_pairs; i += 8) {
            const uint32_t p = s_list[off + i];
            const float4 A = s_pa[p];
            const float dx = (x0 + static_cast<int>(p & (TW - 1)) + 0.5f) - gs.x;
            const float dy = (y0 + static_cast<int>(p >> kLog2TW) + 0.5f) - gs.y;
            const float qq = ms.x * dx * dx + 2.f * ms.y * dx * dy + ms.z * dy * dy;
            const float n = sqrtf(fmaxf(qq, 0.f));
            const float w = __expf(gs.z * (gs.w - n) - A.x) * A.y;
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
          }
        } else {
          const float g01 = 2.f * ms.y;
          const float tsl = gs.z * kLog2e;
          for (uint32_t i = ql; i < n_pairs; i += 8) {
            const uint32_t p = s_list[off + i];
            // A = {M2, 1/Z, g.cbar, gx}, B = {gy, gz, px, py}
            const float4 A = s_pa[p];
            const float4 B = s_pg[p];
            const float dx = B.z - gs.x, dy = B.w - gs.y;
            const float qq = (ms.x * dx + g01 * dy) * dx + ms.z * dy * dy;
            // n and 1/n from one reciprocal square root (the adjoint's
            // tolerance allows its few-ulp error; no division); 1/n is taken
            // as 0 at the site itself, where the position terms vanish
            const float qc = fmaxf(qq, 0.f);
            const float rq = qc > 0.f ? rsqrtf(qc) : 0.f;
            const float n = qc * rq;
            const float w = ex2_approx(fmaf(tsl, gs.w - n, -A.x));
            const float d = w * (A.w * cs.x + B.x * cs.y + B.y * cs.z - A.z);
            acc[0] += w * A.w;
            acc[1] += w * B.x;
            acc[2] += w * B.y;
            acc[3] += d;
            acc[4] += d * n;
            const float a = d * rq;
            const float ax = a * dx, ay = a * dy;
            acc[5] += ax;
            acc[6] += ay;
            acc[7] += ax * dx;
            acc[8] += ax * dy;
            acc[9] += ay * dy;
          }
        }
        // sum the 10 lane partials over each quarter by recursive halving
        // (fixed order): afterwards lane i of a quarter holds the totals of
        // statistics 2i and 2i + 1
        const float2 tot = quarter_sum10_halving(acc, lane);
        if (live) {
          if (ridx < max_records) {
            if (ql < 5) {
              const float v0 = isfinite(tot.x) ? tot.x : 0.f;  // non-finite contributions are dropped
              const float v1 = isfinite(tot.y) ? tot.y : 0.f;
              *reinterpret_cast<float2*>(&records[ridx].acc[2 * ql]) = make_float2(v0, v1);
              pm = max(pm, __float_as_uint(fabsf(v0)));
              pm1 = max(pm1, __float_as_uint(fabsf(v1)));
            }
          } else if (ql == 0) {
            hdr->overflow = 1u;
          }
        }
      }
    }
    if (!__syncthreads_or(pending != 0u)) break;
  }
  // the image's scale of the per-site sums: the largest |record value| of
  // each statistic (the max is order independent)
  if (pm != 0u) atomicMax(&s_pmax[2 * (lane & 7)], pm);  // a bound, not a value
  if (pm1 != 0u) atomicMax(&s_pmax[2 * (lane & 7) + 1], pm1);
  __syncthreads();
  if (t < 10 && s_pmax[t]) atomicMax(&hdr->pmax[c.img][t], s_pmax[t]);
}

}  // namespace sad
