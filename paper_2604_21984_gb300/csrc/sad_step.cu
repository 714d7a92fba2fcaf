// Fused, batched training step (the paper's GPU-resident iteration, Sec. 5;
// Sec. 6.3 epoch = one pass over all pixels) over up to kMaxImages images.
//
// One iteration is five kernels and one small memset, all on one stream.  Each
// image's counters (Adam step, pass index, which map buffer is current) live
// in a device state row that the step itself advances, so a fixed set of
// images always makes the same call, which is captured once in a CUDA graph
// and replayed:
//  1. k_step_tile, one block per tile (16x16 or 32x8) of any image: the tile's pixels
//     run one propagation pass at jump 1 (Sec. 4.3; reads the neighbours' old
//     lists, writes the new ones), then - on the lists just computed, still in
//     registers - the fused render + MSE + adjoint of the tile (per-tile
//     records, deterministic);
//  2. the segmented reduce of the records (sad_reduce.cuh): k_seg_scan of the
//     per-site record counts and k_rec_scatter, which files the records by
//     site;
//  3. k_site_step, one thread per site: the exact sum of the site's records
//     (its warp shares out the records of its 32 sites), the chain rule to
//     the 11 gradients,
//     Adam with the paper's clamps (Sec. 6.1), and the prepared table of the
//     updated site for the next iteration; its blocks also take the
//     per-image mean loss (fixed-order sums) and advance each image's state
//     row.
// Each image uses its own site range, pixel range and injection seed, and a
// site's sum depends on its own records only, so an image's result does not
// depend on the rest of the batch.
#include <cmath>

#include "sad_adam.cuh"
#include "sad_blend.cuh"
#include "sad_host.h"
#include "sad_reduce.cuh"
#include "sad_tile.cuh"
#include "sad_topk.cuh"

namespace sad {

struct BatchImg {
  int32_t H, W;
  uint32_t site_lo, site_n;
  uint64_t pix_off;
  uint32_t tile_off, tiles_x;
  uint64_t seed;
  float s, two_over_P;
  int32_t state;      // row of the image in the per-image state array
  uint32_t site_cum;  // sites of the images before this one
  int32_t flags;      // SAD_STEP_KEEP_LISTS: no propagation this call
};

constexpr int kStateWords = 4;  // per image: {Adam step t, pass index, map parity, reserved}

struct BatchDesc {
  int32_t B;
  int32_t tw;  // tile width: 16 (16x16 tiles) or 32 (32x8 tiles)
  uint32_t n_tiles;
  uint32_t n_sites;  // sites of all images
  BatchImg img[kMaxImages];
};

// image of a block's tile (uniform per block)
__device__ __forceinline__ int image_of_tile(const BatchDesc& d, uint32_t tile) {
  int lo = 0, hi = d.B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d.img[mid].tile_off <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// image of the j-th site of the table (j < n_sites)
__device__ __forceinline__ int image_of_slot(const BatchDesc& d, uint32_t j) {
  int lo = 0, hi = d.B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d.img[mid].site_cum <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ TileCtx tile_ctx(const BatchDesc& d, int b, uint32_t tile) {
  const BatchImg& im = d.img[b];
  const uint32_t lt = tile - im.tile_off;
  TileCtx c;
  c.H = im.H;
  c.W = im.W;
  c.x0 = static_cast<int>(lt % im.tiles_x) * d.tw;
  c.y0 = static_cast<int>(lt / im.tiles_x) * (kTileThreads / d.tw);
  c.pix_off = im.pix_off;
  c.sr = SiteRange{im.site_lo, im.site_n};
  c.site_cum = im.site_cum;
  c.tile = tile;
  c.img = static_cast<uint32_t>(b);
  c.two_over_P = im.two_over_P;
  return c;
}

constexpr int kKeepLists = SAD_STEP_KEEP_LISTS;

// Adam's bias corrections 1 - beta^t of every image of the step, in double,
// by the first threads of block 0 of the tile kernel (the site step, two
// launches later, reads them instead of taking two double-precision powers
// per site).
__device__ __forceinline__ void write_bias(const BatchDesc& d, const int32_t* state, const TileIO& io) {
  if (io.bias == nullptr || blockIdx.x != 0 || static_cast<int>(threadIdx.x) >= d.B) return;
  const int t = state[kStateWords * d.img[threadIdx.x].state];
  io.bias[threadIdx.x] = make_float2(static_cast<float>(1.0 - pow(static_cast<double>(io.beta1), t)),
                                     static_cast<float>(1.0 - pow(static_cast<double>(io.beta2), t)));
}

// Propagation pass + adjoint of the tiles of images that refresh their lists
// this call (UPDATE_ONLY: the pass alone, for extra passes between steps).
template <int K, bool UPDATE_ONLY, int TW>
__global__ void __launch_bounds__(kTileThreads, UPDATE_ONLY ? 3 : 4)
    k_step_tile(const BatchDesc d, TileIO io, uint4* map_a, uint4* map_b, size_t Ptot, int J,
                const int32_t* __restrict__ state) {
  // the propagation's candidate queue and the tile body's tables are never
  // live together: one shared region
  __shared__ union Smem {
    uint32_t q[kQueueStep][kTileThreads];
    TileShared<K, kModeGrad> t;
  } sm;
  auto& s_q = sm.q;
  if (!UPDATE_ONLY) write_bias(d, state, io);
  const int b = image_of_tile(d, blockIdx.x);
  const BatchImg im = d.img[b];
  if (!UPDATE_ONLY && (im.flags & kKeepLists)) return;  // whole block: handled by k_keep_tile
  const int32_t* st = state + kStateWords * im.state;
  const bool swap = st[2] & 1;
  const uint4* map_in = swap ? map_b : map_a;
  uint4* map_out = swap ? map_a : map_b;
  const TileCtx c = tile_ctx(d, b, blockIdx.x);
  const int t = threadIdx.x;
  const int x = c.x0 + (t & (TW - 1)), y = c.y0 + t / TW;
  const bool inimg = x < c.W && y < c.H;
  const uint32_t code = (1u << 16) | (static_cast<uint32_t>(st[1]) & 0xffffu);
  uint64_t v[K];
  pixel_update<K, kTileThreads, 2, !UPDATE_ONLY, kQueueStep>(v, inimg, x, y, c.H, c.W, c.sr, F32Sites{io.geo, io.met}, map_in, Ptot,
                                im.pix_off, code, J, im.seed, s_q, t);
  uint32_t ids[K];
  float lk[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    ids[k] = key_id(v[k]);
    lk[k] = key_logit(v[k]);
  }
  if (inimg) {
    const size_t q = im.pix_off + static_cast<size_t>(y) * c.W + x;
#pragma unroll
    for (int j = 0; j < K / 4; ++j)
      map_out[j * Ptot + q] = make_uint4(ids[4 * j], ids[4 * j + 1], ids[4 * j + 2], ids[4 * j + 3]);
  }
  if (!UPDATE_ONLY) {
    __syncthreads();  // every thread's queue is drained before the tables overwrite it
    TileIO tio = io;
    tio.lists = map_out;  // this thread's own pixel's lists, written just above
    tio.lists_P = Ptot;
    tile_body<K, kModeGrad, true, TW>(c, tio, ids, lk, sm.t);
  }
}

// Adjoint of the tiles of images that keep their lists this call: the lists
// are read from the image's current map (candidate update period > 1).
template <int K, int TW>
__global__ void __launch_bounds__(kTileThreads, 3)
    k_keep_tile(const BatchDesc d, TileIO io, const uint4* map_a, const uint4* map_b, size_t Ptot,
                const int32_t* __restrict__ state) {
  write_bias(d, state, io);
  const int b = image_of_tile(d, blockIdx.x);
  const BatchImg im = d.img[b];
  if (!(im.flags & kKeepLists)) return;
  const int32_t* st = state + kStateWords * im.state;
  const uint4* map = (st[2] & 1) ? map_b : map_a;
  const TileCtx c = tile_ctx(d, b, blockIdx.x);
  const int t = threadIdx.x;
  const int x = c.x0 + (t & (TW - 1)), y = c.y0 + t / TW;
  uint32_t ids[K];
#pragma unroll
  for (int j = 0; j < K / 4; ++j) {
    uint4 w = make_uint4(kInvalid, kInvalid, kInvalid, kInvalid);
    if (x < c.W && y < c.H) w = ldg(&map[j * Ptot + im.pix_off + static_cast<size_t>(y) * c.W + x]);
    ids[4 * j] = w.x;
    ids[4 * j + 1] = w.y;
    ids[4 * j + 2] = w.z;
    ids[4 * j + 3] = w.w;
  }
  float lk[K];  // unused without HAVE_L
#pragma unroll
  for (int k = 0; k < K; ++k) lk[k] = 0.f;
  __shared__ TileShared<K, kModeGrad> sm;
  TileIO tio = io;
  tio.lists = map;
  tio.lists_P = Ptot;
  tile_body<K, kModeGrad, false, TW>(c, tio, ids, lk, sm);
}

// After a propagation-only pass: every image's pass index and map parity advance.
__global__ void k_state_pass(const BatchDesc d, int32_t* __restrict__ state) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.B) return;
  int32_t* st = state + kStateWords * d.img[b].state;
  st[1] += 1;
  st[2] ^= 1;
}

// The filed records of the step (the segmented reduce's output).
struct SiteSums {
  const uint32_t* start;  // local segment start per compacted site index
  const uint32_t* boff;   // offset per block of kSegBlock sites; boff[nb] = records filed
  const uint32_t* dir;    // record indices, by segment
  const Record* rec;
  const WsHeader* hdr;    // per image the scale of the sums
};

// The ten exact statistic sums of site i -> 11 gradients -> Adam -> prepared
// table for the next iteration.  adam = false only prepares.  One thread per
// site of the table (slot ranges of the images only; j is the compacted
// index).
__device__ __forceinline__ void site_work(const BatchDesc& d, uint32_t j, float* __restrict__ params,
                                          float* __restrict__ m, float* __restrict__ v,
                                          float4* __restrict__ geo, float4* __restrict__ met,
                                          float4* __restrict__ col, int cap, const float (&acc)[10],
                                          bool any, const AdamArgs& A,
                                          const float2* __restrict__ bias,
                                          float* __restrict__ grads_out, bool adam) {
  const int b = image_of_slot(d, j);
  const BatchImg im = d.img[b];
  const uint32_t i = im.site_lo + (j - im.site_cum);
  const size_t c = static_cast<size_t>(cap);
  float p[kNParams];
#pragma unroll
  for (int k = 0; k < kNParams; ++k) p[k] = params[k * c + i];
  float m0[kNParams], v0[kNParams];  // issued with the other loads, used by Adam at the end
  if (adam) {
#pragma unroll
    for (int k = 0; k < kNParams; ++k) {
      m0[k] = m[k * c + i];
      v0[k] = v[k * c + i];
    }
  }
  if (adam) {
    float g[kNParams];
#pragma unroll
    for (int k = 0; k < kNParams; ++k) g[k] = 0.f;
    if (any) {
      const float4 gs = geo[i], ms = met[i];
      // chain rule through G(a, b, u) (Sec. 4.1), as in the stand-alone backward
      const float ts = gs.z, r = gs.w;
      const float G00 = ms.x, G01 = ms.y, G11 = ms.z;
      const float rawx = p[PUX], rawy = p[PUY];
      const float nrm2 = rawx * rawx + rawy * rawy;
      float ux = 1.f, uy = 0.f;
      if (nrm2 > 0.f) {
        const float inv = rsqrtf(nrm2);
        ux = rawx * inv;
        uy = rawy * inv;
      }
      const float ep = expf(p[PB] + p[PA]), em = expf(p[PB] - p[PA]);
      const float gG00 = -0.5f * ts * acc[7];
      const float gG01 = -ts * acc[8];
      const float gG11 = -0.5f * ts * acc[9];
      g[PX] = ts * (G00 * acc[5] + G01 * acc[6]);
      g[PY] = ts * (G01 * acc[5] + G11 * acc[6]);
      g[PLOGTAU] = ts * (r * acc[3] - acc[4]);
      g[PR] = ts * acc[3];
      g[PCR] = acc[0];
      g[PCG] = acc[1];
      g[PCB] = acc[2];
      const float xx = ux * ux, yy = uy * uy, xy = ux * uy;
      g[PA] = gG00 * (ep * xx - em * yy) + gG01 * (ep + em) * xy + gG11 * (ep * yy - em * xx);
      g[PB] = gG00 * G00 + gG01 * G01 + gG11 * G11;
      const float gth = (ep - em) * (-2.f * xy * gG00 + (xx - yy) * gG01 + 2.f * xy * gG11);
      g[PUX] = nrm2 > 0.f ? -gth * rawy / nrm2 : 0.f;
      g[PUY] = nrm2 > 0.f ? gth * rawx / nrm2 : 0.f;
    }
    if (grads_out) {
#pragma unroll
      for (int k = 0; k < kNParams; ++k) grads_out[k * c + i] = g[k];
    }
    if (p[PX] >= 0.f) {
      const float2 bc = bias[b];  // written by the tile kernel of this step
      adam_site_mv(p, g, m0, v0, m, v, c, i, A, bc.x, bc.y, im.H, im.W);
#pragma unroll
      for (int k = 0; k < kNParams; ++k) params[k * c + i] = p[k];
    }
  }
  prepare_site(p[PX], p[PY], p[PLOGTAU], p[PR], p[PCR], p[PCG], p[PCB], p[PUX], p[PUY], p[PA],
               p[PB], im.s, geo[i], met[i], col[i], col[c + i], col[2 * c + i],
               reinterpret_cast<float*>(col + 3 * c)[i]);
}

// The step's finish for image b: its mean loss from the tile losses (fixed
// order) and its state row advanced.  Every thread of the block calls it.
__device__ __forceinline__ void finish_image(const BatchDesc& d, int b, const float* __restrict__ tile_loss,
                                             float* __restrict__ loss, int32_t* __restrict__ state,
                                             float* s_w) {
  const BatchImg& im = d.img[b];
  const uint32_t n = (b + 1 < d.B ? d.img[b + 1].tile_off : d.n_tiles) - im.tile_off;
  float v = 0.f;
  for (uint32_t i = threadIdx.x; i < n; i += kSumThreads) v += tile_loss[im.tile_off + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float sum = 0.f;
    for (int w = 0; w < kSumThreads / 32; ++w) sum += s_w[w];
    if (loss) loss[b] = sum / static_cast<float>(static_cast<double>(im.H) * im.W);
    int32_t* st = state + kStateWords * im.state;  // the image's step is done
    st[0] += 1;
    if (!(im.flags & kKeepLists)) {
      st[1] += 1;
      st[2] ^= 1;
    }
  }
  __syncthreads();  // s_w is reused by the next image
}

// Per site: gradient -> Adam -> prepared table; with tile_loss, the blocks
// also do the step's per-image finish (no site step reads a state row, so
// advancing them here is safe).  kSumThreads threads per block.
__global__ void __launch_bounds__(kSumThreads, 4) k_site_step(const BatchDesc d, float* __restrict__ params, float* __restrict__ m,
                            float* __restrict__ v, float4* __restrict__ geo,
                            float4* __restrict__ met, float4* __restrict__ col, int cap,
                            const SiteSums S, AdamArgs A,
                            const float2* __restrict__ bias, float* __restrict__ grads_out,
                            bool adam, const float* __restrict__ tile_loss, float* __restrict__ loss,
                            int32_t* __restrict__ state) {
  __shared__ float s_w[kSumThreads / 32];
  __shared__ WarpSums<10> s_ws[kSumThreads / 32];
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  // the site's exact record sums: every lane of the warp takes part (the
  // warp's records are shared out evenly over its lanes)
  float acc[10];
  bool any = false;
  if (adam) {
    // the image's scale: its largest record values and its own tile count
    // (not the batch's), so that its sums do not depend on the batch
    const int b = j < d.n_sites ? image_of_slot(d, j) : 0;
    const uint32_t nt = (b + 1 < d.B ? d.img[b + 1].tile_off : d.n_tiles) - d.img[b].tile_off;
    const int L = 32 - __clz(nt > 0u ? nt : 1u);  // 2^L > nt
    any = warp_site_sums<10, 2>(j < d.n_sites, j, d.n_sites, S.start, S.boff, S.dir, S.rec, S.hdr->pmax[b], L,
                             s_ws[threadIdx.x >> 5], acc) != 0u;
  }
  if (j < d.n_sites) site_work(d, j, params, m, v, geo, met, col, cap, acc, any, A, bias, grads_out, adam);
  if (tile_loss != nullptr)
    for (int b = blockIdx.x; b < d.B; b += gridDim.x) finish_image(d, b, tile_loss, loss, state, s_w);
}

__global__ void __launch_bounds__(256) k_decode_batch(const BatchDesc d, const float4* __restrict__ ba,
                                                      const float4* __restrict__ bb,
                                                      const float* __restrict__ cbd,
                                                      const uint4* __restrict__ map, size_t Ptot,
                                                      int K, const float2* __restrict__ xy,
                                                      const int32_t* __restrict__ qimg, int64_t n,
                                                      float* __restrict__ rgb) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = qimg[i];
  float3 c = make_float3(0.f, 0.f, 0.f);
  if (b >= 0 && b < d.B) {
    const BatchImg im = d.img[b];
    const float2 p = ldg(&xy[i]);
    int cx = static_cast<int>(floorf(p.x));
    int cy = static_cast<int>(floorf(p.y));
    cx = cx < 0 ? 0 : (cx >= im.W ? im.W - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= im.H ? im.H - 1 : cy);
    const size_t q = im.pix_off + static_cast<size_t>(cy) * im.W + cx;
    const SiteRange sr{im.site_lo, im.site_n};
    switch (K) {
      case 4: c = blend_planes<1>(map, Ptot, q, p.x, p.y, sr, ba, bb, cbd); break;
      case 8: c = blend_planes<2>(map, Ptot, q, p.x, p.y, sr, ba, bb, cbd); break;
      default: c = blend_planes<4>(map, Ptot, q, p.x, p.y, sr, ba, bb, cbd); break;
    }
  }
  rgb[3 * i] = c.x;
  rgb[3 * i + 1] = c.y;
  rgb[3 * i + 2] = c.z;
}

// Copy of one image from the single-image layout into its ranges of the
// shared arrays: parameters (Adam moments cleared), target pixels, and map ids
// offset by the image's first slot (ids outside the image become empty).
__global__ void k_insert_sites(const float* __restrict__ src, int src_cap, int n, int lo,
                               float* __restrict__ params, float* __restrict__ m,
                               float* __restrict__ v, int cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t c = static_cast<size_t>(cap), sc = static_cast<size_t>(src_cap);
#pragma unroll
  for (int k = 0; k < kNParams; ++k) {
    params[k * c + lo + i] = src[k * sc + i];
    m[k * c + lo + i] = 0.f;
    v[k * c + lo + i] = 0.f;
  }
}

__global__ void k_insert_pixels(const uint4* __restrict__ src_map, const float* __restrict__ src_t,
                                size_t P, int NP, uint32_t n, uint32_t lo, size_t pix_off,
                                uint4* __restrict__ map, float* __restrict__ targets, size_t Ptot) {
  const size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= P) return;
  for (int j = 0; j < NP; ++j) {
    uint4 w = src_map[j * P + q];
    w.x = w.x < n ? w.x + lo : kInvalid;
    w.y = w.y < n ? w.y + lo : kInvalid;
    w.z = w.z < n ? w.z + lo : kInvalid;
    w.w = w.w < n ? w.w + lo : kInvalid;
    map[j * Ptot + pix_off + q] = w;
  }
  if (src_t) {
#pragma unroll
    for (int c = 0; c < 3; ++c) targets[3 * (pix_off + q) + c] = src_t[3 * q + c];
  }
}

struct StepLayout {
  size_t hdr, cnt, tile_loss, bias, start, bsums, dir, place, records, total;
  uint32_t max_records;
};

static inline size_t al256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

static StepLayout step_layout(uint32_t n_tiles, uint64_t total_pixels, int K, int total_cap,
                              int64_t max_records) {
  StepLayout L{};
  uint64_t mr = max_records > 0 ? static_cast<uint64_t>(max_records) : total_pixels * K / 8;
  if (max_records <= 0 && mr < 128ull * n_tiles) mr = 128ull * n_tiles;
  if (mr > 0xfffffff0ull) mr = 0xfffffff0ull;
  L.max_records = static_cast<uint32_t>(mr);
  // the per-site record counts keep their offset whatever the table (they
  // must stay zero between calls: the segment scan clears them)
  const size_t c = static_cast<size_t>(total_cap);
  size_t o = 0;
  L.hdr = o;       o = al256(o + sizeof(WsHeader));
  L.cnt = o;       o = al256(o + sizeof(uint32_t) * c);
  L.tile_loss = o; o = al256(o + sizeof(float) * n_tiles);
  L.bias = o;      o = al256(o + sizeof(float2) * kMaxImages);
  L.start = o;     o = al256(o + sizeof(uint32_t) * c);
  L.bsums = o;     o = al256(o + sizeof(uint32_t) * (seg_blocks(c) + 1));
  L.dir = o;       o = al256(o + sizeof(uint32_t) * L.max_records);
  L.place = o;     o = al256(o + sizeof(uint2) * L.max_records);
  L.records = o;   o = al256(o + sizeof(Record) * L.max_records);
  L.total = o;
  return L;
}

// Validates the host image table and fills the device descriptor.
static int make_desc(const sad_batch_image* images, int32_t B, int32_t total_cap,
                     int64_t total_pixels, BatchDesc& d, const char* name, int32_t n_states = -1,
                     int32_t tile_w = kTileSide) {
  if (!images || B < 1 || B > kMaxImages)
    return einval("%s: need 1 <= B <= %d images", name, kMaxImages);
  if (tile_w != 16 && tile_w != 32) return einval("%s: tile_w must be 16 or 32", name);
  const int32_t tile_h = kTileThreads / tile_w;
  d.B = B;
  d.tw = tile_w;
  uint32_t tiles = 0, sites = 0;
  for (int b = 0; b < B; ++b) {
    const sad_batch_image& im = images[b];
    if (int e = check_problem(im.capacity, im.H, im.W, 4, false)) return e;
    if (im.site_offset < 0 || static_cast<int64_t>(im.site_offset) + im.capacity > total_cap)
      return einval("%s: image %d sites outside [0, %d)", name, b, total_cap);
    if (b > 0 && im.site_offset < images[b - 1].site_offset + images[b - 1].capacity)
      return einval("%s: image %d sites overlap the previous image", name, b);
    if (im.pixel_offset < 0 || im.pixel_offset + static_cast<int64_t>(im.H) * im.W > total_pixels)
      return einval("%s: image %d pixels outside [0, %lld)", name, b,
                    static_cast<long long>(total_pixels));
    BatchImg& o = d.img[b];
    o.H = im.H;
    o.W = im.W;
    o.site_lo = static_cast<uint32_t>(im.site_offset);
    o.site_n = static_cast<uint32_t>(im.capacity);
    o.pix_off = static_cast<uint64_t>(im.pixel_offset);
    o.tiles_x = static_cast<uint32_t>((im.W + tile_w - 1) / tile_w);
    o.tile_off = tiles;
    o.seed = im.seed;
    o.s = 1.0f / static_cast<float>(im.H > im.W ? im.H : im.W);
    o.two_over_P = 2.0f / static_cast<float>(static_cast<double>(im.H) * im.W);
    o.state = im.state_index;
    if (n_states >= 0 && (im.state_index < 0 || im.state_index >= n_states))
      return einval("%s: image %d state_index %d outside [0, %d)", name, b, im.state_index, n_states);
    for (int c = 0; c < b && n_states >= 0; ++c)
      if (images[c].state_index == im.state_index)
        return einval("%s: images %d and %d share state row %d", name, c, b, im.state_index);
    if (im.flags & ~SAD_STEP_KEEP_LISTS) return einval("%s: image %d has unknown flags", name, b);
    o.flags = im.flags;
    o.site_cum = sites;
    sites += o.site_n;
    tiles += o.tiles_x * static_cast<uint32_t>((im.H + tile_h - 1) / tile_h);
  }
  for (int b = 0; b < B; ++b)
    for (int c = 0; c < b; ++c) {
      const int64_t a0 = images[b].pixel_offset, a1 = a0 + static_cast<int64_t>(images[b].H) * images[b].W;
      const int64_t c0 = images[c].pixel_offset, c1 = c0 + static_cast<int64_t>(images[c].H) * images[c].W;
      if (a0 < c1 && c0 < a1) return einval("%s: images %d and %d share pixels", name, c, b);
    }
  d.n_tiles = tiles;
  d.n_sites = sites;
  return SAD_OK;
}

}  // namespace sad

using namespace sad;

extern "C" {

size_t sad_step_workspace_bytes(const sad_batch_image* images, int32_t B, int32_t K,
                                int32_t tile_w, int32_t total_capacity, int64_t total_pixels,
                                int64_t max_records) {
  BatchDesc d;
  if (K != 4 && K != 8 && K != 16) return 0;
  if (make_desc(images, B, total_capacity, total_pixels, d, "sad_step_workspace_bytes", -1,
                tile_w) != SAD_OK)
    return 0;
  return step_layout(d.n_tiles, static_cast<uint64_t>(total_pixels), K, total_capacity, max_records)
      .total;
}

int sad_prepare_batch(const sad_batch_image* images, int32_t B, const float* params, float* prep,
                      int32_t total_capacity, int64_t total_pixels, void* stream) {
  BatchDesc d;
  if (int e = make_desc(images, B, total_capacity, total_pixels, d, "sad_prepare_batch")) return e;
  if (d.n_sites == 0) return SAD_OK;
  if (!params || !prep || !aligned16(prep)) return einval("sad_prepare_batch: bad pointer");
  float4* p4 = reinterpret_cast<float4*>(prep);
  AdamArgs A{};
  { TraceScope tr_(as_stream(stream), "k_site_step"); k_site_step<<<(d.n_sites + kSumThreads - 1) / kSumThreads, kSumThreads, 0, as_stream(stream)>>>(
      d, const_cast<float*>(params), nullptr, nullptr, p4, p4 + total_capacity,
      p4 + 2 * static_cast<size_t>(total_capacity), total_capacity, SiteSums{}, A, nullptr,
      nullptr, false, nullptr, nullptr, nullptr); }
  return check_launch("sad_prepare_batch");
}

int sad_train_step(const sad_batch_image* images, int32_t B, int32_t K, int32_t J, int32_t tile_w,
                   float* params, float* m, float* v, float* prep, int32_t total_capacity,
                   uint32_t* map_in, uint32_t* map_out, int64_t total_pixels,
                   const float* targets, float* loss, const sad_adam_hparams* hp,
                   int32_t* image_state, int32_t n_states, float* grads_out, void* workspace,
                   size_t workspace_bytes, void* stream) {
  BatchDesc d;
  if (int e = make_desc(images, B, total_capacity, total_pixels, d, "sad_train_step", n_states,
                        tile_w))
    return e;
  if (K != 4 && K != 8 && K != 16) return einval("sad_train_step: K must be 4, 8 or 16");
  if (J < 0 || J > 16) return einval("sad_train_step: J must be in [0,16]");
  if (static_cast<uint64_t>(total_pixels) * static_cast<uint64_t>(J > 0 ? J : 1) >= (1ull << 32))
    return einval("sad_train_step: pixels * J must be below 2^32");
  if (!params || !m || !v || !prep || !map_in || !map_out || !targets || !hp || !image_state ||
      !workspace)
    return einval("sad_train_step: null pointer");
  if (!aligned16(prep) || !aligned16(map_in) || !aligned16(map_out) ||
      (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return einval("sad_train_step: misaligned pointer");
  const size_t mbytes = static_cast<size_t>(total_pixels) * K * sizeof(uint32_t);
  const char* a = reinterpret_cast<const char*>(map_in);
  const char* bb = reinterpret_cast<const char*>(map_out);
  if (a < bb + mbytes && bb < a + mbytes) return einval("sad_train_step: maps overlap");
  const StepLayout L1 = step_layout(d.n_tiles, static_cast<uint64_t>(total_pixels), K,
                                    total_capacity, 1);
  if (workspace_bytes < L1.total) {
    set_error("sad_train_step: workspace has %zu bytes, needs at least %zu", workspace_bytes,
              L1.total);
    return SAD_EWORKSPACE;
  }
  StepLayout L = L1;
  {
    // per record: its 48 bytes and its directory entry; the two regions'
    // 256-byte alignment can hide up to 512 bytes, so start above and step down
    const uint64_t per = sizeof(Record) + sizeof(uint32_t) + sizeof(uint2);
    uint64_t mr = 1 + (workspace_bytes - L1.total + 512) / per;
    if (mr > 0xfffffff0ull) mr = 0xfffffff0ull;
    for (int it = 0; it < 64 && mr > 1; ++it, --mr) {
      const StepLayout T = step_layout(d.n_tiles, static_cast<uint64_t>(total_pixels), K,
                                       total_capacity, static_cast<int64_t>(mr));
      if (T.total <= workspace_bytes) {
        L = T;
        break;
      }
    }
  }
  cudaStream_t st = as_stream(stream);
  char* base = static_cast<char*>(workspace);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  float* tile_loss = reinterpret_cast<float*>(base + L.tile_loss);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base + L.cnt);
  uint32_t* start = reinterpret_cast<uint32_t*>(base + L.start);
  uint32_t* bsums = reinterpret_cast<uint32_t*>(base + L.bsums);
  uint32_t* dir = reinterpret_cast<uint32_t*>(base + L.dir);
  Record* rec = reinterpret_cast<Record*>(base + L.records);
  uint2* place = reinterpret_cast<uint2*>(base + L.place);
  const cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) {
    set_error("sad_train_step memset: %s", cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  float4* p4 = reinterpret_cast<float4*>(prep);
  TileIO io;
  io.geo = p4;
  io.met = p4 + total_capacity;
  io.col = p4 + 2 * static_cast<size_t>(total_capacity);
  io.grad_rgb = nullptr;
  io.target = targets;
  io.rgb_out = nullptr;
  io.tile_loss = tile_loss;
  io.records = rec;
  io.place = place;
  io.max_records = L.max_records;
  io.hdr = hdr;
  io.site_cnt = cnt;
  float2* bias = reinterpret_cast<float2*>(base + L.bias);
  io.bias = bias;
  io.beta1 = hp->beta1;
  io.beta2 = hp->beta2;
  uint4* mi = reinterpret_cast<uint4*>(map_in);
  uint4* mo = reinterpret_cast<uint4*>(map_out);
  const size_t Ptot = static_cast<size_t>(total_pixels);
  bool any_keep = false, any_refresh = false;
  for (int b = 0; b < B; ++b) {
    any_keep |= (images[b].flags & SAD_STEP_KEEP_LISTS) != 0;
    any_refresh |= (images[b].flags & SAD_STEP_KEEP_LISTS) == 0;
  }
  const int kt = K * 100 + tile_w;  // (K, tile width)
  if (any_refresh) {
    TraceScope tr_(st, "k_step_tile");
#define SAD_STEP(KK, TT) k_step_tile<KK, false, TT><<<d.n_tiles, kTileThreads, 0, st>>>(d, io, mi, mo, Ptot, J, image_state)
    switch (kt) {
      case 416: SAD_STEP(4, 16); break;
      case 432: SAD_STEP(4, 32); break;
      case 816: SAD_STEP(8, 16); break;
      case 832: SAD_STEP(8, 32); break;
      case 1632: SAD_STEP(16, 32); break;
      default: SAD_STEP(16, 16); break;
    }
#undef SAD_STEP
  }
  if (any_keep) {
    TraceScope tr_(st, "k_keep_tile");
#define SAD_KEEP(KK, TT) k_keep_tile<KK, TT><<<d.n_tiles, kTileThreads, 0, st>>>(d, io, mi, mo, Ptot, image_state)
    switch (kt) {
      case 416: SAD_KEEP(4, 16); break;
      case 432: SAD_KEEP(4, 32); break;
      case 816: SAD_KEEP(8, 16); break;
      case 832: SAD_KEEP(8, 32); break;
      case 1632: SAD_KEEP(16, 32); break;
      default: SAD_KEEP(16, 16); break;
    }
#undef SAD_KEEP
  }
  if (int r = check_launch("k_step_tile / k_keep_tile")) return r;
  // the segmented reduce: segment starts of the batch's sites (compacted
  // index), records filed by site
  run_seg_scan(cnt, d.n_sites, start, bsums, hdr, st);
  { TraceScope tr_(st, "k_rec_scatter"); k_rec_scatter<<<152 * 8, 256, 0, st>>>(place, hdr, L.max_records, start, bsums, dir); }
  if (int r = check_launch("k_rec_scatter")) return r;
  const SiteSums S{start, bsums, dir, rec, hdr};
  const AdamArgs A = adam_args(hp);
  {
    // the site step also finishes the step (per-image loss, state rows)
    const unsigned grid = d.n_sites > 0 ? (d.n_sites + kSumThreads - 1) / kSumThreads : 1;
    TraceScope tr_(st, "k_site_step");
    k_site_step<<<grid, kSumThreads, 0, st>>>(d, params, m, v, p4, p4 + total_capacity,
                                      p4 + 2 * static_cast<size_t>(total_capacity), total_capacity,
                                      S, A, bias, grads_out, true, tile_loss, loss, image_state);
  }
  return check_launch("k_site_step");
}

int sad_batch_update(const sad_batch_image* images, int32_t B, int32_t K, int32_t J,
                     const float* prep, int32_t total_capacity, uint32_t* map_in, uint32_t* map_out,
                     int64_t total_pixels, int32_t* image_state, int32_t n_states, void* stream) {
  BatchDesc d;
  if (int e = make_desc(images, B, total_capacity, total_pixels, d, "sad_batch_update", n_states))
    return e;
  if (K != 4 && K != 8 && K != 16) return einval("sad_batch_update: K must be 4, 8 or 16");
  if (J < 0 || J > 16) return einval("sad_batch_update: J must be in [0,16]");
  if (static_cast<uint64_t>(total_pixels) * static_cast<uint64_t>(J > 0 ? J : 1) >= (1ull << 32))
    return einval("sad_batch_update: pixels * J must be below 2^32");
  if (!prep || !map_in || !map_out || !image_state) return einval("sad_batch_update: null pointer");
  if (!aligned16(prep) || !aligned16(map_in) || !aligned16(map_out))
    return einval("sad_batch_update: misaligned pointer");
  const size_t mbytes = static_cast<size_t>(total_pixels) * K * sizeof(uint32_t);
  const char* a = reinterpret_cast<const char*>(map_in);
  const char* bb = reinterpret_cast<const char*>(map_out);
  if (a < bb + mbytes && bb < a + mbytes) return einval("sad_batch_update: maps overlap");
  cudaStream_t st = as_stream(stream);
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  TileIO io{};
  io.geo = p4;
  io.met = p4 + total_capacity;
  io.col = p4 + 2 * static_cast<size_t>(total_capacity);
  uint4* mi = reinterpret_cast<uint4*>(map_in);
  uint4* mo = reinterpret_cast<uint4*>(map_out);
  const size_t Ptot = static_cast<size_t>(total_pixels);
  {
    TraceScope tr_(st, "k_update_tile");
    switch (K) {
      case 4: k_step_tile<4, true, 16><<<d.n_tiles, kTileThreads, 0, st>>>(d, io, mi, mo, Ptot, J, image_state); break;
      case 8: k_step_tile<8, true, 16><<<d.n_tiles, kTileThreads, 0, st>>>(d, io, mi, mo, Ptot, J, image_state); break;
      default: k_step_tile<16, true, 16><<<d.n_tiles, kTileThreads, 0, st>>>(d, io, mi, mo, Ptot, J, image_state); break;
    }
  }
  if (int r = check_launch("k_update_tile")) return r;
  { TraceScope tr_(st, "k_state_pass"); k_state_pass<<<1, 64, 0, st>>>(d, image_state); }
  return check_launch("k_state_pass");
}

int sad_batch_insert(const sad_batch_image* image, int32_t K, const float* src_params,
                     int32_t src_capacity, const uint32_t* src_map, const float* src_target,
                     float* params, float* m, float* v, int32_t total_capacity, uint32_t* map,
                     float* targets, int64_t total_pixels, void* stream) {
  BatchDesc d;
  if (int e = make_desc(image, 1, total_capacity, total_pixels, d, "sad_batch_insert")) return e;
  if (K != 4 && K != 8 && K != 16) return einval("sad_batch_insert: K must be 4, 8 or 16");
  if (src_capacity < image->capacity)
    return einval("sad_batch_insert: src_capacity %d below the image's %d slots", src_capacity,
                  image->capacity);
  if ((image->capacity > 0 && (!src_params || !params || !m || !v)) || !src_map || !map ||
      (src_target && !targets))
    return einval("sad_batch_insert: null pointer");
  if (!aligned16(src_map) || !aligned16(map)) return einval("sad_batch_insert: maps must be 16-byte aligned");
  cudaStream_t st = as_stream(stream);
  if (image->capacity > 0) {
    { TraceScope tr_(st, "k_insert_sites"); k_insert_sites<<<(image->capacity + 255) / 256, 256, 0, st>>>(
        src_params, src_capacity, image->capacity, image->site_offset, params, m, v, total_capacity); }
    if (int r = check_launch("k_insert_sites")) return r;
  }
  const size_t P = static_cast<size_t>(image->H) * image->W;
  { TraceScope tr_(st, "k_insert_pixels"); k_insert_pixels<<<static_cast<unsigned>((P + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const uint4*>(src_map), src_target, P, K / 4,
      static_cast<uint32_t>(image->capacity), static_cast<uint32_t>(image->site_offset),
      static_cast<size_t>(image->pixel_offset), reinterpret_cast<uint4*>(map), targets,
      static_cast<size_t>(total_pixels)); }
  return check_launch("k_insert_pixels");
}

int sad_decode_batch(const sad_batch_image* images, int32_t B, int32_t K, const float* prep,
                     int32_t total_capacity, const uint32_t* map, int64_t total_pixels,
                     const float* xy, const int32_t* query_image, int64_t n, float* rgb,
                     void* stream) {
  BatchDesc d;
  if (int e = make_desc(images, B, total_capacity, total_pixels, d, "sad_decode_batch")) return e;
  if (K != 4 && K != 8 && K != 16) return einval("sad_decode_batch: K must be 4, 8 or 16");
  if (n < 0) return einval("sad_decode_batch: n must be >= 0");
  if (n == 0) return SAD_OK;
  if (!prep || !map || !xy || !query_image || !rgb) return einval("sad_decode_batch: null pointer");
  if (!aligned16(prep) || !aligned16(map) || (reinterpret_cast<uintptr_t>(xy) & 7u))
    return einval("sad_decode_batch: misaligned pointer");
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  { TraceScope tr_(as_stream(stream), "k_decode_batch"); k_decode_batch<<<static_cast<unsigned>((n + 255) / 256), 256, 0, as_stream(stream)>>>(
      d, p4 + 3 * static_cast<size_t>(total_capacity), p4 + 4 * static_cast<size_t>(total_capacity),
      reinterpret_cast<const float*>(p4 + 5 * static_cast<size_t>(total_capacity)),
      reinterpret_cast<const uint4*>(map), static_cast<size_t>(total_pixels), K,
      reinterpret_cast<const float2*>(xy), query_image, n, rgb); }
  return check_launch("k_decode_batch");
}

}  // extern "C"
