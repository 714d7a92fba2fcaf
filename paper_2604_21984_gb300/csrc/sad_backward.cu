// Adjoint of the blend (App. "Gradient Computation and Reduction", Per-pixel
// gradients) with a deterministic gradient reduction that replaces the
// per-tile hash table plus global float atomics of Sec. 4.8, Alg. 1
// (threadgroup hash reduction).
//
// Per 16x16 pixel tile (one CTA, one pixel per thread; sad_tile.cuh):
//  1. forward: every pixel forms its max-subtracted softmax over its K
//     listed sites (recomputed, or from the render's saved max logit, 1/Z
//     and blend), its upstream gradient g (given, or 2(c - I)/P for the
//     fused MSE loss), and parks {m, 1/Z, cbar, g} in shared memory;
//  2. the tile's distinct sites get slots in a shared hash table (the paper's
//     multiplicative hash, linear probing); each warp records, per slot, the
//     bitmask of its 32 pixels that list the site;
//  3. the masks give each slot a stable, pixel-ordered pair list; one warp
//     walks a slot's list 32 pairs at a time with the site's parameters in
//     registers (lane i takes pairs i, i+32, ...) and a fixed-order
//     reduction sums the lane partials, giving ten sufficient statistics per
//     (site, tile):
//       sum w g (3),  sum d,  sum d n,  sum d dx/n,  sum d dy/n,
//       sum d dx^2/n, sum d dx dy/n, sum d dy^2/n,   d = dL/dl = w g.(c_k - cbar)
//     written as one partial record per (site, tile).  If the table fills,
//     the remaining sites are handled in further rounds.
// Then a segmented reduce (sad_reduce.cuh) files the records by site and sums
// each site's records exactly, with no atomic on any gradient value; the
// eleven parameter gradients follow from the statistics by the chain rule
// through G(a, b, u) of Sec. 4.1.
#include "sad_device.cuh"
#include "sad_host.h"
#include "sad_reduce.cuh"
#include "sad_tile.cuh"

#include <mutex>

namespace sad {

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
struct WsLayout {
  size_t hdr, tile_loss, cnt, start, bsums, dir, place, records, total;
  uint32_t max_records, n_tiles;
};

static inline size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

// records: 48 B per (site, tile) plus its 4-byte directory entry; per site a
// record count and a segment start; the scan's block sums
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
  const size_t c = static_cast<size_t>(cap);
  size_t o = 0;
  L.hdr = o;        o = align256(o + sizeof(WsHeader));
  L.tile_loss = o;  o = align256(o + sizeof(float) * L.n_tiles);
  L.cnt = o;        o = align256(o + sizeof(uint32_t) * c);
  L.start = o;      o = align256(o + sizeof(uint32_t) * c);
  L.bsums = o;      o = align256(o + sizeof(uint32_t) * (seg_blocks(c) + 1));
  L.dir = o;        o = align256(o + sizeof(uint32_t) * L.max_records);
  L.place = o;      o = align256(o + sizeof(uint2) * L.max_records);
  L.records = o;    o = align256(o + sizeof(Record) * L.max_records);
  L.total = o;
  return L;
}

// ---------------------------------------------------------------------------
// stand-alone per-tile kernel: the tile's lists come from the map
// ---------------------------------------------------------------------------
// The saved-forward form keeps no per-entry forward state, so it fits 5
// blocks per SM (48 registers, a few spilled) and the extra resident warps
// hide its barrier waits; the recomputing form stays at 4 (64 registers).
template <int K, int MODE, bool SAVED = false>
__global__ void __launch_bounds__(kTileThreads, MODE == kModeStats ? 2 : (SAVED ? 5 : 4))
    k_bwd_tile(TileIO io, int cap, int H, int W, const uint4* __restrict__ map) {
  const uint32_t tiles_x = (W + kTileSide - 1) / kTileSide;
  TileCtx c;
  c.H = H;
  c.W = W;
  c.x0 = static_cast<int>(blockIdx.x % tiles_x) * kTileSide;
  c.y0 = static_cast<int>(blockIdx.x / tiles_x) * kTileSide;
  c.pix_off = 0;
  c.sr = SiteRange{0u, static_cast<uint32_t>(cap)};
  c.site_cum = 0u;
  c.tile = blockIdx.x;
  c.img = 0;
  c.two_over_P = 2.0f / static_cast<float>(static_cast<double>(H) * W);
  const int t = threadIdx.x;
  const int x = c.x0 + (t & (kTileSide - 1)), y = c.y0 + (t >> 4);
  const size_t P = static_cast<size_t>(H) * W;
  uint32_t ids[K];
#pragma unroll
  for (int j = 0; j < K / 4; ++j) {
    uint4 v = make_uint4(kInvalid, kInvalid, kInvalid, kInvalid);
    if (x < W && y < H) v = ldg(&map[j * P + static_cast<size_t>(y) * W + x]);
    ids[4 * j] = v.x;
    ids[4 * j + 1] = v.y;
    ids[4 * j + 2] = v.z;
    ids[4 * j + 3] = v.w;
  }
  float lk[K];  // unused without HAVE_L
#pragma unroll
  for (int k = 0; k < K; ++k) lk[k] = 0.f;
  __shared__ TileShared<K, MODE> sm;
  io.lists = map;
  io.lists_P = P;
  tile_body<K, MODE, false, kTileSide, SAVED>(c, io, ids, lk, sm);
}

// Chain rule from the ten statistics of a site to its 11 parameter gradients
// (through G(a, b, u) of Sec. 4.1); acc as in the records.
__device__ __forceinline__ void grads_from_stats(const float (&acc)[10], float4 gs, float4 ms,
                                                 float rawx, float rawy, float a, float b,
                                                 float (&out)[kNParams]) {
  const float ts = gs.z, r = gs.w;
  const float G00 = ms.x, G01 = ms.y, G11 = ms.z;
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
  out[PUX] = nrm2 > 0.f ? -gth * rawy / nrm2 : 0.f;
  out[PUY] = nrm2 > 0.f ? gth * rawx / nrm2 : 0.f;
}

// Per site (single image): the exact segment sums, then the chain rule.
__global__ void __launch_bounds__(kSumThreads) k_site_grads(const float* __restrict__ params, const float4* __restrict__ geo,
                             const float4* __restrict__ met, int cap,
                             const uint32_t* __restrict__ start, const uint32_t* __restrict__ boff,
                             const uint32_t* __restrict__ dir, const Record* __restrict__ rec,
                             const WsHeader* __restrict__ hdr, int L, float* __restrict__ grads) {
  __shared__ WarpSums<10> s_ws[kSumThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t c = static_cast<size_t>(cap);
  float acc[10];
  const uint32_t n = warp_site_sums<10, 2>(i < cap, static_cast<uint32_t>(i), static_cast<uint32_t>(cap), start, boff,
                                        dir, rec, hdr->pmax[0], L, s_ws[threadIdx.x >> 5], acc);  // every lane takes part
  if (i >= cap) return;
  float out[kNParams];
#pragma unroll
  for (int j = 0; j < kNParams; ++j) out[j] = 0.f;
  if (n)
    grads_from_stats(acc, geo[i], met[i], params[PUX * c + i], params[PUY * c + i],
                     params[PA * c + i], params[PB * c + i], out);
#pragma unroll
  for (int j = 0; j < kNParams; ++j) grads[j * c + i] = out[j];
}

// Per site: the exact segment sums of the statistics (statistics mode).
__global__ void __launch_bounds__(kSumThreads) k_site_stats(int cap, const uint32_t* __restrict__ start,
                             const uint32_t* __restrict__ boff, const uint32_t* __restrict__ dir,
                             const Record* __restrict__ rec, const WsHeader* __restrict__ hdr, int L,
                             float* __restrict__ stats) {
  __shared__ WarpSums<8> s_ws[kSumThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t c = static_cast<size_t>(cap);
  float acc[8];
  warp_site_sums<8>(i < cap, static_cast<uint32_t>(i), static_cast<uint32_t>(cap), start, boff, dir, rec,
                    hdr->pmax[0], L, s_ws[threadIdx.x >> 5], acc);  // every lane takes part
  if (i >= cap) return;
#pragma unroll
  for (int j = 0; j < 8; ++j) stats[j * c + i] = acc[j];
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
                        cudaStream_t st, const char* name, float* stats = nullptr,
                        const float* fwd = nullptr, const float* rgb_in = nullptr) {
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
    // per record: its 48 bytes and its directory entry; the two regions'
    // 256-byte alignment can hide up to 512 bytes, so start above and step down
    const uint64_t per = sizeof(Record) + sizeof(uint32_t) + sizeof(uint2);
    uint64_t mr = 1 + (ws_bytes - L1.total + 512) / per;
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
  uint2* place = reinterpret_cast<uint2*>(base + LL.place);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base + LL.cnt);
  uint32_t* start = reinterpret_cast<uint32_t*>(base + LL.start);
  uint32_t* bsums = reinterpret_cast<uint32_t*>(base + LL.bsums);
  uint32_t* dir = reinterpret_cast<uint32_t*>(base + LL.dir);

  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
  if (e == cudaSuccess && cap > 0) e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * static_cast<size_t>(cap), st);
  if (e != cudaSuccess) {
    set_error("%s memset: %s", name, cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  const float4* p4 = reinterpret_cast<const float4*>(prep);
  const float4 *geo = p4, *met = p4 + cap, *col = p4 + 2 * static_cast<size_t>(cap);
  const uint4* m4 = reinterpret_cast<const uint4*>(map);
  float* tl = (target && loss) ? tile_loss : nullptr;
  TileIO io;
  io.geo = geo;
  io.met = met;
  io.col = col;
  io.grad_rgb = grad_rgb;
  io.target = target;
  io.rgb_out = rgb_out;
  io.tile_loss = tl;
  io.records = rec;
  io.place = place;
  io.max_records = LL.max_records;
  io.hdr = hdr;
  io.site_cnt = cnt;
  io.fwd = fwd;
  io.rgb_in = rgb_in;
#define SAD_TILE_LAUNCH(KK, MM) \
  k_bwd_tile<KK, MM><<<LL.n_tiles, kTileThreads, 0, st>>>(io, cap, H, W, m4)
#define SAD_TILE_SAVED(KK) \
  k_bwd_tile<KK, kModeGrad, true><<<LL.n_tiles, kTileThreads, 0, st>>>(io, cap, H, W, m4)
  {
    TraceScope tr_(st, "k_bwd_tile");
    if (fwd) {
      switch (K) {
        case 4: SAD_TILE_SAVED(4); break;
        case 8: SAD_TILE_SAVED(8); break;
        default: SAD_TILE_SAVED(16); break;
      }
    } else if (stats_mode) {
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
  }
#undef SAD_TILE_LAUNCH
#undef SAD_TILE_SAVED
  if (int r = check_launch("k_bwd_tile")) return r;
  if (target && loss) {
    { TraceScope tr_(st, "k_loss_final"); k_loss_final<<<1, 256, 0, st>>>(tile_loss, LL.n_tiles, 1.0f / static_cast<float>(static_cast<double>(H) * W), loss); }
    if (int r = check_launch("k_loss_final")) return r;
  }
  if (cap == 0) return SAD_OK;
  // the segmented reduce: segment starts, records filed by site, exact sums
  run_seg_scan(cnt, static_cast<uint32_t>(cap), start, bsums, hdr, st);
  const int L = count_bits(LL.n_tiles);
  { TraceScope tr_(st, "k_rec_scatter"); k_rec_scatter<<<152 * 8, 256, 0, st>>>(place, hdr, LL.max_records, start, bsums, dir); }
  if (int r = check_launch("k_rec_scatter")) return r;
  if (stats_mode) {
    { TraceScope tr_(st, "k_site_stats"); k_site_stats<<<(cap + kSumThreads - 1) / kSumThreads, kSumThreads, 0, st>>>(cap, start, bsums, dir, rec, hdr, L, stats); }
    return check_launch("k_site_stats");
  }
  { TraceScope tr_(st, "k_site_grads"); k_site_grads<<<(cap + kSumThreads - 1) / kSumThreads, kSumThreads, 0, st>>>(params, geo, met, cap, start, bsums, dir, rec, hdr, L, grads); }
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

int64_t sad_backward_max_records(int32_t H, int32_t W, int32_t K, int32_t capacity) {
  if (H <= 0 || W <= 0 || capacity < 0 || (K != 4 && K != 8 && K != 16)) return -1;
  const int64_t n_tiles = static_cast<int64_t>((H + kTileSide - 1) / kTileSide) * ((W + kTileSide - 1) / kTileSide);
  const int64_t per_tile = static_cast<int64_t>(kTileThreads) * K;  // each pixel lists K entries
  return n_tiles * (per_tile < capacity ? per_tile : static_cast<int64_t>(capacity));
}

int sad_render_backward(const float* params, const float* prep, int32_t capacity, int32_t H,
                        int32_t W, int32_t K, const uint32_t* map, const float* grad_rgb,
                        float* grads, void* workspace, size_t workspace_bytes, void* stream) {
  if (!grad_rgb) return einval("sad_render_backward: null grad_rgb");
  return run_backward(params, prep, capacity, H, W, K, map, grad_rgb, nullptr, grads, nullptr,
                      nullptr, workspace, workspace_bytes, as_stream(stream), "sad_render_backward");
}

int sad_render_backward_saved(const float* params, const float* prep, int32_t capacity, int32_t H,
                              int32_t W, int32_t K, const uint32_t* map, const float* grad_rgb,
                              const float* rgb, const float* fwd, float* grads, void* workspace,
                              size_t workspace_bytes, void* stream) {
  if (!grad_rgb || !rgb || !fwd) return einval("sad_render_backward_saved: null grad_rgb, rgb or fwd");
  return run_backward(params, prep, capacity, H, W, K, map, grad_rgb, nullptr, grads, nullptr,
                      nullptr, workspace, workspace_bytes, as_stream(stream),
                      "sad_render_backward_saved", nullptr, fwd, rgb);
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
// first call before any stream capture).  The address is kept for the life
// of the process, so a device reset while the library is loaded is not
// supported.  All calls share the one buffer and
// it keeps the previous call's contents: every call clears the parts that
// must start at zero, and calls whose executions overlap on the GPU (two
// streams, or two threads) race on it and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace sad {

constexpr size_t kStaticScratchBytes = SAD_NOALLOC_SCRATCH_BYTES;  // 64 MiB
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
  { TraceScope tr_(as_stream(stream), "k_static_status"); k_static_status<<<1, 32, 0, as_stream(stream)>>>(reinterpret_cast<const WsHeader*>(scratch),
                                                   status_out); }
  return check_launch("k_static_status");
}
