// Adaptive budget: densify (split) and prune (Sec. 4.5; App. "Densification
// and Pruning"), from the per-site statistics of sad_site_stats.
//
//  - densify: among active sites with mass > mass_min and energy > 0, the
//    floor(pct N_active) largest s_i = E_i / max(m_i, eps)^alpha (ties to the
//    smaller id);
//  - prune: among the other active sites, the floor(pct N_active) smallest
//    removal deltas (ties to the smaller id);
//  - the k-th split parent (ascending id) keeps its slot for the '+' child and
//    takes the k-th inactive slot (ascending) for the '-' child; parents beyond
//    the free slots are left as they are;
//  - children: residual-weighted centroid and covariance from the moments,
//    split along the major axis with a = -log(l1/l2)/2 (u = axis), or, with
//    too little energy or an almost isotropic covariance, along the Sobel
//    gradient of the target with a = 0.8 a; offset clamp(0.5 sqrt(m), 1.5,
//    48) px each way, log_tau - 0.25, r * 0.85, colour = target at the child,
//    Adam state zeroed for both;
//  - every '-' child is written into the last list slot of the pixel that
//    contains it (the smallest id wins a pixel), so propagation spreads it.
// Selections use the deterministic radix select; no float atomics.
#include <cmath>

#include "sad_device.cuh"
#include "sad_host.h"
#include "sad_select.cuh"

namespace sad {

struct DpArgs {
  double densify_pct, prune_pct;
  float alpha, eps, mass_min, min_offset, max_offset, log_tau_shift, r_scale;
  float a_min, a_max, a_fallback_scale, energy_min, ratio_min;
};

struct DpState {
  uint32_t n_act, n_cand, n_active_after, n_dens;
  uint32_t pad[60];
  SelState sel_d;
  SelState sel_p;
};

struct DpLayout {
  size_t state, keys, flag_d, flag_p, scan, rank, freepos, freelist, bsums, claim, total;
  uint32_t nb;
};

static DpLayout dp_layout(int cap, int H, int W) {
  DpLayout L{};
  const size_t n = static_cast<size_t>(cap > 0 ? cap : 1);
  const size_t P = static_cast<size_t>(H) * W;
  L.nb = scan_blocks(n);
  auto al = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
  size_t o = 0;
  L.state = o;    o = al(o + sizeof(DpState));
  L.keys = o;     o = al(o + 4 * n);
  L.flag_d = o;   o = al(o + 4 * n);
  L.flag_p = o;   o = al(o + 4 * n);
  L.scan = o;     o = al(o + 4 * n);
  L.rank = o;     o = al(o + 4 * n);
  L.freepos = o;  o = al(o + 4 * n);
  L.freelist = o; o = al(o + 4 * n);
  L.bsums = o;    o = al(o + 4 * (L.nb + 2));
  L.claim = o;    o = al(o + 4 * P);
  L.total = o;
  return L;
}

__device__ __forceinline__ uint32_t orderable(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_dp_state(DpState* __restrict__ st) {
  uint32_t* w = reinterpret_cast<uint32_t*>(st);
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(DpState) / 4); i += blockDim.x) w[i] = 0u;
}

__global__ void k_dp_count(const float* __restrict__ params, const float* __restrict__ stats,
                           int cap, float mass_min, DpState* __restrict__ st,
                           uint32_t* __restrict__ inactive) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t act = 0, cand = 0;
  if (i < cap) {
    const size_t c = static_cast<size_t>(cap);
    act = params[PX * c + i] >= 0.f ? 1u : 0u;
    cand = (act && stats[0 * c + i] > mass_min && stats[1 * c + i] > 0.f) ? 1u : 0u;
    inactive[i] = act ? 0u : 1u;
  }
  const uint32_t a = __reduce_add_sync(0xffffffffu, act);
  const uint32_t b = __reduce_add_sync(0xffffffffu, cand);
  if ((threadIdx.x & 31) == 0) {
    if (a) atomicAdd(&st->n_act, a);
    if (b) atomicAdd(&st->n_cand, b);
  }
}

__global__ void k_dp_need_d(DpState* __restrict__ st, double pct) {
  if (threadIdx.x || blockIdx.x) return;
  const uint64_t want = static_cast<uint64_t>(floor(pct * static_cast<double>(st->n_act)));
  const uint32_t nd = static_cast<uint32_t>(want < st->n_cand ? want : st->n_cand);
  st->n_dens = nd;
  st->sel_d.need = nd;
}

__global__ void k_dp_need_p(DpState* __restrict__ st, double pct) {
  if (threadIdx.x || blockIdx.x) return;
  const uint64_t want = static_cast<uint64_t>(floor(pct * static_cast<double>(st->n_act)));
  const uint32_t rest = st->n_act - st->n_dens;
  st->sel_p.need = static_cast<uint32_t>(want < rest ? want : rest);
}

// densify keys: candidates ordered by score descending (smaller key first)
__global__ void k_dp_keys_d(const float* __restrict__ params, const float* __restrict__ stats,
                            int cap, DpArgs A, uint32_t* __restrict__ keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  const float mass = stats[0 * c + i], energy = stats[1 * c + i];
  const bool cand = params[PX * c + i] >= 0.f && mass > A.mass_min && energy > 0.f;
  const float score = energy / powf(fmaxf(mass, A.eps), A.alpha);
  keys[i] = cand ? ~__float_as_uint(score) : 0xffffffffu;
}

// prune keys: the other active sites by removal delta ascending
__global__ void k_dp_keys_p(const float* __restrict__ params, const float* __restrict__ stats,
                            const uint32_t* __restrict__ flag_d, int cap,
                            uint32_t* __restrict__ keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const size_t c = static_cast<size_t>(cap);
  const bool cand = params[PX * c + i] >= 0.f && !flag_d[i];
  keys[i] = cand ? orderable(stats[7 * c + i]) : 0xffffffffu;
}

__global__ void k_dp_freelist(const uint32_t* __restrict__ inactive,
                              const uint32_t* __restrict__ pos, int cap,
                              uint32_t* __restrict__ freelist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cap && inactive[i]) freelist[pos[i]] = static_cast<uint32_t>(i);
}

__device__ __forceinline__ float target_sum(const float* __restrict__ img, int W, int H, int r, int c) {
  r = r < 0 ? 0 : (r >= H ? H - 1 : r);
  c = c < 0 ? 0 : (c >= W ? W - 1 : c);
  const size_t q = (static_cast<size_t>(r) * W + c) * 3;
  return img[q] + img[q + 1] + img[q + 2];
}

__global__ void k_dp_split(float* __restrict__ params, float* __restrict__ m,
                           float* __restrict__ v, const float* __restrict__ stats,
                           const float* __restrict__ img, int cap, int H, int W,
                           const uint32_t* __restrict__ flag_d, const uint32_t* __restrict__ rank,
                           const uint32_t* __restrict__ freelist, const uint32_t* __restrict__ n_free,
                           uint32_t* __restrict__ claim, DpArgs A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap || !flag_d[i]) return;
  const uint32_t k = rank[i];
  if (k >= *n_free) return;
  const uint32_t j = freelist[k];
  const size_t c = static_cast<size_t>(cap);
  float p[kNParams];
#pragma unroll
  for (int q = 0; q < kNParams; ++q) p[q] = params[q * c + i];
  const float mass = stats[0 * c + i], S0 = stats[1 * c + i];
  bool use_cov = false;
  float ax = 1.f, ay = 0.f, cx = p[PX], cy = p[PY], a_new = A.a_fallback_scale * p[PA];
  if (S0 >= A.energy_min) {
    const float mux = stats[2 * c + i] / S0, muy = stats[3 * c + i] / S0;
    const float cxx = stats[4 * c + i] / S0 - mux * mux;
    const float cxy = stats[5 * c + i] / S0 - mux * muy;
    const float cyy = stats[6 * c + i] / S0 - muy * muy;
    const float tr = 0.5f * (cxx + cyy);
    const float dd = sqrtf(fmaxf(0.25f * (cxx - cyy) * (cxx - cyy) + cxy * cxy, 0.f));
    const float l1 = tr + dd, l2 = tr - dd;
    if (l1 > 0.f && l1 / fmaxf(l2, 1e-12f) >= A.ratio_min) {
      use_cov = true;
      // major eigenvector of [[cxx, cxy], [cxy, cyy]]
      float ex, ey;
      if (fabsf(cxy) > 1e-30f) {
        ex = l1 - cyy;
        ey = cxy;
      } else {
        ex = cxx >= cyy ? 1.f : 0.f;
        ey = cxx >= cyy ? 0.f : 1.f;
      }
      const float en = rsqrtf(ex * ex + ey * ey);
      ax = ex * en;
      ay = ey * en;
      if (ax < 0.f || (ax == 0.f && ay < 0.f)) {  // canonical sign: the '+' child lies at +x
        ax = -ax;
        ay = -ay;
      }
      cx = p[PX] + mux;
      cy = p[PY] + muy;
      a_new = fminf(fmaxf(-0.5f * logf(l1 / fmaxf(l2, 1e-12f)), A.a_min), A.a_max);
    }
  }
  if (!use_cov) {
    const int col = min(max(static_cast<int>(floorf(p[PX])), 0), W - 1);
    const int row = min(max(static_cast<int>(floorf(p[PY])), 0), H - 1);
    const float gx = target_sum(img, W, H, row - 1, col + 1) + 2.f * target_sum(img, W, H, row, col + 1) +
                     target_sum(img, W, H, row + 1, col + 1) - target_sum(img, W, H, row - 1, col - 1) -
                     2.f * target_sum(img, W, H, row, col - 1) - target_sum(img, W, H, row + 1, col - 1);
    const float gy = target_sum(img, W, H, row + 1, col - 1) + 2.f * target_sum(img, W, H, row + 1, col) +
                     target_sum(img, W, H, row + 1, col + 1) - target_sum(img, W, H, row - 1, col - 1) -
                     2.f * target_sum(img, W, H, row - 1, col) - target_sum(img, W, H, row - 1, col + 1);
    const float gn = sqrtf(gx * gx + gy * gy);
    if (gn > 0.f) {
      ax = gx / gn;
      ay = gy / gn;
    }
  }
  const float d = fminf(fmaxf(0.5f * sqrtf(fmaxf(mass, 0.f)), A.min_offset), A.max_offset);
#pragma unroll
  for (int sgn = 0; sgn < 2; ++sgn) {
    const float sg = sgn == 0 ? 1.f : -1.f;
    const uint32_t dst = sgn == 0 ? static_cast<uint32_t>(i) : j;
    float q[kNParams];
#pragma unroll
    for (int t = 0; t < kNParams; ++t) q[t] = p[t];
    q[PX] = fminf(fmaxf(cx + sg * d * ax, 0.f), static_cast<float>(W));
    q[PY] = fminf(fmaxf(cy + sg * d * ay, 0.f), static_cast<float>(H));
    q[PLOGTAU] = p[PLOGTAU] + A.log_tau_shift;
    q[PR] = p[PR] * A.r_scale;
    q[PA] = a_new;
    if (use_cov) {
      q[PUX] = ax;
      q[PUY] = ay;
    }
    const int cc = min(max(static_cast<int>(floorf(q[PX])), 0), W - 1);
    const int rr = min(max(static_cast<int>(floorf(q[PY])), 0), H - 1);
    const size_t pix = static_cast<size_t>(rr) * W + cc;
    q[PCR] = img[3 * pix];
    q[PCG] = img[3 * pix + 1];
    q[PCB] = img[3 * pix + 2];
#pragma unroll
    for (int t = 0; t < kNParams; ++t) {
      params[t * c + dst] = q[t];
      m[t * c + dst] = 0.f;
      v[t * c + dst] = 0.f;
    }
    if (sgn == 1 && claim) atomicMin(&claim[pix], j);
  }
}

__global__ void k_dp_prune(float* __restrict__ params, const uint32_t* __restrict__ flag_p, int cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap || !flag_p[i]) return;
  const size_t c = static_cast<size_t>(cap);
  params[PX * c + i] = -1.f;
  params[PY * c + i] = -1.f;
}

__global__ void k_dp_seed_map(const uint32_t* __restrict__ claim, size_t P, int K,
                              uint32_t* __restrict__ map) {
  const size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= P || claim[q] == kInvalid) return;
  map[(static_cast<size_t>(K / 4 - 1) * P + q) * 4 + 3] = claim[q];
}

__global__ void k_dp_count_after(const float* __restrict__ params, int cap,
                                 DpState* __restrict__ st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t act = (i < cap && params[i] >= 0.f) ? 1u : 0u;
  const uint32_t a = __reduce_add_sync(0xffffffffu, act);
  if ((threadIdx.x & 31) == 0 && a) atomicAdd(&st->n_active_after, a);
}

}  // namespace sad

using namespace sad;

extern "C" {

size_t sad_densify_workspace_bytes(int32_t capacity, int32_t H, int32_t W) {
  if (capacity < 0 || H <= 0 || W <= 0) return 0;
  return dp_layout(capacity, H, W).total;
}

// The whole densify/prune event on the stream; the active count after it is
// left in the workspace's state page (*after_out points there) and, if
// n_active_dev is given, copied to that device int32.  Nothing synchronises.
static int dp_run(float* params, float* m, float* v, int32_t capacity, int32_t H, int32_t W,
                  int32_t K, const float* stats, const float* target, uint32_t* map,
                  const sad_dp_params* dp, int32_t* n_active_dev, void* workspace,
                  size_t workspace_bytes, void* stream, const uint32_t** after_out) {
  if (int e = check_problem(capacity, H, W, K, map != nullptr)) return e;
  if (!dp) return einval("sad_densify_prune: null parameters");
  if (capacity > 0 && (!params || !m || !v || !stats || !target))
    return einval("sad_densify_prune: null pointer");
  if (!(dp->densify_pct >= 0.0 && dp->densify_pct <= 1.0 && dp->prune_pct >= 0.0 &&
        dp->prune_pct <= 1.0))
    return einval("sad_densify_prune: percentiles must be in [0,1]");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return einval("sad_densify_prune: workspace must be 256-byte aligned");
  const DpLayout L = dp_layout(capacity, H, W);
  if (!workspace || workspace_bytes < L.total) {
    set_error("sad_densify_prune: workspace has %zu bytes, needs %zu", workspace_bytes, L.total);
    return SAD_EWORKSPACE;
  }
  cudaStream_t st = as_stream(stream);
  if (capacity == 0) {
    *after_out = nullptr;
    if (n_active_dev) {
      const cudaError_t e = cudaMemsetAsync(n_active_dev, 0, sizeof(int32_t), st);
      if (e != cudaSuccess) {
        set_error("sad_densify_prune: %s", cudaGetErrorString(e));
        return SAD_ECUDA;
      }
    }
    return SAD_OK;
  }
  char* base = static_cast<char*>(workspace);
  DpState* S = reinterpret_cast<DpState*>(base + L.state);
  uint32_t* keys = reinterpret_cast<uint32_t*>(base + L.keys);
  uint32_t* flag_d = reinterpret_cast<uint32_t*>(base + L.flag_d);
  uint32_t* flag_p = reinterpret_cast<uint32_t*>(base + L.flag_p);
  uint32_t* scan = reinterpret_cast<uint32_t*>(base + L.scan);
  uint32_t* rank = reinterpret_cast<uint32_t*>(base + L.rank);
  uint32_t* freepos = reinterpret_cast<uint32_t*>(base + L.freepos);
  uint32_t* freelist = reinterpret_cast<uint32_t*>(base + L.freelist);
  uint32_t* bsums = reinterpret_cast<uint32_t*>(base + L.bsums);
  uint32_t* claim = reinterpret_cast<uint32_t*>(base + L.claim);
  const size_t n = static_cast<size_t>(capacity);
  const size_t P = static_cast<size_t>(H) * W;
  DpArgs A;
  A.densify_pct = dp->densify_pct;
  A.prune_pct = dp->prune_pct;
  A.alpha = dp->alpha;
  A.eps = dp->eps;
  A.mass_min = dp->mass_min;
  A.min_offset = dp->min_offset;
  A.max_offset = dp->max_offset;
  A.log_tau_shift = dp->log_tau_shift;
  A.r_scale = dp->r_scale;
  A.a_min = dp->a_min;
  A.a_max = dp->a_max;
  A.a_fallback_scale = dp->a_fallback_scale;
  A.energy_min = dp->energy_min;
  A.ratio_min = dp->ratio_min;
  const unsigned gs = static_cast<unsigned>((n + 255) / 256);
  const unsigned gp = static_cast<unsigned>((P + 255) / 256);
  { TraceScope tr_(st, "k_dp_state"); k_dp_state<<<1, 256, 0, st>>>(S); }
  // inactive flags go to flag_p for now (reused after the free list is built)
  { TraceScope tr_(st, "k_dp_count"); k_dp_count<<<gs, 256, 0, st>>>(params, stats, capacity, A.mass_min, S, flag_p); }
  run_xscan(flag_p, freepos, n, bsums, st);
  { TraceScope tr_(st, "k_dp_freelist"); k_dp_freelist<<<gs, 256, 0, st>>>(flag_p, freepos, capacity, freelist); }
  // the number of free slots: total of that scan
  uint32_t* n_free = bsums + scan_blocks(n);
  // keep the count in the state page (bsums is reused by later scans)
  uint32_t* n_free_keep = &S->pad[0];
  cudaError_t e = cudaMemcpyAsync(n_free_keep, n_free, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    set_error("sad_densify_prune: %s", cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  { TraceScope tr_(st, "k_dp_need_d"); k_dp_need_d<<<1, 32, 0, st>>>(S, A.densify_pct); }
  { TraceScope tr_(st, "k_dp_keys_d"); k_dp_keys_d<<<gs, 256, 0, st>>>(params, stats, capacity, A, keys); }
  run_select_smallest(keys, n, &S->sel_d, flag_d, scan, bsums, st);
  { TraceScope tr_(st, "k_dp_need_p"); k_dp_need_p<<<1, 32, 0, st>>>(S, A.prune_pct); }
  { TraceScope tr_(st, "k_dp_keys_p"); k_dp_keys_p<<<gs, 256, 0, st>>>(params, stats, flag_d, capacity, keys); }
  run_select_smallest(keys, n, &S->sel_p, flag_p, scan, bsums, st);
  run_xscan(flag_d, rank, n, bsums, st);
  if (map) {
    e = cudaMemsetAsync(claim, 0xff, 4 * P, st);
    if (e != cudaSuccess) {
      set_error("sad_densify_prune: %s", cudaGetErrorString(e));
      return SAD_ECUDA;
    }
  }
  { TraceScope tr_(st, "k_dp_split"); k_dp_split<<<gs, 256, 0, st>>>(params, m, v, stats, target, capacity, H, W, flag_d, rank, freelist,
                                 n_free_keep, map ? claim : nullptr, A); }
  { TraceScope tr_(st, "k_dp_prune"); k_dp_prune<<<gs, 256, 0, st>>>(params, flag_p, capacity); }
  if (map) { TraceScope tr_(st, "k_dp_seed_map"); k_dp_seed_map<<<gp, 256, 0, st>>>(claim, P, K, map); }
  { TraceScope tr_(st, "k_dp_count_after"); k_dp_count_after<<<gs, 256, 0, st>>>(params, capacity, S); }
  if (int r = check_launch("sad_densify_prune")) return r;
  *after_out = &S->n_active_after;
  if (n_active_dev) {
    e = cudaMemcpyAsync(n_active_dev, &S->n_active_after, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      set_error("sad_densify_prune: %s", cudaGetErrorString(e));
      return SAD_ECUDA;
    }
  }
  return SAD_OK;
}

int sad_densify_prune(float* params, float* m, float* v, int32_t capacity, int32_t H, int32_t W,
                      int32_t K, const float* stats, const float* target, uint32_t* map,
                      const sad_dp_params* dp, int32_t* n_active_out, void* workspace,
                      size_t workspace_bytes, void* stream) {
  if (!n_active_out) return einval("sad_densify_prune: null output");
  const uint32_t* after_dev = nullptr;
  if (int r = dp_run(params, m, v, capacity, H, W, K, stats, target, map, dp, nullptr, workspace,
                     workspace_bytes, stream, &after_dev))
    return r;
  if (!after_dev) {
    *n_active_out = 0;
    return SAD_OK;
  }
  cudaStream_t st = as_stream(stream);
  uint32_t after = 0;
  cudaError_t e = cudaMemcpyAsync(&after, after_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error("sad_densify_prune: %s", cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  *n_active_out = static_cast<int32_t>(after);
  return SAD_OK;
}

int sad_densify_prune_async(float* params, float* m, float* v, int32_t capacity, int32_t H, int32_t W,
                            int32_t K, const float* stats, const float* target, uint32_t* map,
                            const sad_dp_params* dp, int32_t* n_active_dev, void* workspace,
                            size_t workspace_bytes, void* stream) {
  if (!n_active_dev) return einval("sad_densify_prune_async: null output");
  if ((reinterpret_cast<uintptr_t>(n_active_dev) & 3u) != 0)
    return einval("sad_densify_prune_async: misaligned output");
  const uint32_t* after_dev = nullptr;
  return dp_run(params, m, v, capacity, H, W, K, stats, target, map, dp, n_active_dev, workspace,
                workspace_bytes, stream, &after_dev);
}

}  // extern "C"
