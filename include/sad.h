/*
 * sad.h -- C-ABI of libsad.so, the GB300 (sm_103a) hot path of Soft
 * Anisotropic Diagrams (SAD, arXiv 2604.21984).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - All array arguments are DEVICE pointers unless stated otherwise; the
 *    caller allocates and owns them (including workspaces).  The library never
 *    allocates device memory, never frees caller memory and does not keep any
 *    pointer after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous on that stream unless stated otherwise.
 *  - Return value: a sad_status code (int).  Argument errors are detected on
 *    the host before any launch and return SAD_EINVAL; a failed launch returns
 *    SAD_ECUDA.  sad_last_error() gives a thread-local message for the last
 *    failure on the calling thread.
 *  - Site parameters are float32[11][capacity] planes in the order
 *      0 x  1 y  2 log_tau  3 r  4 cr  5 cg  6 cb  7 ux  8 uy  9 a  10 b
 *    (Sec. 4.1 "Site Representation": position, temperature, additive radius,
 *    colour, anisotropy direction u (stored unnormalised), log-anisotropy a;
 *    b is a per-site log isotropic metric scale, b = 0 being the paper's
 *    unit-determinant metric).  Positions and radii are in pixels; pixel
 *    (col,row) has its centre at (col+0.5, row+0.5).  A site with x < 0 is
 *    inactive (App. "Data Layout and Packing", Site buffer) and is skipped by every kernel.
 *  - The top-K map is K/4 planes of uint32x4 (App. "Data Layout and Packing", Top-K candidate
 *    list): plane j holds, for every pixel in row-major order, the ids of
 *    list positions 4j..4j+3, i.e. uint32[K/4][H*W][4].  Sentinel 0xffffffff.
 *    K must be 4, 8 or 16.  Lists are ordered by logit descending, ties by
 *    smaller id (for maps produced by sad_update_topk).
 *  - The prepared site table (the "pack" of App. "Data Layout and Packing") is float32[6][capacity][4]:
 *      plane 0 {x, y, tau*s, r}, plane 1 {G00, G01, G11, active},
 *      plane 2 {cr, cg, cb, 0},  with s = 1/max(H,W) (Sec. 4.1); planes 3
 *      and 4 hold the same site folded for the softmax blend (the blend
 *      record): with G' = (tau s)^2 G, plane 3 {x, y, tau s r, G'00} (tau s r
 *      = -inf for an inactive site), plane 4 {G'01, G'11, cr, cg}; plane 5
 *      holds cb densely, one float per site (float32[capacity] at the start
 *      of the plane; the rest of the plane is unused).
 *    Every device pointer must be 16-byte aligned.
 */
#ifndef SAD_H
#define SAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SAD_OK = 0,
  SAD_EINVAL = 1,     /* bad argument (size, alignment, null pointer, K) */
  SAD_ECUDA = 2,      /* a CUDA launch or copy failed */
  SAD_EWORKSPACE = 3, /* workspace too small (detected on the host) */
  SAD_ETIMEOUT = 4,   /* reserved: a bounded device wait gave up */
  SAD_EINTERNAL = 5
};

#define SAD_NPARAMS 11
#define SAD_INVALID_ID 0xffffffffu

/* Static string for a status code; never freed. */
const char* sad_status_string(int status);
/* Thread-local detail message of the last failing call on this thread. */
const char* sad_last_error(void);
/* ABI version of this header (bumped on any signature change). */
int sad_abi_version(void);

/*
 * Stage tracing (library addition with no counterpart in the paper: the
 * measurement side of the kernels).  While on, every kernel launch of the
 * library is bracketed by two CUDA events on its stream (not on a stream
 * being captured into a graph).  sad_trace_enable returns the previous
 * setting.  sad_trace_collect waits for the recorded events, aggregates
 * them per stage (kernel name) since the last collect, writes up to
 * max_entries entries (out: HOST array) and the number of stages to *n_out,
 * and forgets the records.  At most 65536 launches are kept between collects.
 */
typedef struct sad_trace_entry {
  char name[48];      /* kernel (stage) name */
  int64_t launches;   /* launches recorded */
  double total_ms;    /* sum of their event-to-event device times */
} sad_trace_entry;
int sad_trace_enable(int on);
int sad_trace_collect(sad_trace_entry* out, int32_t max_entries, int32_t* n_out);

/*
 * sad_prepare_sites -- per-site derived table ("pack", App. "Data Layout and Packing"; metric G of
 * Sec. 4.1).  For every site i < capacity, in float32 with each operation
 * separately rounded (no fused multiply-add):
 *   s = 1/max(H,W); u = (ux,uy)/|(ux,uy)| (or (1,0) if zero);
 *   e+ = exp(b+a), e- = exp(b-a) with a reproducible exponential (Cody-Waite
 *   reduction + degree-7 Taylor polynomial); G00 = e+ ux^2 + e- uy^2,
 *   G01 = (e+ - e-) ux uy, G11 = e+ uy^2 + e- ux^2; tau*s = exp(log_tau) s;
 *   active = (x >= 0).
 * params: float32[11][capacity] (read).  prep: float32[6][capacity][4] (written).
 */
int sad_prepare_sites(const float* params, int32_t capacity, int32_t H, int32_t W,
                      float* prep, void* stream);

/*
 * sad_topk_seed -- seed pass of the JFA prepass (App. "Candidate Field and Jump Schedule", JFA prepass).
 * Fills the whole map with the sentinel, then every active site writes its id
 * into list position 0 of the pixel that contains it (floor of its position,
 * clamped to the image); on collisions the smallest id wins (deterministic).
 * map: uint32[K/4][H*W][4] (written).
 */
int sad_topk_seed(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                  uint32_t* map, void* stream);

/*
 * sad_jfa_flood -- one flood pass of the JFA prepass (App. "Candidate Field
 * and Jump Schedule", JFA prepass): every pixel pools slots 0..3 (the first
 * candidate plane) of the lists of the 3x3 pixels at offsets {-s, 0, s}^2
 * around it, itself included (s = step_code >> 16; outside pixels skipped),
 * drops invalid / inactive / NaN entries and duplicates, and writes the 4
 * best by (logit descending, id ascending) -- the R2/R13 order and fp32
 * score of sad_update_topk -- into its slots 0..3; the other planes are
 * copied.  No injection.  A full refresh is sad_topk_seed, ceil(log2
 * max(W, H)) flood passes at the jump schedule, then propagation passes.
 * map_in / map_out: K/4 uint4 planes, must not overlap.
 */
int sad_jfa_flood(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                  const uint32_t* map_in, uint32_t* map_out, uint32_t step_code, void* stream);

/*
 * sad_update_topk -- one propagation pass of the per-pixel top-K field
 * (Sec. 4.3, update C_t = topK over C_{t-1} U P_t U G_t).  Pool of pixel x:
 * its own list in map_in, the lists of the 4 neighbours at (+-s,0), (0,+-s)
 * (s = step_code >> 16; neighbours outside the image are skipped), and
 * n_inject ids drawn from SplitMix64 (Steele et al. 2014) at counter
 * ((step_code << 32) | (pixel*n_inject + j)) with `seed`, mapped to
 * [0,capacity) by (hi32 * capacity) >> 32.  Invalid, inactive and NaN-scored
 * candidates are dropped, duplicates collapse, and the K best by
 * (logit descending, id ascending) are written to map_out (sentinel tail).
 * Logits are computed in float32 without contraction:
 *   dx = px-x, dy = py-y, q = ((G00 dx)dx + 2((G01 dx)dy)) + (G11 dy)dy,
 *   n = sqrt(max(q,0)), l = (tau s)(r - n).
 * step_code: low 16 bits = pass index, high 16 bits = jump (App. "Candidate Field and Jump Schedule", Step
 * encoding).  map_in and map_out must not overlap (Jacobi update).
 * Requires H*W*n_inject < 2^32 and 0 <= n_inject <= 16.
 */
int sad_update_topk(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                    const uint32_t* map_in, uint32_t* map_out, uint32_t step_code,
                    int32_t n_inject, uint64_t seed, void* stream);

/*
 * sad_exact_topk -- the exact top-K of sampled pixels by brute force over
 * every site: the set that the propagation of Sec. 4.3 approximates, for
 * measuring the recall and exact-match fraction of a propagated map (Sec. 6.5,
 * Table "Top-K propagation convergence").  Each pixel scores all `capacity`
 * sites with the fp32 score of sad_update_topk (same operation order, inactive
 * and NaN-scored sites dropped) and keeps the K best by (logit descending, id
 * ascending), so a propagated list that has converged equals it bit for bit.
 * pixels: int64[n] pixel indices (row * W + col, each in [0, H*W)), 8-byte
 * aligned; ids_out: uint32[n][K] (sentinel 0xffffffff past the active count).
 * One 256-thread block per pixel: O(n * capacity) work, a measurement tool,
 * not a hot-path call.  Requires 0 <= n < 2^31.
 */
int sad_exact_topk(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                   const int64_t* pixels, int64_t n, uint32_t* ids_out, void* stream);

/*
 * Half2 candidate sites (App. "Data Layout and Packing", Packed candidate
 * sites): a 16-byte per-site record that candidate passes read instead of
 * the prepared table's two 16-byte scoring planes.
 * sad_pack_candidates -- cand: uint32[capacity][4] (written), words
 *   {x, y}, {tau s, r}, {G00, G01}, {G11, active} of the prepared table
 *   `prep`, each word a half2 with the first value in the low 16 bits.
 *   Each value is saturated to [-65504, 65504] (fminf/fmaxf semantics)
 *   and rounded to the nearest half, ties to even.  Regenerate it whenever
 *   the prepared table changes.
 * sad_update_topk_h2 -- sad_update_topk with every candidate scored from
 *   `cand` (the halves widened to float32 exactly, then the same float32
 *   logit).  Lists are ordered by these logits; the render and the adjoint
 *   still take the float32 table.
 * cand must be 16-byte aligned; errors as sad_update_topk.
 */
int sad_pack_candidates(const float* prep, int32_t capacity, uint32_t* cand, void* stream);
int sad_update_topk_h2(const uint32_t* cand, int32_t capacity, int32_t H, int32_t W, int32_t K,
                       const uint32_t* map_in, uint32_t* map_out, uint32_t step_code,
                       int32_t n_inject, uint64_t seed, void* stream);

/*
 * Downscaled candidate grid (App. "Candidate Field and Jump Schedule",
 * Downscaled candidate grid): the lists live on a ceil(H/s) x ceil(W/s)
 * grid of s x s pixel cells, and a cell's candidates are scored at its
 * centre ((col + 0.5) s, (row + 0.5) s) in image pixels; pixels map to cells
 * by integer division (no interpolation).  H, W: the image; s_grid in
 * [1, 64]; grid maps are K/4 uint4 planes over the cells.
 * sad_grid_seed   -- sad_topk_seed onto the grid (a site's clamped pixel's cell).
 * sad_grid_update -- sad_update_topk over the cells (jumps, injection counters
 *                    and the jump schedule are in cells).
 * sad_grid_expand -- per-pixel map (K/4 planes over H*W) from the grid, for
 *                    the render, adjoint and statistics calls.
 * s_grid = 1 reproduces sad_topk_seed / sad_update_topk exactly.
 */
int sad_grid_seed(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t s_grid,
                  int32_t K, uint32_t* map, void* stream);
int sad_grid_update(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t s_grid,
                    int32_t K, const uint32_t* map_in, uint32_t* map_out, uint32_t step_code,
                    int32_t n_inject, uint64_t seed, void* stream);
int sad_grid_expand(const uint32_t* map_grid, int32_t H, int32_t W, int32_t s_grid, int32_t K,
                    uint32_t* map_pixels, void* stream);

/*
 * sad_render -- soft anisotropic additively weighted render (Sec. 4.2):
 * c(x) = sum_i w_i(x) c_i, w = softmax over the listed sites of
 * l_i(x) = -tau_i d_mix(x,i) (max-subtracted).  Pixels whose list holds no
 * valid active site render black.  rgb: float32[H][W][3] (written).
 */
int sad_render(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
               const uint32_t* map, float* rgb, void* stream);

/*
 * sad_render_save -- sad_render that also keeps, per pixel, what the adjoint
 * needs of the forward: fwd = float32[2][H*W] planes {max listed logit m,
 * 1/Z} with Z = sum_i exp(l_i - m) (both 0 for a black pixel).  Together
 * with rgb (the blend) they let sad_render_backward_saved skip recomputing
 * each pixel's softmax normaliser; no per-(pixel, site) weight is stored.
 * rgb is the same as sad_render's, bit for bit.
 */
int sad_render_save(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                    const uint32_t* map, float* rgb, float* fwd, void* stream);

/*
 * sad_decode_points -- random-access decode at float coordinates (the
 * render-only path with cached top-K lists, Sec. 6.6).  Query (x,y) uses the
 * list of pixel (clamp(floor x), clamp(floor y)) and evaluates the blend of
 * Sec. 4.2 at (x,y) itself.  xy: float32[n][2]; rgb: float32[n][3].
 */
int sad_decode_points(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                      const uint32_t* map, const float* xy, int64_t n, float* rgb,
                      void* stream);

/*
 * Workspace of sad_render_backward / sad_train_grads, in bytes, for a problem
 * of H x W pixels, list size K and `capacity` sites, able to hold
 * `max_records` per-tile partial records (0 = default H*W*K/8, at least
 * 128 per 16x16 tile).  The caller allocates it (any content; 256-B aligned).
 */
size_t sad_backward_workspace_bytes(int32_t H, int32_t W, int32_t K, int32_t capacity,
                                    int64_t max_records);

/*
 * The most per-tile partial records that sad_render_backward /
 * sad_render_backward_saved / sad_train_grads can produce for ANY top-K map
 * of an H x W, list size K, `capacity`-site problem: one record per 16x16
 * tile and distinct site listed in it, so n_tiles * min(256 K, capacity)
 * with n_tiles = ceil(H/16) ceil(W/16).  A workspace of
 * sad_backward_workspace_bytes(H, W, K, capacity, this bound) never
 * overflows, so its caller needs no sad_workspace_status read (a bound
 * above 2^32 - 16 cannot be held by one workspace).  Returns -1 for an
 * invalid problem (H or W <= 0, capacity < 0, K not 4, 8 or 16).
 */
int64_t sad_backward_max_records(int32_t H, int32_t W, int32_t K, int32_t capacity);

/*
 * sad_render_backward -- adjoint of sad_render into every site parameter
 * (App. "Gradient Computation and Reduction", Per-pixel gradients), with the top-K map a frozen index set.
 * Per pixel the softmax is recomputed (nothing from the forward is stored);
 * per 16x16 tile the contributions are reduced per site in a fixed order
 * (per-tile partials, no float atomics; replaces the tile hash + global float
 * atomics of Sec. 4.8), then a segmented reduce sums each site's partials in
 * exact 64-bit fixed point (no atomics on the values: integer sums, order
 * independent).  Bitwise reproducible run to run.
 * grad_rgb: float32[H][W][3] = dL/dc.  grads: float32[11][capacity], fully
 * written (zero for sites no pixel lists).  params/prep must describe the
 * same sites.  If more partial records are produced than the workspace holds,
 * the gradients are incomplete and sad_workspace_status reports it.
 */
int sad_render_backward(const float* params, const float* prep, int32_t capacity, int32_t H,
                        int32_t W, int32_t K, const uint32_t* map, const float* grad_rgb,
                        float* grads, void* workspace, size_t workspace_bytes, void* stream);

/*
 * sad_render_backward_saved -- sad_render_backward from the forward that
 * sad_render_save kept: rgb (its output) and fwd (its {m, 1/Z} planes), for
 * the same prep and map.  Each (pixel, site) weight is recomputed from its
 * logit and the pixel's m and 1/Z; the per-tile reduction, the exact sums and
 * the result are as in sad_render_backward (equal up to float rounding).
 * Listed inactive sites get zero weight.
 */
int sad_render_backward_saved(const float* params, const float* prep, int32_t capacity, int32_t H,
                              int32_t W, int32_t K, const uint32_t* map, const float* grad_rgb,
                              const float* rgb, const float* fwd, float* grads, void* workspace,
                              size_t workspace_bytes, void* stream);

/*
 * sad_train_grads -- fused training gradient (Sec. 6.1): renders, forms the
 * MSE loss L = (1/P) sum_x |c(x) - I(x)|^2 against target float32[H][W][3],
 * and back-propagates g = 2(c - I)/P exactly as sad_render_backward does.
 * loss: device float32[1] (written, deterministic); rgb_out may be NULL or
 * float32[H][W][3] to also receive the render.
 */
int sad_train_grads(const float* params, const float* prep, int32_t capacity, int32_t H,
                    int32_t W, int32_t K, const uint32_t* map, const float* target,
                    float* grads, float* loss, float* rgb_out, void* workspace,
                    size_t workspace_bytes, void* stream);

/*
 * sad_render_backward_noalloc -- the same computation as sad_render_backward
 * for callers that cannot allocate device memory for a workspace (they only
 * hold device pointers handed to them, or run where an allocation is not
 * allowed).  The paper has no counterpart; it is a deployment convenience.
 * Scratch is one SAD_NOALLOC_SCRATCH_BYTES buffer inside the library
 * (allocated on every device that loads the library, kept until exit).
 * Limits: H*W <= 4194304 and capacity <= 262144, else SAD_EINVAL; within them
 * about 1.0 million per-tile records fit (a 2048 x 2048 render of 262144
 * random sites at K = 16 makes about 0.83 million; spatially incoherent lists
 * make many more and overflow).  The first call on a device looks up the
 * buffer's device address and keeps it for the life of the process (make that
 * call before any stream capture; a device reset while the library is loaded
 * is not supported).  All calls share the buffer: calls that overlap on the
 * GPU race and must be serialised by the caller.  status_out (device int32)
 * receives SAD_OK, or SAD_EWORKSPACE if the records did not fit (gradients
 * then incomplete).  status_out may be NULL, but then an overflow is not
 * reported anywhere: pass it unless the problem is known to fit.
 * Allocates nothing.
 */
#define SAD_NOALLOC_SCRATCH_BYTES (64ull << 20)
int sad_render_backward_noalloc(const float* params, const float* prep, int32_t capacity,
                                int32_t H, int32_t W, int32_t K, const uint32_t* map,
                                const float* grad_rgb, float* grads, int32_t* status_out,
                                void* stream);

/*
 * Reads the workspace status word of the last backward call on `stream`
 * (synchronises the stream).  *records_used receives the number of partial
 * records written; returns SAD_EWORKSPACE if they overflowed the workspace.
 */
int sad_workspace_status(const void* workspace, int64_t* records_used, void* stream);

/*
 * sad_init_sites -- gradient-weighted initialisation (Sec. 4.4, Eq. P_init).
 * P_init(x) = (1-lambda) |grad I(x)| / sum |grad I| + lambda/(H W), with
 * |grad I| the 2-norm over RGB of central differences (one-sided at the
 * borders); the normaliser is summed exactly in 2^-32 fixed point.  n pixels
 * are drawn without replacement by Efraimidis-Spirakis keys E/P_init,
 * E = -log U with U the 24-bit SplitMix64 draw of `seed` at counter = pixel
 * index (the n smallest keys, ties to the smaller index); site i (in pixel
 * order) sits at the pixel centre plus a U[-0.25,0.25) jitter per axis
 * (draws at counters 2^40 + 2 pixel + {0,1}), takes the image colour there,
 * log_tau = log_tau0, r = 0, u = (1,0), a = b = 0.  Sites n..capacity-1 are
 * set inactive.  Deterministic; fp32 steps are explicitly rounded.
 * img: float32[H][W][3]; params: float32[11][capacity] (written).
 * workspace: sad_init_workspace_bytes(H, W) bytes, 256-B aligned.
 * Requires 0 <= n <= min(capacity, H*W), 0 <= lambda_init <= 1.
 */
size_t sad_init_workspace_bytes(int32_t H, int32_t W);
int sad_init_sites(const float* img, int32_t H, int32_t W, int32_t n, int32_t capacity,
                   float lambda_init, uint64_t seed, float log_tau0, float* params,
                   void* workspace, size_t workspace_bytes, void* stream);

/*
 * sad_site_stats -- per-site statistics of one render for the adaptive
 * budget (Sec. 4.5; App. "Densification and Pruning", densification scores
 * and pruning): float32[8][capacity] planes
 *   0 mass    m_i = sum_x w_i(x)
 *   1 energy  E_i = sum_x w_i(x) |c(x) - I(x)|^2
 *   2..6      sum omega Dx, sum omega Dy, sum omega Dx^2, sum omega Dx Dy,
 *             sum omega Dy^2 with omega = w_i(x) |c(x) - I(x)|^2 and
 *             D = x - p_i (pixel centre minus site position, pixels)
 *   7 removal sum_x of |c'(x) - I(x)|^2 - |c(x) - I(x)|^2, c' the blend
 *             without site i (Sec. 4.5 removal delta; black if i was alone)
 * Same deterministic per-tile reduction and workspace as sad_render_backward.
 */
int sad_site_stats(const float* prep, int32_t capacity, int32_t H, int32_t W, int32_t K,
                   const uint32_t* map, const float* target, float* stats, void* workspace,
                   size_t workspace_bytes, void* stream);

/* Densify/prune parameters (Sec. 4.5; Sec. 6.1 defaults in brackets). */
typedef struct sad_dp_params {
  double densify_pct;      /* fraction of active sites split [0.01] */
  double prune_pct;        /* fraction of active sites pruned [0.033] */
  float alpha;             /* score exponent [0.7] */
  float eps;               /* mass floor in the score [1e-8] */
  float mass_min;          /* sites with mass <= this are not split [1] */
  float min_offset, max_offset; /* child offset clamp, px [1.5, 48] */
  float log_tau_shift;     /* added to log_tau of children [-0.25] */
  float r_scale;           /* r multiplier of children [0.85] */
  float a_min, a_max;      /* clamp of a from the covariance [-2, 2] */
  float a_fallback_scale;  /* a multiplier without statistics [0.8] */
  float energy_min;        /* below: no covariance (fallback) [1e-6] */
  float ratio_min;         /* eigenvalue ratio below: fallback [1.01] */
} sad_dp_params;

/*
 * sad_densify_prune -- one densify-then-prune event (Sec. 4.5) from
 * sad_site_stats output: split the floor(densify_pct N_active) sites with the
 * largest E/max(m,eps)^alpha among those with mass > mass_min and E > 0, and
 * deactivate the floor(prune_pct N_active) other active sites with the
 * smallest removal delta (ties to the smaller id in both).  The k-th split
 * parent (ascending id) keeps its slot for one child and takes the k-th
 * inactive slot for the other (no split when no slot is left).  Children: at
 * the residual centroid +- clamp(0.5 sqrt(m), 1.5, 48) px along the major
 * axis of the residual covariance (u = axis, a = -log(l1/l2)/2 clamped), or
 * along the 3x3 Sobel gradient of the target at the parent (a scaled by
 * a_fallback_scale) when the energy or the anisotropy is too small;
 * log_tau += log_tau_shift, r *= r_scale, colour = target at the child, Adam
 * m and v zeroed.  If map (uint32[K/4][H*W][4], may be NULL) is given, each
 * new child is written into the last list slot of its pixel.  Synchronises
 * the stream; *n_active_out (HOST) receives the active count afterwards.
 * workspace: sad_densify_workspace_bytes(capacity, H, W) bytes, 256-B aligned.
 */
size_t sad_densify_workspace_bytes(int32_t capacity, int32_t H, int32_t W);
int sad_densify_prune(float* params, float* m, float* v, int32_t capacity, int32_t H, int32_t W,
                      int32_t K, const float* stats, const float* target, uint32_t* map,
                      const sad_dp_params* dp, int32_t* n_active_out, void* workspace,
                      size_t workspace_bytes, void* stream);

/*
 * sad_densify_prune_async -- the same event entirely on the stream: nothing
 * synchronises and no host memory is touched, so a training loop with
 * budget events runs without a host round trip and the call can be captured
 * in a CUDA graph (Sec. 5: the whole iteration stays on the GPU).
 * n_active_dev (DEVICE int32, 4-byte aligned) receives the active count
 * after the event, in stream order.  Other arguments as sad_densify_prune.
 */
int sad_densify_prune_async(float* params, float* m, float* v, int32_t capacity, int32_t H,
                            int32_t W, int32_t K, const float* stats, const float* target,
                            uint32_t* map, const sad_dp_params* dp, int32_t* n_active_dev,
                            void* workspace, size_t workspace_bytes, void* stream);

/* Adam hyper-parameters (Sec. 6.1; betas/eps after Kingma & Ba 2015). */
typedef struct sad_adam_hparams {
  float lr[SAD_NPARAMS]; /* per plane; x, y, r step in units of 1/s */
  float beta1, beta2, eps;
  float log_tau_min, log_tau_max; /* clamp (paper: [2, 20]) */
  float r_min, r_max;             /* clamp (paper: [1, 512]) */
  float a_min, a_max;             /* clamp (paper: [-2, 2]) */
  float b_min, b_max;             /* clamp of the log isotropic scale */
} sad_adam_hparams;

/*
 * sad_adam_step -- one bias-corrected Adam step on every active site
 * (Sec. 6.1): m = b1 m + (1-b1) g', v = b2 v + (1-b2) g'^2,
 * p -= lr mhat/(sqrt(vhat)+eps), where g' = g/s and the step is divided by s
 * for x, y and r (normalised units); then positions clamp to [0,W]x[0,H],
 * log_tau/r/a/b to their ranges, colours to [0,1], and (ux,uy) is
 * re-normalised.  Inactive sites are untouched.  t is the 1-based step.
 * params, m, v: float32[11][capacity] (updated in place); grads read.
 * hp: HOST pointer.
 */
int sad_adam_step(float* params, const float* grads, float* m, float* v, int32_t capacity,
                  int32_t H, int32_t W, int32_t t, const sad_adam_hparams* hp, void* stream);

/*
 * sad_tau_diffusion -- one Jacobi smoothing step of the log tau gradients
 * (App. "Tau Diffusion"): for every active site i, g_out[i] = (1 - lambda)
 * g[i] + lambda * mean of g[j] over the entries j of the top-K list of the
 * pixel containing site i (position clamped into the image) that are valid,
 * active and not i; sites that are inactive or have no such neighbour keep
 * g[i].  params: float32[11][capacity]; map: K/4 uint4 planes over H*W;
 * g_logtau, g_out: float32[capacity], distinct; lambda in [0, 1].
 */
int sad_tau_diffusion(const float* params, int32_t capacity, int32_t H, int32_t W, int32_t K,
                      const uint32_t* map, float lambda, const float* g_logtau, float* g_out,
                      void* stream);

/*
 * Batched training (many images, one launch per stage).  Each image owns a
 * contiguous range of site slots in the shared site arrays (ascending,
 * non-overlapping) and a contiguous range of pixels in the packed per-pixel
 * arrays: targets float32[total_pixels][3] (image b's pixel (x,y) at
 * pixel_offset + y*W + x) and the map planes uint32[K/4][total_pixels][4].
 * Site ids in the map are indices into the shared arrays.  At most 64 images.
 */
typedef struct sad_batch_image {
  int32_t H, W;          /* image size */
  int32_t site_offset;   /* first site slot of the image */
  int32_t capacity;      /* number of site slots of the image */
  int64_t pixel_offset;  /* first pixel of the image in the packed arrays */
  uint64_t seed;         /* injection seed of the image */
  int32_t state_index;   /* sad_train_step: the image's row of image_state */
  int32_t flags;         /* sad_train_step: 0, or SAD_STEP_KEEP_LISTS */
} sad_batch_image;

/* Batch-image flag: this call skips the image's propagation pass and runs
 * the adjoint on its current lists (candidate update period f_cand > 1,
 * App. "Candidate Field and Jump Schedule", Candidate update frequency);
 * only the image's Adam step t advances. */
#define SAD_STEP_KEEP_LISTS 1

/* Workspace bytes of sad_train_step (0 = invalid table); same record rule as
 * sad_backward_workspace_bytes with P = total_pixels.  The workspace must be
 * ZEROED once when allocated: its per-site record counts (at a fixed offset
 * that depends on total_capacity only) are cleared by each call after use,
 * so one workspace serves any sequence of tables over the same arrays.  A
 * call that returned an error may leave them dirty: zero the workspace again. */
size_t sad_step_workspace_bytes(const sad_batch_image* images, int32_t B, int32_t K,
                                int32_t tile_w, int32_t total_capacity, int64_t total_pixels,
                                int64_t max_records);

/* sad_prepare_sites for every image of a batch (each with its own s); only
 * the images' slot ranges are touched. */
int sad_prepare_batch(const sad_batch_image* images, int32_t B, const float* params, float* prep,
                      int32_t total_capacity, int64_t total_pixels, void* stream);

/*
 * sad_train_step -- one fused training iteration of every image of a batch
 * (Sec. 5: no host work inside an iteration).  tile_w: 16 (16x16 pixel
 * tiles) or 32 (32x8 tiles), the tile shape of the adjoint's per-tile
 * reduction (an autotuning choice; the lists do not depend on it, the
 * gradients only by rounding).  Per tile: one
 * propagation pass at jump 1 (sad_update_topk semantics with the image's own
 * site range and seed) writing the image's next map, then, on those lists,
 * the fused render + MSE + adjoint of sad_train_grads (one difference: a
 * pixel's list ends at the first entry whose softmax weight is below 1e-7
 * of the running sum, the list being sorted by the pass's logits, so at
 * most 1.6e-6 of the pixel's weight is left out); per site: the
 * gradient, an Adam step (sad_adam_step semantics with the image's H, W) and
 * the prepared table of the new parameters, so `prep` must hold the
 * prepared table of `params` on entry (sad_prepare_batch) and holds it again
 * on exit.
 * image_state: device int32[n_states][4]; image b uses row
 * images[b].state_index (distinct rows) = {t, pass, parity, 0}: t is the
 * Adam step (1-based), pass the pass index of the propagation (step code
 * (1 << 16) | (pass & 0xffff)), parity 0 = its current map is in map_in
 * (then it writes map_out), 1 = the reverse.  The call advances the rows of
 * the images it steps (t + 1, pass + 1, parity ^ 1; only t + 1 for an image
 * flagged SAD_STEP_KEEP_LISTS, whose propagation is skipped), so a fixed
 * batch always makes the same call (capture it once in a CUDA graph and
 * replay it), and an image left out of some calls keeps its own counters
 * and map.
 * loss: device float32[B], the mean loss of each image before the step (may
 * be NULL).  grads_out: optional float32[11][total_capacity].  map_in and
 * map_out must not overlap.  Each image's results are independent of the
 * other images in the batch.  Only the images' slot and pixel ranges and
 * state rows are read or written (besides the workspace), so images can
 * join or leave between calls (continuous batching); images must not share
 * pixels (SAD_EINVAL).
 */
int sad_train_step(const sad_batch_image* images, int32_t B, int32_t K, int32_t J, int32_t tile_w,
                   float* params, float* m, float* v, float* prep, int32_t total_capacity,
                   uint32_t* map_in, uint32_t* map_out, int64_t total_pixels,
                   const float* targets, float* loss, const sad_adam_hparams* hp,
                   int32_t* image_state, int32_t n_states, float* grads_out, void* workspace,
                   size_t workspace_bytes, void* stream);

/*
 * sad_batch_update -- one propagation pass at jump 1 (sad_update_topk
 * semantics, each image with its own site range, seed, pass index and
 * current map from its state row) for every image of the table, advancing
 * each row's pass index and parity (t unchanged): the extra passes of a
 * candidate update with n_cand > 1 (App. "Candidate Field and Jump
 * Schedule", Candidate update frequency).  Arguments as sad_train_step
 * (the pass does not depend on a tile shape).
 */
int sad_batch_update(const sad_batch_image* images, int32_t B, int32_t K, int32_t J,
                     const float* prep, int32_t total_capacity, uint32_t* map_in, uint32_t* map_out,
                     int64_t total_pixels, int32_t* image_state, int32_t n_states, void* stream);

/*
 * sad_batch_insert -- place one image, prepared with the single-image calls
 * (sad_init_sites, sad_topk_seed, sad_update_topk), into its ranges of the
 * shared batch arrays: params[:, site_offset + i] = src_params[:, i] for
 * i < capacity (src plane stride src_capacity >= capacity) with m and v
 * cleared there; map cell ids shifted by site_offset (ids >= capacity become
 * 0xffffffff); the target pixels copied when src_target is not NULL
 * (float32[H*W][3]).  `image`: HOST pointer to the image's table entry.
 * Library addition with no counterpart in the paper (the batching layer).
 */
int sad_batch_insert(const sad_batch_image* image, int32_t K, const float* src_params,
                     int32_t src_capacity, const uint32_t* src_map, const float* src_target,
                     float* params, float* m, float* v, int32_t total_capacity, uint32_t* map,
                     float* targets, int64_t total_pixels, void* stream);

/*
 * sad_decode_batch -- random-access decode (as sad_decode_points) of queries
 * against several resident images at once: query i at xy[i] (image pixel
 * units) uses image query_image[i] of the table (its map cell, its sites).
 * xy: float32[n][2]; query_image: int32[n]; rgb: float32[n][3].
 */
int sad_decode_batch(const sad_batch_image* images, int32_t B, int32_t K, const float* prep,
                     int32_t total_capacity, const uint32_t* map, int64_t total_pixels,
                     const float* xy, const int32_t* query_image, int64_t n, float* rgb,
                     void* stream);

/*
 * Packed 16-byte evaluation sites (App. "Data Layout and Packing", Packed
 * storage for evaluation).  Per site four 32-bit words:
 *   w0 = x/W, y/H as 15-bit UNORM (bits 0-14, 15-29), active flag bit 31
 *   w1 = colour r, g, b as 11/11/10-bit UNORM over the per-image ranges
 *   w2 = (log tau', r') as 16/16-bit UNORM over the per-image ranges
 *   w3 = angle of u as a 16-bit UNORM code over [-pi, pi] (bits 0-15), a as
 *        float16 (bits 16-31)
 * with b folded in exactly: log tau' = log tau + b/2, r' = r e^{-b/2} (the
 * unpacked sites have b = 0).  q = float32[10]: (lo, hi) of log tau', r',
 * colour r, g, b over the active sites.  Codes are round-half-even of
 * (v - lo)/(hi - lo) * (2^bits - 1) computed in double; inactive sites pack
 * to four zero words and unpack with x = y = -1.
 *
 * sad_pack_sites: params float32[11][capacity] -> packed uint32[capacity][4]
 *   (16-byte aligned) and q (DEVICE float32[10]).
 * sad_unpack_sites: packed + q (DEVICE) -> params float32[11][capacity].
 * sad_decode_packed: sad_decode_points reading the packed records (each
 *   listed site unpacked in float32 on the fly); q_host: HOST float32[10].
 * sad_render_packed: sad_render reading the packed records (the paper's
 *   evaluation render); q_host: HOST float32[10].
 * Library additions with no counterpart in the paper beyond the format.
 */
int sad_pack_sites(const float* params, int32_t capacity, int32_t H, int32_t W, uint32_t* packed,
                   float* q, void* stream);
int sad_unpack_sites(const uint32_t* packed, const float* q, int32_t capacity, int32_t H, int32_t W,
                     float* params, void* stream);
int sad_decode_packed(const uint32_t* packed, const float* q_host, int32_t capacity, int32_t H,
                      int32_t W, int32_t K, const uint32_t* map, const float* xy, int64_t n,
                      float* rgb, void* stream);
int sad_render_packed(const uint32_t* packed, const float* q_host, int32_t capacity, int32_t H,
                      int32_t W, int32_t K, const uint32_t* map, float* rgb, void* stream);

/*
 * 1-D SAD (Sec. "1D Signal Fitting"): the soft partition of unity of Sec. 4.2
 * on a line.  A batch of B independent signals of L samples each (sample k at
 * x = k + 0.5, s = 1/L), each with its own N sites of four parameters,
 * float32[4][B*N] planes (p position in samples, c value, log_tau, r radius
 * in samples; site i of signal b at column b*N + i):
 *   l_i(x) = tau_i s (r_i - |x - p_i|),   tau = exp(log_tau),
 * the value at x is the softmax blend of the K sites of the signal with the
 * largest logit (ties to the smaller index); K >= N blends all N sites (the
 * paper's 64-site fits).  Limits: 1 <= N <= 1024; K >= N, or K <= 16.
 *
 * sad1d_render -- values: float32[B][L] (written).
 */
int sad1d_render(const float* params, int32_t B, int32_t N, int32_t L, int32_t K, float* values,
                 void* stream);

/* Adam of the 1-D sites (Sec. 6.1 conventions; Kingma & Ba 2015). */
typedef struct sad1d_adam_hparams {
  float lr[4];          /* per plane p, c, log_tau, r; p and r in normalised units (value * s) */
  float beta1, beta2, eps;
  float log_tau_min, log_tau_max; /* clamp of log_tau after the step */
} sad1d_adam_hparams;

/*
 * sad1d_train_step -- one fused training iteration of every signal: render,
 * L_b = mean over samples of (c(x) - y(x))^2 (loss: float32[B], written),
 * the adjoint with the top-K sets held fixed (dL/dc_i = sum w_i g,
 * delta_i = w_i g (c_i - cbar) = dL/dl_i, dl/dlog_tau = l, dl/dr = tau s,
 * dl/dp = tau s sign(x - p), 0 at x = p; g = 2 (c - y) / L), summed per site
 * in a fixed order (no atomics), then bias-corrected Adam with Adam step t
 * (1-based) and the clamps p, r in [0, L], log_tau in [log_tau_min,
 * log_tau_max].  params, m, v: float32[4][B*N] (updated); target:
 * float32[B][L]; grads_out: float32[4][B*N] or NULL.  One 256-thread block
 * per signal: the results of a signal do not depend on the rest of the batch.
 */
int sad1d_train_step(float* params, float* m, float* v, int32_t B, int32_t N, int32_t L, int32_t K,
                     const float* target, float* loss, const sad1d_adam_hparams* hp, int32_t t,
                     float* grads_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SAD_H */
