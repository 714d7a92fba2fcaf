"""CPU oracle for Soft Anisotropic Diagrams (SAD).

TEST INFRASTRUCTURE.  This is a plain, slow, obviously correct restatement of
what the SAD hot path computes, written from the paper (arXiv 2604.21984).
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  It shares no code,
header, table or constant with the CUDA path and never imports it; the only
module both sides use is the seeded input generator
``paper_2604_21984_gb300.inputs``, which holds none of the method's arithmetic.

Site parameters: ``float[11, N]`` planes (x, y, log_tau, r, cr, cg, cb, ux, uy,
a, b), positions and radii in pixels, pixel (col, row) centred at
(col + 0.5, row + 0.5).  Index maps: ``uint32[P, K]`` with sentinel 0xffffffff.

Part 1 (fp64, the definitions):
  metric            Sec. 4.1, metric G_i (+ log isotropic scale b; b = 0 is the paper)
  logits            Sec. 4.1 score d_mix and Sec. 4.2 logit l_i = -tau_i d_mix
  render            Sec. 4.2 softmax weights w_i and colour c(x)
  exact_topk        Sec. 4.3: the set the propagation approximates (brute force)
  render_backward   App. "Gradient Computation and Reduction", Per-pixel gradients: adjoint of the blend
  removal_delta     Sec. 4.5 removal delta
  adam_step         Sec. 6.1 (Adam, clamps, re-normalised u)
Part 2 (fp32, the top-K propagation as the kernel's precision decides it):
  exp32             Cody-Waite reduced Taylor exponential (see its docstring)
  prepare_fp32      per-site derived table ("pack", App. "Data Layout and Packing")
  score_fp32        l_i(x) in a fixed fp32 operation order
  jump_step         Sec. 4.3 jump schedule s_t;  step_code: App. "Candidate Field and Jump Schedule", Step encoding
  splitmix64 / inject_ids   App. "Candidate Field and Jump Schedule" seeded stochastic injection (counter-based)
  topk_seed_fp32    App. "Candidate Field and Jump Schedule", JFA prepass seed pass
  topk_pass_fp32    Sec. 4.3 update C_t = topK(C_{t-1} U P_t U G_t)
  jfa_flood_fp32    App. "Candidate Field and Jump Schedule", JFA prepass flood pass (3x3, first 4 slots)
  grid_dims / expand_grid   App. "Candidate Field and Jump Schedule", downscaled candidate grid
Part 3: gradient-weighted initialisation (Sec. 4.4).
Part 4: adaptive budget: statistics, densify split, prune (Sec. 4.5).
Part 5: packed 16-byte evaluation sites (App. "Data Layout and Packing",
  Packed storage for evaluation): pack_eval / unpack_eval.
Part 6: tau diffusion (App. "Tau Diffusion").
Part 7: half2 candidate sites (App. "Data Layout and Packing", Packed
  candidate sites): candidate_halves / candidate_words / candidate_table_fp32.
Part 8: 1-D SAD (Sec. "1D Signal Fitting"): sad1d_logits / sad1d_topk /
  sad1d_render / sad1d_backward / sad1d_adam_step / sad1d_train_step.
"""
from __future__ import annotations

import math

import numpy as np

N_PARAMS = 11
PX, PY, PLOGTAU, PR, PCR, PCG, PCB, PUX, PUY, PA, PB = range(N_PARAMS)
INVALID = 0xFFFFFFFF


# =============================================================================
# Part 1: fp64 definitions
# =============================================================================

def scale_s(H: int, W: int) -> float:
    """s = 1 / max(H, W) (Sec. 4.1, resolution-invariant score)."""
    return 1.0 / max(H, W)


def unit_direction(ux, uy):
    """u = (ux, uy) / |(ux, uy)|; a zero vector reads as u = (1, 0)."""
    ux = np.asarray(ux, dtype=np.float64)
    uy = np.asarray(uy, dtype=np.float64)
    nrm = np.hypot(ux, uy)
    ok = nrm > 0
    safe = np.where(ok, nrm, 1.0)
    return np.where(ok, ux / safe, 1.0), np.where(ok, uy / safe, 0.0)


def metric(params):
    """Per-site SPD metric G = e^b (e^a u u^T + e^-a v v^T), v = u rotated by +90 deg.

    Sec. 4.1 (metric G_i): eigenvalue e^a along u and e^-a along v, det = 1.
    The factor e^b is the log isotropic scale read from the configs' "metric
    scale" (b = 0 reproduces the paper exactly).  Returns (G00, G01, G11).
    """
    p = np.asarray(params, dtype=np.float64)
    ux, uy = unit_direction(p[PUX], p[PUY])
    vx, vy = -uy, ux
    ea = np.exp(p[PB] + p[PA])
    eb = np.exp(p[PB] - p[PA])
    G00 = ea * ux * ux + eb * vx * vx
    G01 = ea * ux * uy + eb * vx * vy
    G11 = ea * uy * uy + eb * vy * vy
    return G00, G01, G11


def active_mask(params):
    """Inactive sentinel: x < 0 (App. "Data Layout and Packing", Site buffer)."""
    return np.asarray(params, dtype=np.float64)[PX] >= 0


def pixel_centres(H: int, W: int):
    """Centres (col + 0.5, row + 0.5) of all pixels in row-major order."""
    row, col = np.divmod(np.arange(H * W), W)
    return col + 0.5, row + 0.5


def logits(params, H, W, ids, px, py):
    """l_i(x) = -tau_i * d_mix(x, i) for every (query point, listed id).

    Sec. 4.1: d_mix = |x - p_i|_{G_i} s - r_i s with |v|_G = sqrt(v^T G v);
    Sec. 4.2: l_i(x) = -tau_i d_mix(x, i), tau_i = exp(log_tau_i).
    ``ids`` is int64[Q, M] of valid site ids, px/py are float[Q].
    """
    p = np.asarray(params, dtype=np.float64)
    G00, G01, G11 = metric(p)
    s = scale_s(H, W)
    dx = np.asarray(px, np.float64)[:, None] - p[PX][ids]
    dy = np.asarray(py, np.float64)[:, None] - p[PY][ids]
    quad = G00[ids] * dx * dx + 2.0 * G01[ids] * dx * dy + G11[ids] * dy * dy
    norm = np.sqrt(np.maximum(quad, 0.0))
    d_mix = norm * s - p[PR][ids] * s
    return -np.exp(p[PLOGTAU][ids]) * d_mix


def _valid_entries(params, ids):
    """Mask of list entries that name an existing, active site."""
    ids = np.asarray(ids)
    n = np.asarray(params).shape[1]
    valid = (ids != INVALID) & (ids.astype(np.int64) < n)
    safe = np.where(valid, ids, 0).astype(np.int64)
    valid &= active_mask(params)[safe]
    return valid, safe


def weights(params, H, W, ids, px=None, py=None):
    """Softmax weights w_i(x) over the listed set C(x) (Sec. 4.2).

    Invalid or inactive entries get weight 0; a pixel with no valid entry gets
    all-zero weights.  Returns (w[Q,K], logits[Q,K] with -inf at invalid,
    valid mask, safe ids).
    """
    if px is None:
        px, py = pixel_centres(H, W)
    valid, safe = _valid_entries(params, ids)
    ell = np.where(valid, logits(params, H, W, safe, px, py), -np.inf)
    any_valid = valid.any(axis=1)
    m = np.where(any_valid, np.max(np.where(valid, ell, -np.inf), axis=1), 0.0)
    e = np.where(valid, np.exp(ell - m[:, None]), 0.0)
    z = e.sum(axis=1)
    w = e / np.where(z > 0, z, 1.0)[:, None]
    return w, ell, valid, safe


def render(params, H, W, ids, px=None, py=None):
    """c(x) = sum_{i in C(x)} w_i(x) c_i (Sec. 4.2).  Returns float64[Q, 3]."""
    p = np.asarray(params, dtype=np.float64)
    w, _, _, safe = weights(p, H, W, ids, px, py)
    col = np.stack([p[PCR], p[PCG], p[PCB]], axis=1)   # [N, 3]
    return np.einsum("qk,qkc->qc", w, col[safe])


def exact_topk(params, H, W, K, pixels=None, chunk=4096):
    """Exact top-K ids under l_i(x) over ALL active sites (brute force).

    This is the set the propagation of Sec. 4.3 approximates.  Order: l
    descending, ties to the smaller id; fewer than K active sites leaves
    trailing sentinels.  Returns (uint32[Q, K], float64 logits[Q, K]).
    """
    p = np.asarray(params, dtype=np.float64)
    act = np.nonzero(active_mask(p))[0]
    if pixels is None:
        pixels = np.arange(H * W)
    pixels = np.asarray(pixels)
    out = np.full((len(pixels), K), INVALID, dtype=np.uint32)
    out_l = np.full((len(pixels), K), -np.inf)
    kk = min(K, len(act))
    if kk == 0:
        return out, out_l
    for c0 in range(0, len(pixels), chunk):
        pix = pixels[c0:c0 + chunk]
        row, col = np.divmod(pix, W)
        ids = np.broadcast_to(act, (len(pix), len(act)))
        ell = logits(p, H, W, ids, col + 0.5, row + 0.5)
        sel = select_topk(ids, ell, np.ones(ell.shape, bool), kk)
        out[c0:c0 + len(pix), :kk] = sel
        pos = np.searchsorted(act, sel.astype(np.int64))
        out_l[c0:c0 + len(pix), :kk] = np.take_along_axis(ell, pos, axis=1)
    return out, out_l


def select_topk(pool_ids, ell, valid, K):
    """Per row: drop invalid entries, collapse duplicate ids, keep the K best
    by (l descending, id ascending), pad with the sentinel.

    A duplicate id in one row carries the same logit, so after sorting rows by
    (row, -l, id) duplicates are adjacent.  Returns uint32[Q, K].
    """
    pool_ids = np.asarray(pool_ids)
    Q, M = pool_ids.shape
    rows = np.repeat(np.arange(Q), M)[valid.ravel()]
    ids = pool_ids.ravel()[valid.ravel()].astype(np.int64)
    neg = -np.asarray(ell).ravel()[valid.ravel()]
    order = np.lexsort((ids, neg, rows))
    rows, ids = rows[order], ids[order]
    keep = np.ones(len(rows), dtype=bool)
    keep[1:] = ~((rows[1:] == rows[:-1]) & (ids[1:] == ids[:-1]))
    rows, ids = rows[keep], ids[keep]
    rank = np.arange(len(rows)) - np.searchsorted(rows, rows, side="left")
    take = rank < K
    out = np.full((Q, K), INVALID, dtype=np.uint32)
    out[rows[take], rank[take]] = ids[take]
    return out


def render_backward(params, H, W, ids, grad_rgb, px=None, py=None):
    """Adjoint of the blend into every site parameter (App. "Gradient Computation and Reduction"), fp64.

    Given g(x) = dL/dc(x) (``grad_rgb`` [Q, 3]) and a frozen index set C(x),
    returns dL/dparams as float64[11, N] in plane order.  Per pixel, with the
    max-subtracted softmax w and blended colour cbar:
      dL/dc_k      = w_k g
      dL/dl_k      = delta_k = w_k g . (c_k - cbar)
      dl/dlog_tau  = l_k                 dl/dr = tau s
      Delta = x - p, alpha = u.Delta, beta = v.Delta,
      q = e^b (e^a alpha^2 + e^-a beta^2), n = sqrt(q), dl/dn = -tau s
      dn/dp = -G Delta / n
      dn/da = e^b (e^a alpha^2 - e^-a beta^2) / (2n),   dn/db = n / 2
      dn/dtheta = e^b alpha beta (e^a - e^-a) / n,  theta = atan2(uy, ux),
      dtheta/d(ux, uy) = (-uy, ux) / (ux^2 + uy^2).
    At n = 0 (query exactly on a site) the geometric terms (p, a, b, u) are
    taken as 0; invalid/inactive entries contribute nothing.
    """
    p = np.asarray(params, dtype=np.float64)
    N = p.shape[1]
    if px is None:
        px, py = pixel_centres(H, W)
    px = np.asarray(px, np.float64)
    py = np.asarray(py, np.float64)
    g = np.asarray(grad_rgb, dtype=np.float64).reshape(-1, 3)
    w, ell, valid, sid = weights(p, H, W, ids, px, py)
    col = np.stack([p[PCR], p[PCG], p[PCB]], axis=1)
    ck = col[sid]                                        # [Q, K, 3]
    cbar = np.einsum("qk,qkc->qc", w, ck)
    delta = w * np.einsum("qc,qkc->qk", g, ck - cbar[:, None, :])

    s = scale_s(H, W)
    tau = np.exp(p[PLOGTAU])[sid]
    a, b = p[PA][sid], p[PB][sid]
    ux, uy = unit_direction(p[PUX], p[PUY])
    ux, uy = ux[sid], uy[sid]
    vx, vy = -uy, ux
    dx = px[:, None] - p[PX][sid]
    dy = py[:, None] - p[PY][sid]
    alpha = ux * dx + uy * dy
    beta = vx * dx + vy * dy
    ea, em, eb = np.exp(a), np.exp(-a), np.exp(b)
    q = eb * (ea * alpha ** 2 + em * beta ** 2)
    n = np.sqrt(q)
    has_n = valid & (n > 0)
    inv_n = np.where(has_n, 1.0 / np.where(has_n, n, 1.0), 0.0)
    dl_dn = -tau * s
    G00, G01, G11 = metric(p)
    GDx = G00[sid] * dx + G01[sid] * dy
    GDy = G01[sid] * dx + G11[sid] * dy
    dn_dpx = -GDx * inv_n
    dn_dpy = -GDy * inv_n
    dn_da = eb * (ea * alpha ** 2 - em * beta ** 2) * 0.5 * inv_n
    dn_db = 0.5 * n * has_n
    dn_dth = eb * alpha * beta * (ea - em) * inv_n
    rawx, rawy = p[PUX][sid], p[PUY][sid]
    r2 = rawx ** 2 + rawy ** 2
    r2 = np.where(r2 > 0, r2, 1.0)
    dth_dux, dth_duy = -rawy / r2, rawx / r2

    dv = np.where(valid, delta, 0.0)
    contrib = np.zeros((N_PARAMS,) + sid.shape)
    contrib[PX] = dv * dl_dn * dn_dpx
    contrib[PY] = dv * dl_dn * dn_dpy
    contrib[PLOGTAU] = dv * np.where(valid, ell, 0.0)
    contrib[PR] = dv * tau * s
    for c, plane in enumerate((PCR, PCG, PCB)):
        contrib[plane] = np.where(valid, w * g[:, c:c + 1], 0.0)
    contrib[PUX] = dv * dl_dn * dn_dth * dth_dux
    contrib[PUY] = dv * dl_dn * dn_dth * dth_duy
    contrib[PA] = dv * dl_dn * dn_da
    contrib[PB] = dv * dl_dn * dn_db

    grads = np.zeros((N_PARAMS, N))
    flat_ids = np.where(valid, sid, 0).ravel()
    for j in range(N_PARAMS):
        np.add.at(grads[j], flat_ids, np.where(valid, contrib[j], 0.0).ravel())
    return grads


def mse_loss_and_grad_rgb(rgb, target):
    """L = E_x |c(x) - I(x)|^2 (Sec. 6.1) and g = dL/dc = 2 (c - I) / P."""
    c = np.asarray(rgb, np.float64).reshape(-1, 3)
    t = np.asarray(target, np.float64).reshape(-1, 3)
    P = c.shape[0]
    diff = c - t
    return float((diff ** 2).sum() / P), 2.0 * diff / P


def removal_delta(params, H, W, ids, target):
    """Per-site removal delta summed over pixels (Sec. 4.5, removal delta).

    For each listed site k at pixel x with weight w_k: c' = (c - w_k c_k) /
    (1 - w_k) and dL(x) = |c' - I|^2 - |c - I|^2, summed per site.  c' is
    the blend of the remaining sites; for the pixel's dominant site (largest
    logit, where 1 - w_k may be tiny) it is evaluated as that blend directly,
    with its own max subtracted, which is the same value in exact arithmetic.
    Removing the only valid site leaves black: dL = |I|^2 - |c - I|^2.
    Returns float64[N].
    """
    p = np.asarray(params, dtype=np.float64)
    w, ell, valid, sid = weights(p, H, W, ids)
    col = np.stack([p[PCR], p[PCG], p[PCB]], axis=1)
    ck = col[sid]
    c = np.einsum("qk,qkc->qc", w, ck)
    I = np.asarray(target, np.float64).reshape(-1, 3)
    base = ((c - I) ** 2).sum(1)
    Q, K = ids.shape
    dom = np.argmax(np.where(valid, ell, -np.inf), axis=1)
    others = valid.copy()
    others[np.arange(Q), dom] = False
    has_o = others.any(axis=1)
    l2 = np.where(others, ell, -np.inf)
    m2 = np.where(has_o, l2.max(axis=1), 0.0)
    e2 = np.where(others, np.exp(l2 - m2[:, None]), 0.0)
    z2 = e2.sum(axis=1)
    c_dom = np.einsum("qk,qkc->qc", e2, ck) / np.where(z2 > 0, z2, 1.0)[:, None]
    c_dom = np.where(has_o[:, None], c_dom, 0.0)
    out = np.zeros(p.shape[1])
    for k in range(K):
        wk = w[:, k]
        is_dom = dom == k
        denom = np.where(is_dom, 1.0, 1.0 - wk)
        cprime = np.where(is_dom[:, None], c_dom, (c - wk[:, None] * ck[:, k]) / denom[:, None])
        dl = ((cprime - I) ** 2).sum(1) - base
        np.add.at(out, sid[valid[:, k], k], dl[valid[:, k]])
    return out


# ---------------------------------------------------------------------------
# Adam (Sec. 6.1): per-parameter learning rates, fixed betas / eps, clamps,
# re-normalised direction.  Positions and radii step in normalised units p*s.
# ---------------------------------------------------------------------------

DEFAULT_LR = {
    "x": 1e-3, "y": 1e-3, "log_tau": 1e-2, "r": 1e-3, "cr": 5e-3, "cg": 5e-3,
    "cb": 5e-3, "ux": 1e-2, "uy": 1e-2, "a": 1e-2, "b": 0.0,
}
PLANE_NAMES = ("x", "y", "log_tau", "r", "cr", "cg", "cb", "ux", "uy", "a", "b")


def adam_step(params, grads, m, v, t, H, W, lr=None, beta1=0.9, beta2=0.999,
              eps=1e-8, log_tau_range=(2.0, 20.0), r_range=(1.0, 512.0),
              a_range=(-2.0, 2.0), b_range=(-8.0, 8.0)):
    """One bias-corrected Adam step (Kingma & Ba 2015) with the paper's clamps.

    Sec. 6.1: positions clamped to the image, log_tau in [2, 20], r in [1, 512],
    a in [-2, 2], colours in [0, 1], u re-normalised after the step.  x, y and
    r are optimised in normalised units (value * s), so their gradient is
    divided by s and their step multiplied by 1/s.  Inactive sites (x < 0) are
    left untouched.  ``t`` is the 1-based step count.  Returns new
    (params, m, v) as float64.
    """
    lr = dict(DEFAULT_LR if lr is None else lr)
    p = np.array(params, dtype=np.float64)
    g = np.asarray(grads, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    s = scale_s(H, W)
    act = p[PX] >= 0
    for j, name in enumerate(PLANE_NAMES):
        unit = s if j in (PX, PY, PR) else 1.0
        gj = g[j] / unit
        mj = beta1 * m[j] + (1 - beta1) * gj
        vj = beta2 * v[j] + (1 - beta2) * gj * gj
        mhat = mj / (1 - beta1 ** t)
        vhat = vj / (1 - beta2 ** t)
        step = lr[name] * mhat / (np.sqrt(vhat) + eps) / unit
        p[j] = np.where(act, p[j] - step, p[j])
        m[j] = np.where(act, mj, m[j])
        v[j] = np.where(act, vj, v[j])
    clip = lambda j, lo, hi: np.where(act, np.clip(p[j], lo, hi), p[j])
    p[PX] = clip(PX, 0.0, float(W))
    p[PY] = clip(PY, 0.0, float(H))
    p[PLOGTAU] = clip(PLOGTAU, *log_tau_range)
    p[PR] = clip(PR, *r_range)
    p[PA] = clip(PA, *a_range)
    p[PB] = clip(PB, *b_range)
    for j in (PCR, PCG, PCB):
        p[j] = clip(j, 0.0, 1.0)
    ux, uy = unit_direction(p[PUX], p[PUY])
    p[PUX] = np.where(act, ux, p[PUX])
    p[PUY] = np.where(act, uy, p[PUY])
    return p, m, v


# =============================================================================
# Part 2: the fp32 top-K propagation, decided in the kernel's precision
# =============================================================================

F32 = np.float32
# 1/k! for k = 2..7, each the float32 nearest to the exact rational (hex).
_INV_FACT = [F32(float.fromhex(h)) for h in (
    "0x1.000000p-1",   # 1/2
    "0x1.555556p-3",   # 1/6
    "0x1.555556p-5",   # 1/24
    "0x1.111112p-7",   # 1/120
    "0x1.6c16c2p-10",  # 1/720
    "0x1.a01a02p-13",  # 1/5040
)]
_LOG2E = F32(float.fromhex("0x1.715476p+0"))     # 1/ln 2, nearest float32
_LN2_HI = F32(45426.0 / 65536.0)                  # ln 2 cut to 16 bits: k*LN2_HI exact
_LN2_LO = F32(math.log(2.0) - 45426.0 / 65536.0)  # remainder of ln 2


def exp32(x):
    """Reproducible float32 e^x (every step a rounded fp32 + or *).

    Published method: Cody & Waite (1980) argument reduction with ln 2 split
    into a 16-bit head and a tail, x = k ln2 + r, |r| <= ln2/2, then the
    degree-7 Taylor polynomial of e^r (coefficients 1/k!) by Horner's rule,
    then scaling by 2^k.  Inputs are clamped to [-80, 80] so 2^k and the
    result stay normal.  Accuracy: a few ulp (pinned in the tests).  The same
    definition is implemented independently on the GPU so that the derived
    site table, and hence the top-K decisions, agree bit for bit.
    """
    x = np.clip(np.asarray(x, dtype=F32), F32(-80.0), F32(80.0)).astype(F32)
    k = np.rint((x * _LOG2E).astype(F32)).astype(F32)
    r = (x - (k * _LN2_HI).astype(F32)).astype(F32)
    r = (r - (k * _LN2_LO).astype(F32)).astype(F32)
    p = _INV_FACT[5]
    for c in (_INV_FACT[4], _INV_FACT[3], _INV_FACT[2], _INV_FACT[1], _INV_FACT[0], F32(1.0), F32(1.0)):
        p = ((p * r).astype(F32) + c).astype(F32)
    scale = np.ldexp(np.ones_like(k, dtype=F32), k.astype(np.int32)).astype(F32)
    return (p * scale).astype(F32)


def prepare_fp32(params, H, W):
    """Per-site derived table for scoring (App. "Data Layout and Packing", packed candidate sites).

    In float32, operation by operation:
      s = 1 / max(H, W);  nrm = sqrt(ux*ux + uy*uy);  u = (ux, uy)/nrm (or (1,0))
      e+ = exp32(b + a);  e- = exp32(b - a)
      G00 = e+ (ux ux) + e- (uy uy);  G01 = (e+ - e-)(ux uy);  G11 = e+ (uy uy) + e- (ux ux)
      tau_s = exp32(log_tau) * s;   active = x >= 0
    Returns dict of float32 arrays x, y, ts, r, G00, G01, G11, active(bool),
    cr, cg, cb.
    """
    p = np.asarray(params, dtype=F32)
    s = F32(F32(1.0) / F32(max(H, W)))
    ux, uy = p[PUX], p[PUY]
    nrm = np.sqrt(((ux * ux).astype(F32) + (uy * uy).astype(F32)).astype(F32)).astype(F32)
    ok = nrm > F32(0)
    safe = np.where(ok, nrm, F32(1)).astype(F32)
    uxn = np.where(ok, (ux / safe).astype(F32), F32(1)).astype(F32)
    uyn = np.where(ok, (uy / safe).astype(F32), F32(0)).astype(F32)
    ep = exp32((p[PB] + p[PA]).astype(F32))
    em = exp32((p[PB] - p[PA]).astype(F32))
    xx = (uxn * uxn).astype(F32)
    yy = (uyn * uyn).astype(F32)
    xy = (uxn * uyn).astype(F32)
    G00 = ((ep * xx).astype(F32) + (em * yy).astype(F32)).astype(F32)
    G01 = ((ep - em).astype(F32) * xy).astype(F32)
    G11 = ((ep * yy).astype(F32) + (em * xx).astype(F32)).astype(F32)
    ts = (exp32(p[PLOGTAU]) * s).astype(F32)
    return {
        "x": p[PX].copy(), "y": p[PY].copy(), "ts": ts, "r": p[PR].copy(),
        "G00": G00, "G01": G01, "G11": G11, "active": p[PX] >= F32(0),
        "cr": p[PCR].copy(), "cg": p[PCG].copy(), "cb": p[PCB].copy(),
    }


def score_fp32(prep, ids, px, py):
    """l_i(x) in float32, fixed order, no fused multiply-add:

    dx = px - x; dy = py - y; t0 = (G00 dx) dx; t1 = (G01 dx) dy; t1 = t1 + t1;
    t2 = (G11 dy) dy; q = (t0 + t1) + t2; n = sqrt(max(q, 0)); l = ts (r - n).
    (l = -tau d_mix = tau s (r - |x - p|_G), Sec. 4.1-4.2.)  ``ids`` int64
    array of valid ids; px, py broadcastable float32.
    """
    px = np.asarray(px, F32)
    py = np.asarray(py, F32)
    dx = (px - prep["x"][ids]).astype(F32)
    dy = (py - prep["y"][ids]).astype(F32)
    t0 = ((prep["G00"][ids] * dx).astype(F32) * dx).astype(F32)
    t1 = ((prep["G01"][ids] * dx).astype(F32) * dy).astype(F32)
    t1 = (t1 + t1).astype(F32)
    t2 = ((prep["G11"][ids] * dy).astype(F32) * dy).astype(F32)
    q = ((t0 + t1).astype(F32) + t2).astype(F32)
    n = np.sqrt(np.fmax(q, F32(0))).astype(F32)
    return (prep["ts"][ids] * (prep["r"][ids] - n).astype(F32)).astype(F32)


def jump_step(t: int, H: int, W: int) -> int:
    """s_t = max(1, B / 2^(min(t, log2 B - 1) + 1)), B = 2^ceil(log2 max(H, W)) (Sec. 4.3)."""
    L = max(H, W)
    log2B = max(0, math.ceil(math.log2(L))) if L > 1 else 0
    B = 1 << log2B
    return max(1, B >> (min(t, log2B - 1) + 1)) if log2B > 0 else 1


def step_code(t: int, H: int, W: int) -> int:
    """32-bit step parameter: low 16 bits step index, high 16 bits jump (App. "Candidate Field and Jump Schedule")."""
    return ((jump_step(t, H, W) & 0xFFFF) << 16) | (t & 0xFFFF)


_M64 = (1 << 64) - 1


def splitmix64(seed: int, counter):
    """Output number counter+1 of SplitMix64 started at ``seed``.

    Steele, Lea & Flood (2014): state_n = seed + n * 0x9E3779B97F4A7C15, and
    the output function z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
    z *= 0x94D049BB133111EB; z ^= z >> 31.  Vectorised over ``counter``.
    """
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (c + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def inject_ids(seed: int, code: int, pixels, J: int, capacity: int):
    """The J injected candidate ids of each pixel for one pass (App. "Candidate Field and Jump Schedule").

    Counter = (step_code << 32) | (pixel * J + j), draw = SplitMix64 output,
    id = (draw_hi32 * capacity) >> 32 (Lemire's multiply-shift range map).
    Returns int64[len(pixels), J].
    """
    pix = np.asarray(pixels, dtype=np.uint64)
    j = np.arange(J, dtype=np.uint64)
    ctr = (np.uint64(code) << np.uint64(32)) | (pix[:, None] * np.uint64(J) + j[None, :])
    h = splitmix64(seed, ctr)
    hi = h >> np.uint64(32)
    with np.errstate(over="ignore"):
        ids = (hi * np.uint64(capacity)) >> np.uint64(32)
    return ids.astype(np.int64)


def topk_seed_fp32(prep, H, W, K, cell=1, image=None):
    """Seed pass of the JFA prepass (App. "Candidate Field and Jump Schedule"): every active site writes its id
    into slot 0 of the pixel that contains it; on a collision the smaller id
    wins.  All other entries are the sentinel.  With a candidate grid of
    cell x cell pixels (App. "Candidate Field and Jump Schedule", Downscaled
    candidate grid) H, W are the grid's size, ``image`` = (H, W) of the
    image, and the site's pixel (clamped to the image) maps to cell
    (col // cell, row // cell).  Returns uint32[H*W, K]."""
    Hi, Wi = (H, W) if image is None else image
    out = np.full((H * W, K), INVALID, dtype=np.uint32)
    for i in np.nonzero(prep["active"])[0]:
        col = min(max(int(math.floor(float(prep["x"][i]))), 0), Wi - 1) // cell
        row = min(max(int(math.floor(float(prep["y"][i]))), 0), Hi - 1) // cell
        pix = row * W + col
        out[pix, 0] = min(int(out[pix, 0]), int(i))
    return out


def grid_dims(H, W, cell):
    """Size of the candidate grid of an H x W image with cell x cell cells."""
    return (H + cell - 1) // cell, (W + cell - 1) // cell


def expand_grid(ids_grid, H, W, cell):
    """Per-pixel lists from a candidate grid: pixel (x, y) takes the list of
    cell (x // cell, y // cell) (integer mapping, no interpolation)."""
    Hc, Wc = grid_dims(H, W, cell)
    rows, cols = np.divmod(np.arange(H * W), W)
    return np.asarray(ids_grid)[(rows // cell) * Wc + cols // cell]


def topk_pass_fp32(prep, ids_in, H, W, K, code, J, seed, pixels=None, cell=1):
    """One propagation pass (Sec. 4.3, update of C_t), for all or some pixels.
    With a candidate grid (cell > 1) H, W are the grid's size, the "pixels"
    are its cells, and a cell's scores are taken at its centre
    ((col + 0.5) cell, (row + 0.5) cell) in image pixels (App. "Candidate
    Field and Jump Schedule", Downscaled candidate grid: the centred UV of
    the cell).

    Pool = C_{t-1}(x) (the pixel's own list) U P_t(x) (the lists of the four
    neighbours at (+-s, 0), (0, +-s), s = jump distance in ``code``; neighbours
    outside the image are skipped) U G_t(x) (J injected ids).  Entries that are
    the sentinel, out of range, inactive or score NaN are dropped; duplicates
    collapse; the K best by (l descending, id ascending) are kept, the rest of
    the list is the sentinel.  Reads ``ids_in`` only (Jacobi update).
    Returns uint32[len(pixels), K].
    """
    cap = len(prep["x"])
    if pixels is None:
        pixels = np.arange(H * W)
    pixels = np.asarray(pixels, dtype=np.int64)
    s = (code >> 16) & 0xFFFF
    row, col = np.divmod(pixels, W)
    pools = [ids_in[pixels].astype(np.int64)]
    for ddx, ddy in ((-s, 0), (s, 0), (0, -s), (0, s)):
        nc, nr = col + ddx, row + ddy
        inside = (nc >= 0) & (nc < W) & (nr >= 0) & (nr < H)
        nb = np.where(inside, nr * W + nc, 0)
        lst = ids_in[nb].astype(np.int64)
        pools.append(np.where(inside[:, None], lst, INVALID))
    if J > 0:
        pools.append(inject_ids(seed, code, pixels, J, cap))
    pool = np.concatenate(pools, axis=1)                  # [Q, M]
    valid = (pool != INVALID) & (pool >= 0) & (pool < cap)
    safe = np.where(valid, pool, 0)
    valid &= prep["active"][safe]
    px = ((col.astype(F32) + F32(0.5)).astype(F32) * F32(cell)).astype(F32)[:, None]
    py = ((row.astype(F32) + F32(0.5)).astype(F32) * F32(cell)).astype(F32)[:, None]
    ell = score_fp32(prep, safe, px, py)
    valid &= ~np.isnan(ell)
    return select_topk(pool, ell, valid, K)


def jfa_flood_fp32(prep, ids_in, H, W, code, slots=4):
    """One flood pass of the JFA prepass (App. "Candidate Field and Jump
    Schedule", JFA prepass): each pixel pools the first ``slots`` entries
    (the first candidate texture) of the lists of the 3x3 pixels at offsets
    {-s, 0, s}^2 around it, itself included (s = jump distance in ``code``;
    pixels outside the image are skipped), drops the sentinel, out-of-range,
    inactive and NaN-score entries, collapses duplicates, and writes the
    ``slots`` best by (l descending, id ascending) into its first ``slots``
    entries; the rest of its list is copied unchanged.  No injection.  Reads
    ``ids_in`` only (Jacobi).  Returns uint32[P, K]."""
    ids_in = np.asarray(ids_in, dtype=np.uint32)
    cap = len(prep["x"])
    pixels = np.arange(H * W, dtype=np.int64)
    s = (code >> 16) & 0xFFFF
    row, col = np.divmod(pixels, W)
    pools = []
    for ddy in (-s, 0, s):
        for ddx in (-s, 0, s):
            nc, nr = col + ddx, row + ddy
            inside = (nc >= 0) & (nc < W) & (nr >= 0) & (nr < H)
            nb = np.where(inside, nr * W + nc, 0)
            lst = ids_in[nb, :slots].astype(np.int64)
            pools.append(np.where(inside[:, None], lst, INVALID))
    pool = np.concatenate(pools, axis=1)
    valid = (pool != INVALID) & (pool >= 0) & (pool < cap)
    safe = np.where(valid, pool, 0)
    valid &= prep["active"][safe]
    px = (col.astype(F32) + F32(0.5)).astype(F32)[:, None]
    py = (row.astype(F32) + F32(0.5)).astype(F32)[:, None]
    ell = score_fp32(prep, safe, px, py)
    valid &= ~np.isnan(ell)
    out = ids_in.copy()
    out[:, :slots] = select_topk(pool, ell, valid, slots)
    return out


def propagate_fp32(params, H, W, K, passes, J, seed, ids_in=None, t0=0):
    """Seed (unless ``ids_in`` is given) then ``passes`` propagation passes
    with the jump schedule starting at step index t0.  Returns uint32[P, K]."""
    prep = prepare_fp32(params, H, W)
    ids = topk_seed_fp32(prep, H, W, K) if ids_in is None else np.asarray(ids_in, np.uint32)
    for t in range(t0, t0 + passes):
        ids = topk_pass_fp32(prep, ids, H, W, K, step_code(t, H, W), J, seed)
    return ids


def topk_match_stats(approx, exact):
    """Recall (fraction of exact top-K ids present) and exact-match fraction
    (pixels whose K-sets agree), as used for Table "Top-K propagation
    convergence" (Sec. 6.5)."""
    rec, match = [], []
    for a, e in zip(approx, exact):
        ea = set(int(v) for v in e if v != INVALID)
        aa = set(int(v) for v in a if v != INVALID)
        rec.append(len(ea & aa) / max(len(ea), 1))
        match.append(ea == aa)
    return float(np.mean(rec)), float(np.mean(match))


# =============================================================================
# Part 3: gradient-weighted initialisation (Sec. 4.4), decided in fp32
# =============================================================================

_LN2_HI_L = F32(45426.0 / 65536.0)
_LN2_LO_L = F32(math.log(2.0) - 45426.0 / 65536.0)
_SQRT2 = F32(float.fromhex("0x1.6a09e6p+0"))      # sqrt(2) rounded to float32
_INV_ODD = [F32(float.fromhex(h)) for h in ("0x1.555556p-2",   # 1/3
                                              "0x1.99999ap-3",   # 1/5
                                              "0x1.24924ap-3",   # 1/7
                                              "0x1.c71c72p-4")]  # 1/9


def log32(x):
    """Reproducible float32 natural log of positive normal x, every step a
    rounded fp32 op.  Published method (Cody & Waite 1980): x = 2^e m with
    m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1), log m = 2 atanh(s) =
    2s + 2s (s^2/3 + s^4/5 + s^6/7 + s^8/9) by Horner in s^2, and
    log x = e ln2_hi + (e ln2_lo + log m) with ln 2 split at 2^-16."""
    x = np.asarray(x, dtype=F32)
    bits = x.view(np.uint32).astype(np.int64)
    e = ((bits >> 23) & 0xFF) - 127
    m = ((bits & 0x7FFFFF) | (127 << 23)).astype(np.uint32).view(F32)
    big = m > _SQRT2
    m = np.where(big, (m * F32(0.5)).astype(F32), m).astype(F32)
    e = np.where(big, e + 1, e)
    ef = e.astype(F32)
    s = ((m - F32(1)).astype(F32) / (m + F32(1)).astype(F32)).astype(F32)
    s2 = (s * s).astype(F32)
    p = _INV_ODD[3]
    for c in (_INV_ODD[2], _INV_ODD[1], _INV_ODD[0]):
        p = ((p * s2).astype(F32) + c).astype(F32)
    p = (p * s2).astype(F32)
    s2x = (s + s).astype(F32)
    lm = (s2x + (s2x * p).astype(F32)).astype(F32)
    return ((ef * _LN2_HI_L).astype(F32) + ((ef * _LN2_LO_L).astype(F32) + lm).astype(F32)).astype(F32)


def grad_magnitude_fp32(img):
    """|grad I|_2 over the three channels with central differences (one-sided
    at the borders, zero across a single-pixel axis), float32:
    per channel dx = (I[x+1] - I[x-1]) * inv_dist, dy likewise, then
    g^2 = sum over channels in order of (dx^2 + dy^2), g = sqrt(g^2)."""
    I = np.asarray(img, dtype=F32)
    H, W, _ = I.shape
    cols = np.arange(W)
    rows = np.arange(H)
    cR, cL = np.minimum(cols + 1, W - 1), np.maximum(cols - 1, 0)
    rD, rU = np.minimum(rows + 1, H - 1), np.maximum(rows - 1, 0)
    invx = np.where(cR - cL == 2, F32(0.5), np.where(cR - cL == 1, F32(1.0), F32(0.0))).astype(F32)
    invy = np.where(rD - rU == 2, F32(0.5), np.where(rD - rU == 1, F32(1.0), F32(0.0))).astype(F32)
    g2 = np.zeros((H, W), dtype=F32)
    for c in range(3):
        dx = ((I[:, cR, c] - I[:, cL, c]).astype(F32) * invx[None, :]).astype(F32)
        dy = ((I[rD, :, c] - I[rU, :, c]).astype(F32) * invy[:, None]).astype(F32)
        g2 = (g2 + (dx * dx).astype(F32)).astype(F32)
        g2 = (g2 + (dy * dy).astype(F32)).astype(F32)
    return np.sqrt(g2).astype(F32)


def init_weights_fp32(img, lam):
    """P_init(x) = (1 - lam) |grad I(x)| / sum |grad I| + lam / (H W)
    (Sec. 4.4, Eq. P_init).  The normaliser is summed exactly: each |grad I|
    rounded to a 2^-32 fixed-point integer, summed in int64, converted back
    (so the result does not depend on summation order)."""
    g = grad_magnitude_fp32(img).ravel()
    P = g.size
    fx = np.rint((g.astype(F32) * F32(2.0 ** 32)).astype(F32)).astype(np.int64)
    S = F32(float(int(fx.sum())) * 2.0 ** -32)
    a = F32(F32(1.0) - F32(lam))
    b = F32(F32(lam) / F32(P))
    if S > 0:
        t = (g / S).astype(F32)
    else:
        t = np.zeros_like(g)
    return ((a * t).astype(F32) + b).astype(F32)


def _u24(seed, counters):
    """24-bit uniform draws u = hi24(SplitMix64) * 2^-24 in [0, 1)."""
    h = splitmix64(seed, counters)
    return ((h >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(F32)


def init_keys_fp32(w, seed):
    """Efraimidis-Spirakis (2006) weighted sampling without replacement: key =
    E / w with E = -log(U) ~ Exp(1), U in (0, 1] the 24-bit draw at counter =
    pixel index (+2^-24); the n smallest keys form the sample.  w = 0 gives
    +inf.  float32 throughout."""
    P = len(w)
    u = (_u24(seed, np.arange(P, dtype=np.uint64)) + F32(2.0 ** -24)).astype(F32)
    E = (-log32(u)).astype(F32)
    E = np.where(u == F32(1.0), F32(0.0), E).astype(F32)
    with np.errstate(divide="ignore", invalid="ignore"):
        k = (E / w).astype(F32)
    return np.where(w > F32(0), k, F32(np.inf)).astype(F32)


def init_select(keys, n):
    """Indices of the n smallest keys, ties by smaller index, returned in
    ascending index order."""
    order = np.lexsort((np.arange(len(keys)), keys))
    return np.sort(order[:n])


def init_sites(img, n, capacity, lam, seed, log_tau0):
    """Site set of Sec. 4.4: positions sampled at pixel centres by P_init
    (without replacement) plus a U[-0.25, 0.25) jitter per axis (24-bit draws
    at counters 2^40 + 2 pixel + {0, 1}), colour = target at the pixel, and
    the fixed defaults log_tau = log_tau0, r = 0, u = (1, 0), a = b = 0.
    Sites n..capacity-1 are inactive.  Returns float32[11, capacity]."""
    I = np.asarray(img, dtype=F32)
    H, W, _ = I.shape
    n = min(n, H * W)
    w = init_weights_fp32(I, lam)
    pix = init_select(init_keys_fp32(w, seed), n)
    row, col = np.divmod(pix, W)
    cnt = np.uint64(1 << 40) + np.uint64(2) * pix.astype(np.uint64)
    jx = ((_u24(seed, cnt) - F32(0.5)).astype(F32) * F32(0.5)).astype(F32)
    jy = ((_u24(seed, cnt + np.uint64(1)) - F32(0.5)).astype(F32) * F32(0.5)).astype(F32)
    p = np.zeros((N_PARAMS, capacity), dtype=F32)
    p[PX, :n] = ((col.astype(F32) + F32(0.5)).astype(F32) + jx).astype(F32)
    p[PY, :n] = ((row.astype(F32) + F32(0.5)).astype(F32) + jy).astype(F32)
    p[PLOGTAU, :n] = F32(log_tau0)
    p[PCR:PCB + 1, :n] = I[row, col].T
    p[PUX, :] = 1.0
    p[PX, n:] = -1.0
    p[PY, n:] = -1.0
    return p


# =============================================================================
# Part 4: adaptive budget -- statistics, densify (split) and prune (Sec. 4.5;
# App. "Densification and Pruning")
# =============================================================================

STAT_NAMES = ("mass", "energy", "mx", "my", "mxx", "mxy", "myy", "removal")


def site_stats(params, H, W, ids, target):
    """Per-site statistics of one render, fp64, float64[8, N]:
      mass    m_i = sum_x w_i(x)                            (Sec. 4.5)
      energy  E_i = sum_x w_i(x) |c(x) - I(x)|^2            (Sec. 4.5)
      mx..myy residual-weighted moments of D = x - p_i with omega = w_i e(x):
              sum omega Dx, sum omega Dy, sum omega Dx^2, sum omega Dx Dy,
              sum omega Dy^2 (the 'weighted second moments' of the
              statistics pass; the zeroth moment is the energy)
      removal sum_x of the removal delta (Sec. 4.5, as removal_delta())."""
    p = np.asarray(params, dtype=np.float64)
    N = p.shape[1]
    px, py = pixel_centres(H, W)
    w, _, valid, sid = weights(p, H, W, ids, px, py)
    col = np.stack([p[PCR], p[PCG], p[PCB]], axis=1)
    c = np.einsum("qk,qkc->qc", w, col[sid])
    I = np.asarray(target, np.float64).reshape(-1, 3)
    e = ((c - I) ** 2).sum(1)
    om = w * e[:, None]
    dx = px[:, None] - p[PX][sid]
    dy = py[:, None] - p[PY][sid]
    out = np.zeros((8, N))
    vals = [w, om, om * dx, om * dy, om * dx * dx, om * dx * dy, om * dy * dy]
    flat = np.where(valid, sid, 0).ravel()
    for j, v in enumerate(vals):
        np.add.at(out[j], flat, np.where(valid, v, 0.0).ravel())
    out[7] = removal_delta(p, H, W, ids, target)
    return out


def sobel_direction(target, x, y):
    """Unit direction of the 3x3 Sobel gradient of the RGB-summed target at
    the pixel containing (x, y) (borders clamp); (1, 0) if it vanishes."""
    I = np.asarray(target, np.float64).sum(axis=2)
    H, W = I.shape
    c = min(max(int(math.floor(x)), 0), W - 1)
    r = min(max(int(math.floor(y)), 0), H - 1)
    at = lambda rr, cc: I[min(max(rr, 0), H - 1), min(max(cc, 0), W - 1)]
    gx = (at(r - 1, c + 1) + 2 * at(r, c + 1) + at(r + 1, c + 1)
          - at(r - 1, c - 1) - 2 * at(r, c - 1) - at(r + 1, c - 1))
    gy = (at(r + 1, c - 1) + 2 * at(r + 1, c) + at(r + 1, c + 1)
          - at(r - 1, c - 1) - 2 * at(r - 1, c) - at(r - 1, c + 1))
    n = math.hypot(gx, gy)
    return (1.0, 0.0) if n == 0 else (gx / n, gy / n)


def densify_prune_select(params, stats, densify_pct, prune_pct, alpha=0.7, eps=1e-8):
    """Which sites split and which are pruned (Sec. 4.5).

    Densify: among active sites with mass > 1 and residual energy > 0 (a
    site with no residual has nothing to split), the top floor(pct N_active)
    by s_i = E_i / max(m_i, eps)^alpha (ties to the smaller id).  Prune: among the
    other active sites, the bottom floor(pct N_active) by removal delta (ties
    to the smaller id).  Returns (densify ids ascending, prune ids ascending).
    """
    p = np.asarray(params)
    act = np.nonzero(p[PX] >= 0)[0]
    n_act = len(act)
    m, E, R = stats[0], stats[1], stats[7]
    cand = act[(m[act] > 1.0) & (E[act] > 0.0)]
    score = E[cand] / np.maximum(m[cand], eps) ** alpha
    nd = min(int(math.floor(densify_pct * n_act)), len(cand))
    dens = np.sort(cand[np.lexsort((cand, -score))[:nd]]) if nd > 0 else np.zeros(0, np.int64)
    rest = np.setdiff1d(act, dens)
    npr = min(int(math.floor(prune_pct * n_act)), len(rest))
    prune = np.sort(rest[np.lexsort((rest, R[rest]))[:npr]]) if npr > 0 else np.zeros(0, np.int64)
    return dens, prune


def split_site(params, stats, target, i, H, W):
    """The two children of site i (Sec. 4.5; App. "Densification and Pruning"):
    residual-weighted centroid mu and covariance C from the moments; axis =
    major eigenvector of C (sign: positive x component, or positive y when x
    is 0) and a = -log(l1/l2)/2 clamped to [-2, 2] (u = axis);
    if the energy is below 1e-6 or l1/l2 < 1.01 the axis is the Sobel
    gradient direction of the target, the centre the parent position and
    a = 0.8 a_parent (u kept).  Children at centre +- d axis,
    d = clamp(0.5 sqrt(m_i), 1.5, 48) px, clamped to the image; both inherit
    the parent, log_tau -= 0.25, r *= 0.85, colour = target at the child.
    Returns two float64[11] parameter vectors (plus, minus)."""
    p = np.asarray(params, dtype=np.float64)[:, i].copy()
    st = stats[:, i]
    S0 = st[1]
    use_cov = False
    if S0 >= 1e-6:
        mux, muy = st[2] / S0, st[3] / S0
        C = np.array([[st[4] / S0 - mux * mux, st[5] / S0 - mux * muy],
                      [st[5] / S0 - mux * muy, st[6] / S0 - muy * muy]])
        lam, vec = np.linalg.eigh(C)
        l1, l2 = lam[1], lam[0]
        if l1 > 0 and l1 / max(l2, 1e-12) >= 1.01:
            use_cov = True
            axis = vec[:, 1]
            if axis[0] < 0 or (axis[0] == 0 and axis[1] < 0):   # canonical sign
                axis = -axis
            centre = (p[PX] + mux, p[PY] + muy)
            a_new = float(np.clip(-0.5 * math.log(l1 / max(l2, 1e-12)), -2.0, 2.0))
    if not use_cov:
        axis = np.array(sobel_direction(target, p[PX], p[PY]))
        centre = (p[PX], p[PY])
        a_new = 0.8 * p[PA]
    d = min(max(0.5 * math.sqrt(max(st[0], 0.0)), 1.5), 48.0)
    I = np.asarray(target, np.float64)
    kids = []
    for sgn in (1.0, -1.0):
        q = p.copy()
        q[PX] = min(max(centre[0] + sgn * d * axis[0], 0.0), float(W))
        q[PY] = min(max(centre[1] + sgn * d * axis[1], 0.0), float(H))
        q[PLOGTAU] -= 0.25
        q[PR] *= 0.85
        q[PA] = a_new
        if use_cov:
            q[PUX], q[PUY] = axis[0], axis[1]
        cc = min(max(int(math.floor(q[PX])), 0), W - 1)
        rr = min(max(int(math.floor(q[PY])), 0), H - 1)
        q[PCR:PCB + 1] = I[rr, cc]
        kids.append(q)
    return kids[0], kids[1]


def densify_prune(params, m, v, stats, target, H, W, densify_pct, prune_pct, alpha=0.7):
    """Apply one densify-then-prune event.  Parent i becomes the '+' child;
    the k-th split parent (ascending id) takes the k-th inactive slot
    (ascending) for its '-' child, and parents beyond the free slots are not
    split.  Adam state of parents and children is zeroed; pruned sites are set
    to (-1, -1).  Returns (params, m, v, n_active) as float64."""
    p = np.array(params, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    dens, prune = densify_prune_select(p, stats, densify_pct, prune_pct, alpha)
    free = np.nonzero(p[PX] < 0)[0]
    base = p.copy()
    for k, i in enumerate(dens):
        if k >= len(free):
            break
        plus, minus = split_site(base, stats, target, i, H, W)
        j = free[k]
        p[:, i], p[:, j] = plus, minus
        for arr in (m, v):
            arr[:, i] = 0.0
            arr[:, j] = 0.0
    p[PX, prune] = -1.0
    p[PY, prune] = -1.0
    return p, m, v, int((p[PX] >= 0).sum())


# ---------------------------------------------------------------------------
# Part 5: packed 16-byte evaluation sites (App. "Data Layout and Packing",
# Packed storage for evaluation)
# ---------------------------------------------------------------------------
# Four 32-bit words per site:
#   w0  x, y as 15-bit UNORM of x/W, y/H (bits 0-14, 15-29), active flag bit 31
#   w1  colour r, g, b as 11/11/10-bit UNORM with per-image min/scale
#   w2  (log tau, r) as 16/16-bit UNORM with per-image min/scale
#   w3  bits 0-15: the angle of u as a 16-bit UNORM code over [-pi, pi];
#       bits 16-31: a as float16
# The per-image min and max of log tau, r and the colour channels (over the
# active sites) are kept beside the words: q = float32[10] (lo, hi) x 5.
# The paper's sites have no b; b is folded into (log tau, r) exactly, since
# tau s (r - e^{b/2} n0) = (tau e^{b/2}) s (r e^{-b/2} - n0): log tau' =
# log tau + b/2, r' = r e^{-b/2}, b' = 0.  Quantisation arithmetic is carried
# out in float64 from the float32 inputs (codes = round half to even).

PACK_BITS = (16, 16, 11, 11, 10)   # log tau, r, colour r, g, b


def _fold_b(p):
    """float32 (log tau', r') with b folded in (float64 arithmetic)."""
    lt = (p[PLOGTAU].astype(np.float64) + p[PB].astype(np.float64) / 2.0).astype(np.float32)
    rr = (p[PR].astype(np.float64) * np.exp(-p[PB].astype(np.float64) / 2.0)).astype(np.float32)
    return lt, rr


def _code(v, lo, hi, bits):
    """UNORM code of float32 v in [lo, hi] (float64 arithmetic)."""
    top = float((1 << bits) - 1)
    d = float(hi) - float(lo)
    if d <= 0.0:
        return np.zeros(np.shape(v), dtype=np.uint32)
    t = (np.asarray(v, np.float64) - float(lo)) / d * top
    return np.rint(np.clip(t, 0.0, top)).astype(np.uint32)


def _uncode(c, lo, hi, bits):
    top = float((1 << bits) - 1)
    return (float(lo) + np.asarray(c, np.float64) / top * (float(hi) - float(lo))).astype(np.float32)


def pack_eval(params, H, W):
    """Pack float32[11, N] sites: returns (uint32[N, 4] words, float32[10] q)."""
    p = np.asarray(params, dtype=np.float32)
    N = p.shape[1]
    act = p[PX] >= 0
    lt, rr = _fold_b(p)
    vals = (lt, rr, p[PCR], p[PCG], p[PCB])
    q = np.zeros(10, dtype=np.float32)
    for i, v in enumerate(vals):
        if act.any():
            q[2 * i], q[2 * i + 1] = v[act].min(), v[act].max()
    codes = [_code(v, q[2 * i], q[2 * i + 1], PACK_BITS[i]) for i, v in enumerate(vals)]
    xq = np.rint(np.clip(p[PX].astype(np.float64) / W, 0.0, 1.0) * 32767.0).astype(np.uint32)
    yq = np.rint(np.clip(p[PY].astype(np.float64) / H, 0.0, 1.0) * 32767.0).astype(np.uint32)
    th = np.arctan2(p[PUY].astype(np.float64), p[PUX].astype(np.float64))
    aq = np.rint(np.clip((th + math.pi) / (2.0 * math.pi), 0.0, 1.0) * 65535.0).astype(np.uint32)
    ah = p[PA].astype(np.float16).view(np.uint16).astype(np.uint32)
    w = np.zeros((N, 4), dtype=np.uint32)
    w[:, 0] = xq | (yq << np.uint32(15)) | (np.uint32(1) << np.uint32(31))
    w[:, 1] = codes[2] | (codes[3] << np.uint32(11)) | (codes[4] << np.uint32(22))
    w[:, 2] = codes[0] | (codes[1] << np.uint32(16))
    w[:, 3] = aq | (ah << np.uint32(16))
    w[~act] = 0
    return w, q


def unpack_eval(words, q, H, W):
    """float32[11, N] sites from packed words (b = 0; inactive: x = y = -1)."""
    w = np.asarray(words, dtype=np.uint32)
    N = w.shape[0]
    p = np.zeros((N_PARAMS, N), dtype=np.float32)
    act = (w[:, 0] >> np.uint32(31)) & np.uint32(1) == 1
    p[PX] = ((w[:, 0] & np.uint32(0x7FFF)).astype(np.float64) / 32767.0 * W).astype(np.float32)
    p[PY] = (((w[:, 0] >> np.uint32(15)) & np.uint32(0x7FFF)).astype(np.float64) / 32767.0 * H).astype(np.float32)
    p[PLOGTAU] = _uncode(w[:, 2] & np.uint32(0xFFFF), q[0], q[1], 16)
    p[PR] = _uncode(w[:, 2] >> np.uint32(16), q[2], q[3], 16)
    p[PCR] = _uncode(w[:, 1] & np.uint32(0x7FF), q[4], q[5], 11)
    p[PCG] = _uncode((w[:, 1] >> np.uint32(11)) & np.uint32(0x7FF), q[6], q[7], 11)
    p[PCB] = _uncode(w[:, 1] >> np.uint32(22), q[8], q[9], 10)
    th = (w[:, 3] & np.uint32(0xFFFF)).astype(np.float64) / 65535.0 * (2.0 * math.pi) - math.pi
    p[PUX] = np.cos(th).astype(np.float32)
    p[PUY] = np.sin(th).astype(np.float32)
    p[PA] = (w[:, 3] >> np.uint32(16)).astype(np.uint16).view(np.float16).astype(np.float32)
    p[PX, ~act] = -1.0
    p[PY, ~act] = -1.0
    return p


# ---------------------------------------------------------------------------
# Part 6: tau diffusion (App. "Tau Diffusion")
# ---------------------------------------------------------------------------

def tau_diffusion(params, H, W, ids, lam, g_logtau):
    """One Jacobi step that smooths the log tau gradients over each site's
    candidate neighbourhood: g'_i = (1 - lam) g_i + lam * mean_{j in N(i)} g_j,
    N(i) = the valid, active sites other than i listed at the pixel that
    contains site i (position clamped into the image).  Inactive sites and
    sites with an empty neighbourhood keep their gradient.  fp64; returns
    float64[N]."""
    p = np.asarray(params, dtype=np.float64)
    g = np.asarray(g_logtau, dtype=np.float64)
    ids = np.asarray(ids)
    N = p.shape[1]
    out = g.copy()
    for i in range(N):
        if not p[PX, i] >= 0:
            continue
        col = min(max(int(math.floor(p[PX, i])), 0), W - 1)
        row = min(max(int(math.floor(p[PY, i])), 0), H - 1)
        nb = [int(j) for j in ids[row * W + col]
              if int(j) != INVALID and int(j) < N and int(j) != i and p[PX, int(j)] >= 0]
        if nb:
            out[i] = (1.0 - lam) * g[i] + lam * float(np.mean(g[nb]))
    return out


# ---------------------------------------------------------------------------
# Part 7: half2 candidate sites (App. "Data Layout and Packing", Packed
# candidate sites)
# ---------------------------------------------------------------------------

HALF_MAX = 65504.0   # largest finite IEEE binary16 value
_CAND_FIELDS = ("x", "y", "ts", "r", "G00", "G01", "G11", "active")


def candidate_halves(prep):
    """The 16-byte candidate record of every site as float16[N, 8]: the
    scoring values x, y, tau s, r, G00, G01, G11 and the active flag (1 or 0)
    of the float32 table, each saturated to [-HALF_MAX, HALF_MAX] (NaN-
    ignoring min/max, like C's fminf/fmaxf) and rounded to the nearest
    binary16 value, ties to even (IEEE 754 conversion)."""
    cols = []
    for f in _CAND_FIELDS:
        v = prep[f].astype(F32)
        v = np.fmin(np.fmax(v, F32(-HALF_MAX)), F32(HALF_MAX)).astype(F32)
        cols.append(v.astype(np.float16))
    return np.stack(cols, axis=1)


def candidate_words(prep):
    """candidate_halves as the record's four little-endian 32-bit words
    (first value of each pair in the low 16 bits): uint32[N, 4]."""
    h = np.ascontiguousarray(candidate_halves(prep))
    bits = h.view(np.uint16).astype(np.uint32)
    return bits[:, 0::2] | (bits[:, 1::2] << np.uint32(16))


def candidate_table_fp32(prep):
    """The table a half2 candidate pass scores from: prepare_fp32's dict with
    the scoring values replaced by their binary16 records widened back to
    float32 (exact), and active = record flag != 0.  Passing it to
    topk_pass_fp32 is the candidate pass on half2 sites."""
    h = candidate_halves(prep).astype(F32)
    out = dict(prep)
    for k, f in enumerate(_CAND_FIELDS[:-1]):
        out[f] = h[:, k].copy()
    out["active"] = h[:, 7] != F32(0)
    return out


# =============================================================================
# Part 8: 1-D SAD (Sec. "1D Signal Fitting"), fp64
# =============================================================================
# Each site of a 1-D signal has a position p (samples), a value c, a log
# temperature and a radius r (four parameters).  The 2-D score with the 1-D
# distance: sample k sits at x = k + 0.5, s = 1/L, d_i(x) = |x - p_i| s -
# r_i s, l_i(x) = -tau_i d_i(x) (Sec. 4.1-4.2); the value at x is the softmax
# blend over the K sites of largest logit (ties to the smaller index; K = N
# blends over every site: the soft partition of unity of the paper's 64-site
# fits).  Parameters: float[4, N] planes (p, c, log_tau, r).

P1_P, P1_C, P1_LOGTAU, P1_R = range(4)
SAD1D_PLANES = ("p", "c", "log_tau", "r")
SAD1D_LR = {"p": 2e-3, "c": 1e-2, "log_tau": 1e-2, "r": 1e-3}


def sad1d_samples(L):
    """Sample centres x_k = k + 0.5 of a signal of L samples."""
    return np.arange(L, dtype=np.float64) + 0.5


def sad1d_logits(params, L, xs=None):
    """l_i(x) = -tau_i (|x - p_i| s - r_i s), float64[X, N]."""
    p = np.asarray(params, dtype=np.float64)
    xs = sad1d_samples(L) if xs is None else np.asarray(xs, dtype=np.float64)
    s = 1.0 / L
    tau = np.exp(p[P1_LOGTAU])
    d = np.abs(xs[:, None] - p[P1_P][None, :]) * s - p[P1_R][None, :] * s
    return -tau[None, :] * d


def sad1d_topk(params, L, K, xs=None):
    """Indices of the K largest logits per sample (ties to the smaller index):
    int64[X, min(K, N)]."""
    ell = sad1d_logits(params, L, xs)
    X, N = ell.shape
    kk = min(K, N)
    idx = np.broadcast_to(np.arange(N), (X, N))
    sel = select_topk(idx, ell, np.ones(ell.shape, bool), kk)
    return sel.astype(np.int64)


def sad1d_render(params, L, K, xs=None):
    """Blended value per sample: float64[X]."""
    p = np.asarray(params, dtype=np.float64)
    ell = sad1d_logits(p, L, xs)
    ids = sad1d_topk(p, L, K, xs)
    l = np.take_along_axis(ell, ids, axis=1)
    w = np.exp(l - l.max(axis=1, keepdims=True))
    w /= w.sum(axis=1, keepdims=True)
    return (w * p[P1_C][ids]).sum(axis=1)


def sad1d_backward(params, L, K, g, xs=None):
    """Adjoint of the 1-D blend for upstream dL/dc(x) = g (float[X]), with the
    top-K sets held fixed: float64[4, N] gradients.  Per sample and listed
    site: dL/dc_i = w_i g; delta_i = w_i g (c_i - cbar) = dL/dl_i; dl/dlog_tau
    = l; dl/dr = tau s; dl/dp = tau s sign(x - p) (0 at x = p, where the
    distance has its kink)."""
    p = np.asarray(params, dtype=np.float64)
    xs = sad1d_samples(L) if xs is None else np.asarray(xs, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    ell = sad1d_logits(p, L, xs)
    ids = sad1d_topk(p, L, K, xs)
    l = np.take_along_axis(ell, ids, axis=1)
    w = np.exp(l - l.max(axis=1, keepdims=True))
    w /= w.sum(axis=1, keepdims=True)
    ck = p[P1_C][ids]
    cbar = (w * ck).sum(axis=1, keepdims=True)
    delta = w * g[:, None] * (ck - cbar)
    s = 1.0 / L
    tau = np.exp(p[P1_LOGTAU])[ids]
    sgn = np.sign(xs[:, None] - p[P1_P][ids])
    N = p.shape[1]
    out = np.zeros((4, N))
    np.add.at(out[P1_C], ids, w * g[:, None])
    np.add.at(out[P1_LOGTAU], ids, delta * l)
    np.add.at(out[P1_R], ids, delta * tau * s)
    np.add.at(out[P1_P], ids, delta * tau * s * sgn)
    return out


def sad1d_loss_and_grad(values, target):
    """L = mean over samples of (c(x) - y(x))^2 and dL/dc = 2 (c - y) / L."""
    r = np.asarray(values, dtype=np.float64) - np.asarray(target, dtype=np.float64)
    return float(np.mean(r * r)), 2.0 * r / len(r)


def sad1d_adam_step(params, grads, m, v, t, L, lr=None, beta1=0.9, beta2=0.999, eps=1e-8,
                    log_tau_range=(2.0, 20.0)):
    """One bias-corrected Adam step (Kingma & Ba 2015) of the 1-D sites, with
    the 2-D conventions of Sec. 6.1: p and r optimised in normalised units
    (value * s: gradient / s, step / s), p clamped to [0, L], r to [0, L],
    log_tau to [2, 20]; values unclamped.  Returns new (params, m, v), fp64."""
    lr = dict(SAD1D_LR if lr is None else lr)
    p = np.array(params, dtype=np.float64)
    g = np.asarray(grads, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    s = 1.0 / L
    for j, name in enumerate(SAD1D_PLANES):
        unit = s if j in (P1_P, P1_R) else 1.0
        gj = g[j] / unit
        m[j] = beta1 * m[j] + (1 - beta1) * gj
        v[j] = beta2 * v[j] + (1 - beta2) * gj * gj
        mhat = m[j] / (1 - beta1 ** t)
        vhat = v[j] / (1 - beta2 ** t)
        p[j] = p[j] - lr[name] * mhat / (np.sqrt(vhat) + eps) / unit
    p[P1_P] = np.clip(p[P1_P], 0.0, float(L))
    p[P1_R] = np.clip(p[P1_R], 0.0, float(L))
    p[P1_LOGTAU] = np.clip(p[P1_LOGTAU], *log_tau_range)
    return p, m, v


def sad1d_train_step(params, m, v, t, target, K, lr=None):
    """One 1-D training iteration: render over the top-K sets, MSE, adjoint,
    Adam.  Returns (params, m, v, loss, grads), fp64."""
    L = len(target)
    vals = sad1d_render(params, L, K)
    loss, g = sad1d_loss_and_grad(vals, target)
    grads = sad1d_backward(params, L, K, g)
    p2, m2, v2 = sad1d_adam_step(params, grads, m, v, t, L, lr)
    return p2, m2, v2, loss, grads
