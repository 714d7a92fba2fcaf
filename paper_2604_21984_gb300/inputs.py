"""Seeded synthetic inputs for Soft Anisotropic Diagrams (SAD).

This module is the only code that the CUDA path and the CPU oracle share.
It draws random images, random site sets and random top-K index maps from
numpy's PCG64 and holds none of the method's arithmetic: no metric, no score,
no softmax, no propagation.  Every function is deterministic in its seed.

Site parameters use the 11-plane structure-of-arrays layout of the C-ABI
(``float32[11][capacity]``), plane order::

    0 x   1 y   2 log_tau   3 r   4 cr   5 cg   6 cb   7 ux   8 uy   9 a   10 b

Positions and radii are in pixels; pixel (col, row) has its centre at
(col + 0.5, row + 0.5).  ``b`` is a log isotropic metric scale (b = 0 gives the
unit-determinant metric of the paper's site representation, Sec. 4.1).
An inactive site has x < 0 (the paper stores (-1, -1), App. "Data Layout and Packing", Site buffer).

Index maps are ``uint32[P, K]`` (pixel-major, P = H*W, row-major pixels) with
the invalid sentinel 0xffffffff (App. "Data Layout and Packing", Top-K candidate list).
"""
from __future__ import annotations

import math

import numpy as np

N_PARAMS = 11
PX, PY, PLOGTAU, PR, PCR, PCG, PCB, PUX, PUY, PA, PB = range(N_PARAMS)
PARAM_NAMES = ("x", "y", "log_tau", "r", "cr", "cg", "cb", "ux", "uy", "a", "b")
INVALID = np.uint32(0xFFFFFFFF)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# images
# ----------------------------------------------------------------------------

def _fill_polygon(img, verts, colour):
    """Even-odd fill at pixel centres of one polygon (vertices in pixels)."""
    H, W, _ = img.shape
    x0 = max(int(math.floor(verts[:, 0].min())), 0)
    x1 = min(int(math.ceil(verts[:, 0].max())) + 1, W)
    y0 = max(int(math.floor(verts[:, 1].min())), 0)
    y1 = min(int(math.ceil(verts[:, 1].max())) + 1, H)
    if x0 >= x1 or y0 >= y1:
        return
    py, px = np.mgrid[y0:y1, x0:x1].astype(np.float64) + 0.5
    inside = np.zeros(px.shape, dtype=bool)
    nv = len(verts)
    for e in range(nv):
        xa, ya = verts[e]
        xb, yb = verts[(e + 1) % nv]
        crosses = (ya > py) != (yb > py)
        with np.errstate(divide="ignore", invalid="ignore"):
            xint = xa + (py - ya) * (xb - xa) / (yb - ya)
        inside ^= crosses & (px < xint)
    img[y0:y1, x0:x1][inside] = colour


def _random_polygon(g, H, W, rmin, rmax):
    cx, cy = g.uniform(0, W), g.uniform(0, H)
    rad = g.uniform(rmin, rmax) * max(H, W)
    nv = int(g.integers(3, 9))
    ang = g.uniform(0, 2 * math.pi, nv)
    rr = rad * g.uniform(0.3, 1.0, nv)
    return np.stack([cx + rr * np.cos(ang), cy + rr * np.sin(ang)], axis=1)


def image_sinusoid_polygons(H: int = 64, W: int = 64, seed: int = 1000,
                            n_polygons: int = 12) -> np.ndarray:
    """Smooth 2-D sinusoid gradients plus filled random polygons, in [0,1].

    I_c = 0.5 + 0.25 sin(2 pi (fx x + fy y) + phi) per channel with
    (fx, fy) ~ U[1,4]/W, then ``n_polygons`` polygons (3-8 vertices,
    even-odd fill at pixel centres, colour U[0,1]^3), clipped to [0,1].
    Returns float32[H, W, 3].
    """
    g = rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64) + 0.5
    img = np.empty((H, W, 3), dtype=np.float64)
    for c in range(3):
        fx, fy = g.uniform(1, 4, 2) / W
        phi = g.uniform(0, 2 * math.pi)
        img[..., c] = 0.5 + 0.25 * np.sin(2 * math.pi * (fx * xx + fy * yy) + phi)
    for _ in range(n_polygons):
        verts = _random_polygon(g, H, W, 0.08, 0.35)
        _fill_polygon(img, verts, g.uniform(0, 1, 3))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def _draw_segment(img, x0, y0, x1, y1, width, colour, bx0, bx1, by0, by1):
    """Paint the pixels whose centre lies within width/2 of the segment.
    Works in strips of 64 rows, each restricted to the columns the segment can
    reach inside the strip (a margin of one pixel beyond the exact reach), so
    a long diagonal stroke costs its area, not its bounding box."""
    dx, dy = x1 - x0, y1 - y0
    L2 = dx * dx + dy * dy + 1e-12
    half = 0.5 * width
    for r0 in range(by0, by1, 64):
        r1 = min(r0 + 64, by1)
        ylo, yhi = r0 + 0.5 - half, r1 - 0.5 + half
        if abs(dy) < 1e-12:
            if not ylo <= y0 <= yhi:
                continue
            tlo, thi = 0.0, 1.0
        else:
            ta, tb = (ylo - y0) / dy, (yhi - y0) / dy
            tlo, thi = max(0.0, min(ta, tb)), min(1.0, max(ta, tb))
            if tlo > thi:
                continue
        xa, xb = sorted((x0 + tlo * dx, x0 + thi * dx))
        c0 = max(bx0, int(math.floor(xa - half - 1.5)))
        c1 = min(bx1, int(math.ceil(xb + half + 1.5)) + 1)
        if c0 >= c1:
            continue
        py, px = np.mgrid[r0:r1, c0:c1].astype(np.float64) + 0.5
        t = np.clip(((px - x0) * dx + (py - y0) * dy) / L2, 0, 1)
        dist = np.hypot(px - (x0 + t * dx), py - (y0 + t * dy))
        img[r0:r1, c0:c1][dist <= half] = colour


def _value_noise(g, H, W, cell):
    """One octave of bilinear value noise with lattice spacing ``cell``."""
    ny, nx = H // cell + 2, W // cell + 2
    lat = g.uniform(0, 1, (ny, nx, 3))
    ys = (np.arange(H) + 0.5) / cell
    xs = (np.arange(W) + 0.5) / cell
    iy, ix = ys.astype(int), xs.astype(int)
    ty, tx = (ys - iy)[:, None, None], (xs - ix)[None, :, None]
    ty, tx = ty * ty * (3 - 2 * ty), tx * tx * (3 - 2 * tx)
    # separable: interpolate each lattice row along x, then rows along y
    # (the same products and sums per pixel as the 4-corner form)
    rows = lat[:, ix] * (1 - tx) + lat[:, ix + 1] * tx
    return rows[iy] * (1 - ty) + rows[iy + 1] * ty


def image_noise_polygons_lines(H: int = 512, W: int = 768, seed: int = 2000,
                               n_polygons: int = 40, n_lines: int = 24) -> np.ndarray:
    """Multi-octave value noise plus random polygons and thin 1-3 px lines.

    5 octaves, base lattice cell 64 px, persistence 0.5; then ``n_polygons``
    filled polygons and ``n_lines`` straight strokes of width U{1,2,3} px.
    Returns float32[H, W, 3] in [0,1].
    """
    g = rng(seed)
    img = np.zeros((H, W, 3), dtype=np.float64)
    amp, total, cell = 1.0, 0.0, 64
    for _ in range(5):
        img += amp * _value_noise(g, H, W, max(cell, 1))
        total += amp
        amp *= 0.5
        cell //= 2
    img /= total
    for _ in range(n_polygons):
        _fill_polygon(img, _random_polygon(g, H, W, 0.02, 0.15), g.uniform(0, 1, 3))
    for _ in range(n_lines):
        x0, x1 = g.uniform(0, W, 2)
        y0, y1 = g.uniform(0, H, 2)
        width = float(g.integers(1, 4))
        colour = g.uniform(0, 1, 3)
        bx0 = max(int(min(x0, x1) - width - 1), 0)
        bx1 = min(int(max(x0, x1) + width + 2), W)
        by0 = max(int(min(y0, y1) - width - 1), 0)
        by1 = min(int(max(y0, y1) + width + 2), H)
        if bx0 >= bx1 or by0 >= by1:
            continue
        _draw_segment(img, x0, y0, x1, y1, width, colour, bx0, bx1, by0, by1)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


# ----------------------------------------------------------------------------
# site sets
# ----------------------------------------------------------------------------

def _colour_at(img, x, y):
    H, W, _ = img.shape
    col = np.clip(np.floor(x).astype(np.int64), 0, W - 1)
    row = np.clip(np.floor(y).astype(np.int64), 0, H - 1)
    return img[row, col]


def sites_isotropic(img: np.ndarray, n: int, seed: int, scale_px: float = 4.0,
                    tau: float = 1.0, radius: float = 0.0,
                    capacity: int | None = None) -> np.ndarray:
    """Uniform random positions, isotropic metric of scale ``scale_px``.

    'Isotropic metric scale s px' means |x - p|_G = |x - p| / s, i.e. a = 0,
    b = -2 ln s, u = (1, 0).  Temperature ``tau`` (log_tau = ln tau), additive
    radius ``radius`` px, colour = image at the site's pixel.  Sites beyond
    ``n`` up to ``capacity`` are inactive.  Returns float32[11, capacity].
    """
    H, W, _ = img.shape
    cap = n if capacity is None else capacity
    g = rng(seed)
    p = np.zeros((N_PARAMS, cap), dtype=np.float64)
    p[PX, :n] = g.uniform(0, W, n)
    p[PY, :n] = g.uniform(0, H, n)
    p[PLOGTAU, :n] = math.log(tau)
    p[PR, :n] = radius
    p[PCR:PCB + 1, :n] = _colour_at(img, p[PX, :n], p[PY, :n]).T
    p[PUX, :n] = 1.0
    p[PUY, :n] = 0.0
    p[PA, :n] = 0.0
    p[PB, :n] = -2.0 * math.log(scale_px)
    _mark_inactive(p, np.arange(n, cap))
    return p.astype(np.float32)


def sites_random_spd(H: int, W: int, n: int, seed: int,
                     capacity: int | None = None) -> np.ndarray:
    """Random anisotropic sites (differentiation workload).

    Positions uniform over the image; metric log-eigenvalues lam1, lam2 ~
    U[-2, 2] along u = (cos t, sin t), t ~ U[0, pi), stored as a = (lam1 -
    lam2)/2, b = (lam1 + lam2)/2; radius ~ N(0, 2) px; temperature
    log-uniform on [0.1, 10]; colours U[0,1]^3.  Returns float32[11, capacity].
    """
    cap = n if capacity is None else capacity
    g = rng(seed)
    p = np.zeros((N_PARAMS, cap), dtype=np.float64)
    p[PX, :n] = g.uniform(0, W, n)
    p[PY, :n] = g.uniform(0, H, n)
    lam = g.uniform(-2, 2, (2, n))
    th = g.uniform(0, math.pi, n)
    p[PLOGTAU, :n] = g.uniform(math.log(0.1), math.log(10.0), n)
    p[PR, :n] = g.normal(0.0, 2.0, n)
    p[PCR:PCB + 1, :n] = g.uniform(0, 1, (3, n))
    p[PUX, :n] = np.cos(th)
    p[PUY, :n] = np.sin(th)
    p[PA, :n] = 0.5 * (lam[0] - lam[1])
    p[PB, :n] = 0.5 * (lam[0] + lam[1])
    _mark_inactive(p, np.arange(n, cap))
    return p.astype(np.float32)


def _mark_inactive(p, idx):
    p[PX, idx] = -1.0
    p[PY, idx] = -1.0


def deactivate_random(params: np.ndarray, frac: float, seed: int) -> np.ndarray:
    """Copy of ``params`` with a random fraction of sites set inactive."""
    g = rng(seed)
    q = params.copy()
    n = q.shape[1]
    idx = g.choice(n, size=int(frac * n), replace=False)
    q[PX, idx] = -1.0
    q[PY, idx] = -1.0
    return q


# ----------------------------------------------------------------------------
# index maps
# ----------------------------------------------------------------------------

def knn_map(params: np.ndarray, H: int, W: int, K: int, seed: int,
            truncate_frac: float = 0.0, shuffle: bool = False,
            include_inactive_frac: float = 0.0, pixels=None) -> np.ndarray:
    """Spatially coherent random top-K index map (uint32[P, K]; with
    ``pixels``, only those pixel indices: uint32[len(pixels), K]).

    Each pixel lists the K sites whose positions are nearest to its centre in
    plain Euclidean distance (scipy cKDTree; this is not the method's score).
    Optional perturbations for edge cases: ``truncate_frac`` of the pixels keep
    only a random prefix (the rest is the invalid sentinel), ``shuffle``
    permutes each list, ``include_inactive_frac`` of the pixels get one entry
    replaced by an inactive site id (if any exists).
    """
    from scipy.spatial import cKDTree

    g = rng(seed)
    pix = np.arange(H * W) if pixels is None else np.asarray(pixels, dtype=np.int64)
    P = len(pix)
    active = np.nonzero(params[PX] >= 0)[0]
    ids = np.full((P, K), INVALID, dtype=np.uint32)
    kk = min(K, len(active))
    if kk > 0:
        tree = cKDTree(np.stack([params[PX, active], params[PY, active]], 1).astype(np.float64))
        yy, xx = np.divmod(pix, W)
        q = np.stack([xx + 0.5, yy + 0.5], 1)
        _, nn = tree.query(q, k=kk, workers=-1)
        nn = nn.reshape(P, kk)
        ids[:, :kk] = active[nn].astype(np.uint32)
    if shuffle:
        perm = np.argsort(g.random((P, K)), axis=1)
        ids = np.take_along_axis(ids, perm, axis=1)
    if truncate_frac > 0:
        rows = np.nonzero(g.random(P) < truncate_frac)[0]
        keep = g.integers(0, K, len(rows))
        for r_, k_ in zip(rows, keep):
            ids[r_, k_:] = INVALID
    if include_inactive_frac > 0:
        inactive = np.nonzero(params[PX] < 0)[0]
        if len(inactive):
            rows = np.nonzero(g.random(P) < include_inactive_frac)[0]
            cols = g.integers(0, K, len(rows))
            ids[rows, cols] = inactive[g.integers(0, len(inactive), len(rows))].astype(np.uint32)
    return ids


def random_map(P: int, K: int, n_sites: int, seed: int, invalid_frac: float = 0.1) -> np.ndarray:
    """Spatially incoherent map: K distinct random ids per pixel (uint32[P, K]).

    A fraction ``invalid_frac`` of the entries is replaced by the sentinel.
    Stresses the per-tile site tables (many distinct sites per tile).
    """
    g = rng(seed)
    assert n_sites >= K
    if n_sites <= 64:
        ids = np.argsort(g.random((P, n_sites)), axis=1)[:, :K].astype(np.uint32)
    else:
        # distinct by construction: strictly increasing offsets below n_sites
        span = max(1, min(8, (n_sites - 1) // K))
        offs = np.cumsum(g.integers(1, span + 1, (P, K)), axis=1)
        base = g.integers(0, n_sites, P)[:, None]
        ids = ((base + offs) % n_sites).astype(np.uint32)
        perm = np.argsort(g.random((P, K)), axis=1)
        ids = np.take_along_axis(ids, perm, axis=1)
    ids[g.random((P, K)) < invalid_frac] = INVALID
    return ids


def grad_image(H: int, W: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Upstream gradient dL/dc: float32[H, W, 3] ~ N(0, 1) * scale."""
    return (rng(seed).standard_normal((H, W, 3)) * scale).astype(np.float32)


def uniform_points(n: int, H: int, W: int, seed: int) -> np.ndarray:
    """Uniform float query coordinates in [0,W) x [0,H): float32[n, 2]."""
    g = rng(seed)
    return np.stack([g.uniform(0, W, n), g.uniform(0, H, n)], 1).astype(np.float32)


# ----------------------------------------------------------------------------
# workload mixes: uneven image batches and request streams
# ----------------------------------------------------------------------------

def _log_uniform(g, lo, hi):
    return math.exp(g.uniform(math.log(lo), math.log(hi)))


def batch_sizes(n: int, seed: int, lo: int = 256, hi: int = 2048,
                aspect=(1.0, 1.5)) -> list:
    """n image sizes (H, W): long side log-uniform in [lo, hi], aspect ratio
    uniform in `aspect`, short side round(long / ratio), orientation random."""
    g = rng(seed)
    out = []
    for _ in range(n):
        L = int(round(_log_uniform(g, lo, hi)))
        S = max(1, int(round(L / g.uniform(*aspect))))
        out.append((S, L) if g.uniform() < 0.5 else (L, S))
    return out


def serve_stream(seed: int, seconds: float, rate: float, decode_frac: float = 0.7,
                 n_residents: int = 4, coords=(1e3, 1e6), side=(128, 4096),
                 iters: int = 1000) -> list:
    """Poisson request stream: exponential inter-arrival times with mean
    1/rate until `seconds`; each request is a decode with probability
    decode_frac (a resident set index uniform in [0, n_residents), a
    log-uniform coordinate count in `coords`, a coordinate seed) or else an
    encode (square-ish image with log-uniform side in `side`, aspect in
    [1, 1.5], an image seed, `iters` iterations).  Returns a list of dicts
    sorted by arrival."""
    g = rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t >= seconds:
            break
        if g.uniform() < decode_frac:
            out.append(dict(kind="decode", arrival=t, resident=int(g.integers(0, n_residents)),
                            n=int(round(_log_uniform(g, *coords))), seed=int(g.integers(1 << 31))))
        else:
            L = int(round(_log_uniform(g, *side)))
            S = max(1, int(round(L / g.uniform(1.0, 1.5))))
            H, W = (S, L) if g.uniform() < 0.5 else (L, S)
            out.append(dict(kind="encode", arrival=t, H=H, W=W, seed=int(g.integers(1 << 31)),
                            iters=iters))
    return out


def resident_sets(seed: int, n: int, sites=(16384, 1 << 20), sites_per_pixel: float = 0.06) -> list:
    """n decode site sets: N log-uniform in `sites`, a square image of
    P = N / sites_per_pixel pixels, random anisotropic sites
    (sites_random_spd).  Returns [(H, W, N, site seed)]."""
    g = rng(seed)
    out = []
    for _ in range(n):
        N = int(round(_log_uniform(g, *sites)))
        side = max(1, int(round(math.sqrt(N / sites_per_pixel))))
        out.append((side, side, N, int(g.integers(1 << 31))))
    return out


# ----------------------------------------------------------------------------
# 1-D signals (Sec. "1D Signal Fitting")
# ----------------------------------------------------------------------------

def signals_1d(B: int, L: int, seed: int) -> np.ndarray:
    """B synthetic 1-D targets of L samples, float32[B, L]: the three target
    families of the paper's 1-D experiment, chosen per signal with seeded
    random parameters -- a smooth sine, a step plus a sine, and a
    multi-frequency periodic signal (three sines, frequencies 1..12 periods
    per signal).  Samples at t = (k + 0.5) / L."""
    g = rng(seed)
    t = (np.arange(L) + 0.5) / L
    kind = g.integers(0, 3, B)
    f = g.uniform(1.0, 4.0, (B, 1))
    ph = g.uniform(0.0, 2 * math.pi, (B, 3))
    amp = g.uniform(0.2, 0.5, (B, 1))
    smooth = 0.5 + amp * np.sin(2 * math.pi * f * t[None, :] + ph[:, :1])
    edge = g.uniform(0.25, 0.75, (B, 1))
    lo, hi = g.uniform(0.1, 0.4, (B, 1)), g.uniform(0.6, 0.9, (B, 1))
    step = np.where(t[None, :] < edge, lo, hi) + 0.1 * np.sin(2 * math.pi * 3 * f * t[None, :] + ph[:, 1:2])
    fr = g.uniform(1.0, 12.0, (B, 3))
    w = g.uniform(0.05, 0.25, (B, 3))
    multi = 0.5 + sum(w[:, j:j + 1] * np.sin(2 * math.pi * fr[:, j:j + 1] * t[None, :] + ph[:, j:j + 1])
                      for j in range(3))
    out = np.where((kind == 0)[:, None], smooth, np.where((kind == 1)[:, None], step, multi))
    return out.astype(np.float32)


def sites_1d(targets: np.ndarray, N: int) -> np.ndarray:
    """Initial 1-D sites for float[B, L] targets, float32[4, B*N] planes (p, c,
    log_tau, r): N sites per signal at the centres of N equal cells, each
    taking the target's value at its sample, tau with tau s (L/N) = 4, r = 0."""
    B, L = targets.shape
    p = np.zeros((4, B, N), dtype=np.float64)
    pos = (np.arange(N) + 0.5) * L / N
    p[0] = pos[None, :]
    p[1] = targets[:, np.minimum(pos.astype(np.int64), L - 1)]
    p[2] = math.log(4.0 * N)
    return p.reshape(4, B * N).astype(np.float32)
