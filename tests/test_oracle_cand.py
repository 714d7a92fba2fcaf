"""Pins of the oracle's half2 candidate sites (App. "Data Layout and
Packing", Packed candidate sites): binary16 bit patterns worked out by hand
from the IEEE 754 format, ties to even, saturation, the word layout, the
relative rounding bound of binary16, and the special case where every value
is a binary16 number (the half2 pass then equals the float32 pass)."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen


def _prep_one(o, **vals):
    """A one-site prepared dict with the given scoring values."""
    base = {"x": 0.0, "y": 0.0, "ts": 0.0, "r": 0.0, "G00": 0.0, "G01": 0.0, "G11": 0.0}
    base.update(vals)
    d = {k: np.float32([v]) for k, v in base.items()}
    d["active"] = np.array([vals.get("active", True)])
    for c in ("cr", "cg", "cb"):
        d[c] = np.float32([0.0])
    return d


def test_hand_worked_bit_patterns(oracle):
    """binary16: sign | 5-bit exponent (bias 15) | 10-bit fraction."""
    o = oracle
    # 1.0 = 0x3C00, 2.0 = 0x4000, 0.5 = 0x3800, -2.0 = 0xC000, 0 = 0x0000
    d = _prep_one(o, x=1.0, y=2.0, ts=0.5, r=-2.0, G00=0.0, G01=1.0, G11=2.0)
    w = o.candidate_words(d)
    assert w.dtype == np.uint32 and w.shape == (1, 4)
    assert int(w[0, 0]) == 0x3C00 | (0x4000 << 16)
    assert int(w[0, 1]) == 0x3800 | (0xC000 << 16)
    assert int(w[0, 2]) == 0x0000 | (0x3C00 << 16)
    assert int(w[0, 3]) == 0x4000 | (0x3C00 << 16)       # G11 = 2, active flag 1.0


def test_ties_to_even_and_saturation(oracle):
    o = oracle
    # In [2048, 4096) the binary16 spacing is 2: 2049 lies halfway between
    # 2048 (fraction 0, even) and 2050 (fraction 1, odd) -> 2048 = 0x6800;
    # 2051 lies between 2050 (odd) and 2052 (fraction 2, even) -> 0x6802.
    # 1e6 saturates to 65504 = 0x7BFF, -1e6 to -65504 = 0xFBFF.
    d = _prep_one(o, x=2049.0, y=2051.0, ts=1e6, r=-1e6, active=False)
    w = o.candidate_words(d)
    assert int(w[0, 0]) == 0x6800 | (0x6802 << 16)
    assert int(w[0, 1]) == 0x7BFF | (0xFBFF << 16)
    assert int(w[0, 3]) >> 16 == 0                        # inactive flag 0.0
    t = o.candidate_table_fp32(d)
    assert t["x"][0] == 2048.0 and t["y"][0] == 2052.0 and t["ts"][0] == 65504.0
    assert not t["active"][0]


def test_relative_rounding_bound(oracle):
    """Round to nearest in binary16: |half(v) - v| <= 2^-11 |v| for v in the
    normal range [2^-14, 65504]."""
    o = oracle
    rng = np.random.default_rng(7)
    v = np.float32(np.exp(rng.uniform(np.log(2.0 ** -14), np.log(60000.0), 5000)))
    d = _prep_one(o)
    for f in ("x", "y", "ts", "r", "G00", "G01", "G11"):
        d[f] = v * np.float32(rng.choice([-1, 1], v.size)) if f in ("G01", "r") else v.copy()
    d["active"] = np.ones(v.size, bool)
    for c in ("cr", "cg", "cb"):
        d[c] = np.zeros(v.size, np.float32)
    t = o.candidate_table_fp32(d)
    for f in ("x", "y", "ts", "r", "G00", "G01", "G11"):
        err = np.abs(t[f].astype(np.float64) - d[f].astype(np.float64))
        assert np.all(err <= 2.0 ** -11 * np.abs(d[f].astype(np.float64))), f


def test_half_exact_table_gives_the_float32_pass(oracle):
    """Sites whose scoring values are all binary16 numbers (positions on a
    quarter-pixel lattice, radii and tau s powers of two, axis-aligned metric
    with G entries powers of two): the half2 table equals the float32 table
    and the candidate pass is identical."""
    o = oracle
    H, W, K, n = 40, 56, 8, 300
    rng = np.random.default_rng(3)
    p = np.zeros((o.N_PARAMS, n), np.float32)
    p[o.PX] = np.floor(rng.uniform(0, W, n) * 4) / 4
    p[o.PY] = np.floor(rng.uniform(0, H, n) * 4) / 4
    p[o.PLOGTAU] = 0.0
    p[o.PR] = 2.0 ** rng.integers(-2, 3, n)
    p[o.PUX] = 1.0
    p[o.PA] = 0.0
    p[o.PB] = 0.0
    prep = o.prepare_fp32(p, H, W)
    prep["ts"] = np.float32(2.0 ** rng.integers(-3, 3, n))       # powers of two
    t = o.candidate_table_fp32(prep)
    for f in ("x", "y", "ts", "r", "G00", "G01", "G11"):
        assert np.array_equal(t[f], prep[f]), f
    ids = o.topk_seed_fp32(prep, H, W, K)
    code = o.step_code(2, H, W)
    a = o.topk_pass_fp32(prep, ids, H, W, K, code, 2, 11)
    b = o.topk_pass_fp32(t, ids, H, W, K, code, 2, 11)
    assert np.array_equal(a, b)


def test_quantised_pass_stays_close_to_float32(oracle):
    """On a realistic site set the half2 pass keeps most of the float32
    pass's lists (the scores differ only by binary16 rounding of the
    inputs), and every list is valid: distinct, active ids, sentinel tail."""
    o = oracle
    H, W, K = 48, 64, 8
    img = gen.image_noise_polygons_lines(H, W, seed=5, n_polygons=5, n_lines=3)
    p = gen.sites_isotropic(img, 400, seed=6)
    prep = o.prepare_fp32(p, H, W)
    t = o.candidate_table_fp32(prep)
    ids = o.propagate_fp32(p, H, W, K, passes=6, J=2, seed=9)
    code = (1 << 16) | 6
    a = o.topk_pass_fp32(prep, ids, H, W, K, code, 2, 9)
    b = o.topk_pass_fp32(t, ids, H, W, K, code, 2, 9)
    same = np.mean([set(a[i][a[i] != o.INVALID]) == set(b[i][b[i] != o.INVALID]) for i in range(H * W)])
    assert same > 0.8, same
    for row in b:
        v = row[row != o.INVALID]
        assert len(set(v.tolist())) == len(v)
        assert np.all(row[len(v):] == o.INVALID)
        assert np.all(prep["active"][v.astype(np.int64)])


def test_words_match_halves(oracle):
    o = oracle
    p = gen.sites_random_spd(30, 40, 64, seed=2)
    prep = o.prepare_fp32(p, 30, 40)
    h = o.candidate_halves(prep)
    w = o.candidate_words(prep)
    back = np.stack([(w & 0xFFFF).astype(np.uint16), (w >> 16).astype(np.uint16)], axis=2).reshape(-1, 8)
    assert np.array_equal(back.view(np.float16).view(np.uint16), h.view(np.uint16))
    with pytest.raises(KeyError):
        o.candidate_words({"x": np.float32([1.0])})
