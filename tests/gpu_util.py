"""Helpers for the GPU parity tests: build/load the library once, move seeded
inputs to the device, and compare against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_21984_gb300 import build, capi
    build.build()
    capi.lib()
    return capi


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def prepare(capi, params_np, H, W):
    p = dev(params_np.astype(np.float32))
    cap = params_np.shape[1]
    prep = capi.empty_prep(cap)
    capi.sad_prepare_sites(p, H, W, prep)
    return p, prep


def prep_to_oracle_dict(prep_t, cap):
    """Device prep planes -> host dict keyed like the oracle's (for equality checks)."""
    a = prep_t.cpu().numpy()[:, :cap]
    return {"x": a[0, :, 0], "y": a[0, :, 1], "ts": a[0, :, 2], "r": a[0, :, 3],
            "G00": a[1, :, 0], "G01": a[1, :, 1], "G11": a[1, :, 2], "active": a[1, :, 3] != 0,
            "cr": a[2, :, 0], "cg": a[2, :, 1], "cb": a[2, :, 2]}


def prep_blend_copies(prep_t, cap):
    """The verbatim copies in the blend record and the dense blue plane:
    {x, y, cr, cg, cb} from planes 3, 4 and 5."""
    a = prep_t.cpu().numpy()
    return {"x": a[3, :cap, 0], "y": a[3, :cap, 1], "cr": a[4, :cap, 2], "cg": a[4, :cap, 3],
            "cb": a[5].reshape(-1)[:cap]}


def assert_grads_close(got, ref, rel=1e-4, floor_frac=1e-4, planes=range(11), names=None):
    """Norm-relative per parameter plane, with an absolute floor of
    floor_frac * max|ref| of that plane.  Returns, per plane, the largest
    element-wise relative error without the floor (over the entries whose
    reference is not zero), printed for the record: the floor is what
    admits the sites whose gradient is many orders of magnitude below the
    plane's largest."""
    worst = {}
    for j in planes:
        r = ref[j]
        g = got[j]
        scale = np.abs(r).max()
        if scale == 0:
            assert np.abs(g).max() == 0, (j, np.abs(g).max())
            continue
        err = np.abs(g - r)
        tol = rel * np.abs(r) + floor_frac * scale
        bad = err > tol
        assert not bad.any(), (
            f"plane {j if names is None else names[j]}: {bad.sum()} of {len(r)} out of tolerance, "
            f"max err {err.max():.3e}, scale {scale:.3e}")
        nr = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300)
        assert nr <= rel, (j, nr)
        nz = r != 0
        worst[j if names is None else names[j]] = float((err[nz] / np.abs(r[nz])).max()) if nz.any() else 0.0
    print("largest relative error per plane without the floor:", {k: f"{v:.2e}" for k, v in worst.items()})
    return worst
