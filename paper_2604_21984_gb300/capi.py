"""Thin Python binding of libsad.so (the C-ABI declared in include/sad.h).

Argument marshalling only: every function checks tensor dtypes, devices,
shapes and contiguity, passes raw device pointers and the current CUDA
stream, and raises ``SadError`` on a non-zero status.  All arithmetic runs in
the library's CUDA kernels; there is no CPU fallback.  If the library is
missing or cannot be loaded, ``lib()`` raises and nothing else works.

Layouts (see include/sad.h): params float32[11, cap]; prep float32[3, cap, 4];
map uint32 planes stored as int32[K/4, H*W, 4] (torch has no uint32 kernels
on all versions, the bits are the same); rgb float32[H, W, 3].
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libsad.so")
_lib = None

N_PARAMS = 11
INVALID = 0xFFFFFFFF
STEP_KEEP_LISTS = 1   # batch-image flag (include/sad.h SAD_STEP_KEEP_LISTS)
PLANE_LOGTAU = 2      # plane of log tau in the site parameter and gradient arrays
SAD_EWORKSPACE = 3    # status: per-tile records did not fit the workspace
PREP_PLANES = 6       # float4 planes of the prepared site table (include/sad.h)
NOALLOC_SCRATCH_BYTES = 64 << 20   # include/sad.h SAD_NOALLOC_SCRATCH_BYTES: held on every device


class SadError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


class DpParams(ctypes.Structure):
    _fields_ = [
        ("densify_pct", ctypes.c_double), ("prune_pct", ctypes.c_double),
        ("alpha", ctypes.c_float), ("eps", ctypes.c_float), ("mass_min", ctypes.c_float),
        ("min_offset", ctypes.c_float), ("max_offset", ctypes.c_float),
        ("log_tau_shift", ctypes.c_float), ("r_scale", ctypes.c_float),
        ("a_min", ctypes.c_float), ("a_max", ctypes.c_float), ("a_fallback_scale", ctypes.c_float),
        ("energy_min", ctypes.c_float), ("ratio_min", ctypes.c_float),
    ]


class BatchImage(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("site_offset", ctypes.c_int32),
                ("capacity", ctypes.c_int32), ("pixel_offset", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("state_index", ctypes.c_int32), ("flags", ctypes.c_int32)]


class Sad1dAdam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 4), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("log_tau_min", ctypes.c_float), ("log_tau_max", ctypes.c_float)]


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class AdamHparams(ctypes.Structure):
    _fields_ = [
        ("lr", ctypes.c_float * N_PARAMS),
        ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
        ("log_tau_min", ctypes.c_float), ("log_tau_max", ctypes.c_float),
        ("r_min", ctypes.c_float), ("r_max", ctypes.c_float),
        ("a_min", ctypes.c_float), ("a_max", ctypes.c_float),
        ("b_min", ctypes.c_float), ("b_max", ctypes.c_float),
    ]


_SIGS = {
    "sad_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sad_last_error": (ctypes.c_char_p, []),
    "sad_abi_version": (ctypes.c_int, []),
    "sad_trace_enable": (ctypes.c_int, [ctypes.c_int]),
    "sad_trace_collect": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "sad_prepare_sites": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "sad_topk_seed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "sad_update_topk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32,
                                       ctypes.c_uint64, ctypes.c_void_p]),
    "sad1d_render": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "sad1d_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.POINTER(Sad1dAdam), ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "sad_exact_topk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "sad_pack_candidates": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "sad_update_topk_h2": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32,
                                          ctypes.c_uint64, ctypes.c_void_p]),
    "sad_jfa_flood": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                     ctypes.c_void_p]),
    "sad_grid_seed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "sad_grid_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p]),
    "sad_grid_expand": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "sad_tau_diffusion": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "sad_render": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]),
    "sad_render_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sad_render_backward_saved": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_size_t, ctypes.c_void_p]),
    "sad_decode_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "sad_backward_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32,
                                                       ctypes.c_int32, ctypes.c_int32,
                                                       ctypes.c_int64]),
    "sad_backward_max_records": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_int32]),
    "sad_render_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "sad_train_grads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_size_t, ctypes.c_void_p]),
    "sad_workspace_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.c_void_p]),
    "sad_render_backward_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p]),
    "sad_init_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "sad_init_sites": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, ctypes.c_float,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p]),
    "sad_site_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "sad_densify_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "sad_densify_prune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(DpParams),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]),
    "sad_densify_prune_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.POINTER(DpParams), ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_size_t, ctypes.c_void_p]),
    "sad_step_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                                   ctypes.c_int64]),
    "sad_prepare_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p]),
    "sad_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(AdamHparams),
                                      ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_void_p]),
    "sad_pack_sites": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sad_unpack_sites": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "sad_decode_packed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "sad_render_packed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "sad_batch_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "sad_batch_insert": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p]),
    "sad_decode_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "sad_adam_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(AdamHparams), ctypes.c_void_p]),
}


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Loads libsad.so once (raises if it is missing: no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libsad.so not built at {_LIB_PATH}; run "
                              "paper_2604_21984_gb300.build.build() first")
        L = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status, what):
    if status != 0:
        msg = lib().sad_last_error().decode(errors="replace")
        raise SadError(status, f"{what}: {msg}")


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype, name, numel=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------------------------
# allocation helpers (torch owns all device memory)
# ----------------------------------------------------------------------------

def empty_prep(cap, device="cuda"):
    return torch.empty((PREP_PLANES, max(cap, 1), 4), dtype=torch.float32, device=device)


def empty_map(H, W, K, device="cuda"):
    return torch.empty((K // 4, H * W, 4), dtype=torch.int32, device=device)


def map_from_ids(ids, device="cuda"):
    """uint32[P, K] (numpy or torch) -> device planes int32[K/4, P, 4]."""
    if isinstance(ids, np.ndarray):
        ids = torch.from_numpy(ids.astype(np.uint32).view(np.int32))
    P, K = ids.shape
    return ids.reshape(P, K // 4, 4).permute(1, 0, 2).contiguous().to(device)


def ids_from_map(m):
    """device planes int32[K/4, P, 4] -> numpy uint32[P, K]."""
    Kq, P, _ = m.shape
    return m.permute(1, 0, 2).reshape(P, Kq * 4).cpu().numpy().view(np.uint32)


def backward_workspace(H, W, K, cap, max_records=0, device="cuda"):
    n = lib().sad_backward_workspace_bytes(H, W, K, cap, max_records)
    if n == 0:
        raise ValueError("invalid problem for sad_backward_workspace_bytes")
    return torch.empty(n, dtype=torch.uint8, device=device)


def sad_backward_max_records(H, W, K, cap):
    n = lib().sad_backward_max_records(H, W, K, cap)
    if n < 0:
        raise ValueError("invalid problem for sad_backward_max_records")
    return int(n)


# ----------------------------------------------------------------------------
# entry points (same names as the C-ABI)
# ----------------------------------------------------------------------------

def sad_prepare_sites(params, H, W, prep, stream=None):
    cap = params.shape[1]
    _check(lib().sad_prepare_sites(_ptr(params, torch.float32, "params", N_PARAMS * cap), cap, H, W,
                                   _ptr(prep, torch.float32, "prep"), _stream(stream)),
           "sad_prepare_sites")
    return prep


def sad_topk_seed(prep, cap, H, W, K, map_out, stream=None):
    _check(lib().sad_topk_seed(_ptr(prep, torch.float32, "prep"), cap, H, W, K,
                               _ptr(map_out, torch.int32, "map", H * W * K), _stream(stream)),
           "sad_topk_seed")
    return map_out


def sad_update_topk(prep, cap, H, W, K, map_in, map_out, step_code, n_inject, seed, stream=None):
    _check(lib().sad_update_topk(_ptr(prep, torch.float32, "prep"), cap, H, W, K,
                                 _ptr(map_in, torch.int32, "map_in", H * W * K),
                                 _ptr(map_out, torch.int32, "map_out", H * W * K),
                                 step_code & 0xFFFFFFFF, n_inject, seed & ((1 << 64) - 1),
                                 _stream(stream)), "sad_update_topk")
    return map_out


def sad_exact_topk(prep, cap, H, W, K, pixels, ids_out=None, stream=None):
    """Exact top-K ids of the pixels (int64[n] device indices) by brute force
    over every site: uint32 values in an int32[n, K] device tensor."""
    n = pixels.numel()
    if ids_out is None:
        ids_out = torch.empty((n, K), dtype=torch.int32, device=pixels.device)
    _check(lib().sad_exact_topk(_ptr(prep, torch.float32, "prep"), cap, H, W, K,
                                _ptr(pixels, torch.int64, "pixels", n), n,
                                _ptr(ids_out, torch.int32, "ids_out", n * K), _stream(stream)),
           "sad_exact_topk")
    return ids_out


def sad_pack_candidates(prep, cap, cand, stream=None):
    """cand: int32 tensor of cap*4 words (the half2 candidate records)."""
    _check(lib().sad_pack_candidates(_ptr(prep, torch.float32, "prep"), cap,
                                     _ptr(cand, torch.int32, "cand", cap * 4), _stream(stream)),
           "sad_pack_candidates")
    return cand


def sad_update_topk_h2(cand, cap, H, W, K, map_in, map_out, step_code, n_inject, seed, stream=None):
    _check(lib().sad_update_topk_h2(_ptr(cand, torch.int32, "cand"), cap, H, W, K,
                                    _ptr(map_in, torch.int32, "map_in", H * W * K),
                                    _ptr(map_out, torch.int32, "map_out", H * W * K),
                                    step_code & 0xFFFFFFFF, n_inject, seed & ((1 << 64) - 1),
                                    _stream(stream)), "sad_update_topk_h2")
    return map_out


def sad_render(prep, cap, H, W, K, map_in, rgb, stream=None):
    _check(lib().sad_render(_ptr(prep, torch.float32, "prep"), cap, H, W, K,
                            _ptr(map_in, torch.int32, "map", H * W * K),
                            _ptr(rgb, torch.float32, "rgb", H * W * 3), _stream(stream)),
           "sad_render")
    return rgb


def sad_render_save(prep, cap, H, W, K, map_in, rgb, fwd, stream=None):
    """sad_render that also writes fwd = float32[2, H*W] {max logit, 1/Z}."""
    _check(lib().sad_render_save(_ptr(prep, torch.float32, "prep"), cap, H, W, K,
                                 _ptr(map_in, torch.int32, "map", H * W * K),
                                 _ptr(rgb, torch.float32, "rgb", H * W * 3),
                                 _ptr(fwd, torch.float32, "fwd", 2 * H * W), _stream(stream)),
           "sad_render_save")
    return rgb


def sad_decode_points(prep, cap, H, W, K, map_in, xy, rgb, stream=None):
    n = xy.shape[0]
    _check(lib().sad_decode_points(_ptr(prep, torch.float32, "prep"), cap, H, W, K,
                                   _ptr(map_in, torch.int32, "map", H * W * K),
                                   _ptr(xy, torch.float32, "xy", 2 * n), n,
                                   _ptr(rgb, torch.float32, "rgb", 3 * n), _stream(stream)),
           "sad_decode_points")
    return rgb


def sad_render_backward(params, prep, H, W, K, map_in, grad_rgb, grads, ws, stream=None):
    cap = params.shape[1]
    _check(lib().sad_render_backward(_ptr(params, torch.float32, "params", N_PARAMS * cap),
                                     _ptr(prep, torch.float32, "prep"), cap, H, W, K,
                                     _ptr(map_in, torch.int32, "map", H * W * K),
                                     _ptr(grad_rgb, torch.float32, "grad_rgb", H * W * 3),
                                     _ptr(grads, torch.float32, "grads", N_PARAMS * cap),
                                     _ptr(ws, torch.uint8, "workspace"), ws.numel(),
                                     _stream(stream)), "sad_render_backward")
    return grads


def sad_render_backward_saved(params, prep, H, W, K, map_in, grad_rgb, rgb, fwd, grads, ws,
                              stream=None):
    """sad_render_backward from sad_render_save's rgb and fwd."""
    cap = params.shape[1]
    _check(lib().sad_render_backward_saved(_ptr(params, torch.float32, "params", N_PARAMS * cap),
                                           _ptr(prep, torch.float32, "prep"), cap, H, W, K,
                                           _ptr(map_in, torch.int32, "map", H * W * K),
                                           _ptr(grad_rgb, torch.float32, "grad_rgb", H * W * 3),
                                           _ptr(rgb, torch.float32, "rgb", H * W * 3),
                                           _ptr(fwd, torch.float32, "fwd", 2 * H * W),
                                           _ptr(grads, torch.float32, "grads", N_PARAMS * cap),
                                           _ptr(ws, torch.uint8, "workspace"), ws.numel(),
                                           _stream(stream)), "sad_render_backward_saved")
    return grads


def sad_render_backward_noalloc(params, prep, H, W, K, map_in, grad_rgb, grads, status=None,
                                stream=None):
    """sad_render_backward for callers that cannot allocate a workspace: the
    library's own fixed scratch buffer is used instead (see include/sad.h for
    its limits; concurrent calls on different streams race on it).  `status`
    is an optional device int32[1] that receives 0, or SAD_EWORKSPACE if the
    per-tile records did not fit; without it an overflow goes unreported."""
    cap = params.shape[1]
    _check(lib().sad_render_backward_noalloc(
        _ptr(params, torch.float32, "params", N_PARAMS * cap), _ptr(prep, torch.float32, "prep"),
        cap, H, W, K, _ptr(map_in, torch.int32, "map", H * W * K),
        _ptr(grad_rgb, torch.float32, "grad_rgb", H * W * 3),
        _ptr(grads, torch.float32, "grads", N_PARAMS * cap),
        _ptr(status, torch.int32, "status", 1), _stream(stream)), "sad_render_backward_noalloc")
    return grads


def sad_train_grads(params, prep, H, W, K, map_in, target, grads, loss, ws, rgb_out=None,
                    stream=None):
    cap = params.shape[1]
    _check(lib().sad_train_grads(_ptr(params, torch.float32, "params", N_PARAMS * cap),
                                 _ptr(prep, torch.float32, "prep"), cap, H, W, K,
                                 _ptr(map_in, torch.int32, "map", H * W * K),
                                 _ptr(target, torch.float32, "target", H * W * 3),
                                 _ptr(grads, torch.float32, "grads", N_PARAMS * cap),
                                 _ptr(loss, torch.float32, "loss", 1),
                                 _ptr(rgb_out, torch.float32, "rgb_out", H * W * 3),
                                 _ptr(ws, torch.uint8, "workspace"), ws.numel(),
                                 _stream(stream)), "sad_train_grads")
    return grads


def sad_workspace_status(ws, stream=None):
    used = ctypes.c_int64(0)
    st = lib().sad_workspace_status(_ptr(ws, torch.uint8, "workspace"), ctypes.byref(used),
                                    _stream(stream))
    return st, int(used.value)


def sad_init_sites(img, n, capacity, lambda_init, seed, log_tau0, params=None, ws=None,
                   stream=None):
    """Gradient-weighted initial site set (see include/sad.h); returns params."""
    H, W, _ = img.shape
    if params is None:
        params = torch.empty((N_PARAMS, capacity), dtype=torch.float32, device=img.device)
    if ws is None:
        ws = torch.empty(lib().sad_init_workspace_bytes(H, W), dtype=torch.uint8, device=img.device)
    _check(lib().sad_init_sites(_ptr(img, torch.float32, "img", H * W * 3), H, W, n, capacity,
                                lambda_init, seed & ((1 << 64) - 1), log_tau0,
                                _ptr(params, torch.float32, "params", N_PARAMS * capacity),
                                _ptr(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)),
           "sad_init_sites")
    return params


def sad_site_stats(prep, cap, H, W, K, map_in, target, stats, ws, stream=None):
    """Per-site mass, energy, residual moments and removal delta (float32[8, cap])."""
    _check(lib().sad_site_stats(_ptr(prep, torch.float32, "prep"), cap, H, W, K,
                                _ptr(map_in, torch.int32, "map", H * W * K),
                                _ptr(target, torch.float32, "target", H * W * 3),
                                _ptr(stats, torch.float32, "stats", 8 * cap),
                                _ptr(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)),
           "sad_site_stats")
    return stats


def dp_params(densify_pct=0.01, prune_pct=0.033, alpha=0.7, eps=1e-8, mass_min=1.0,
              min_offset=1.5, max_offset=48.0, log_tau_shift=-0.25, r_scale=0.85,
              a_range=(-2.0, 2.0), a_fallback_scale=0.8, energy_min=1e-6, ratio_min=1.01):
    """Densify/prune parameters; defaults are the paper's (Sec. 4.5, Sec. 6.1)."""
    d = DpParams()
    d.densify_pct, d.prune_pct, d.alpha, d.eps, d.mass_min = densify_pct, prune_pct, alpha, eps, mass_min
    d.min_offset, d.max_offset, d.log_tau_shift, d.r_scale = min_offset, max_offset, log_tau_shift, r_scale
    d.a_min, d.a_max = a_range
    d.a_fallback_scale, d.energy_min, d.ratio_min = a_fallback_scale, energy_min, ratio_min
    return d


def densify_workspace(cap, H, W, device="cuda"):
    return torch.empty(lib().sad_densify_workspace_bytes(cap, H, W), dtype=torch.uint8, device=device)


def sad_densify_prune(params, m, v, H, W, K, stats, target, map_inout, dp, ws, stream=None):
    """One densify-then-prune event; returns the number of active sites (syncs)."""
    cap = params.shape[1]
    n = ctypes.c_int32(0)
    _check(lib().sad_densify_prune(_ptr(params, torch.float32, "params", N_PARAMS * cap),
                                   _ptr(m, torch.float32, "m", N_PARAMS * cap),
                                   _ptr(v, torch.float32, "v", N_PARAMS * cap), cap, H, W, K,
                                   _ptr(stats, torch.float32, "stats", 8 * cap),
                                   _ptr(target, torch.float32, "target", H * W * 3),
                                   _ptr(map_inout, torch.int32, "map", H * W * K),
                                   ctypes.byref(dp), ctypes.byref(n),
                                   _ptr(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)),
           "sad_densify_prune")
    return int(n.value)


def sad_densify_prune_async(params, m, v, H, W, K, stats, target, map_inout, dp, n_active, ws,
                            stream=None):
    """The same event entirely in stream order: no synchronisation; the
    active count afterwards goes to `n_active` (device int32[1])."""
    cap = params.shape[1]
    _check(lib().sad_densify_prune_async(_ptr(params, torch.float32, "params", N_PARAMS * cap),
                                         _ptr(m, torch.float32, "m", N_PARAMS * cap),
                                         _ptr(v, torch.float32, "v", N_PARAMS * cap), cap, H, W, K,
                                         _ptr(stats, torch.float32, "stats", 8 * cap),
                                         _ptr(target, torch.float32, "target", H * W * 3),
                                         _ptr(map_inout, torch.int32, "map", H * W * K),
                                         ctypes.byref(dp), _ptr(n_active, torch.int32, "n_active", 1),
                                         _ptr(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)),
           "sad_densify_prune_async")
    return n_active


# Per-plane Adam learning rates (x, y, log_tau, r, cr, cg, cb, ux, uy, a, b);
# x, y and r step in normalised units (p s).  LR_DEFAULT is the best of a
# sweep on the 768x512 encode workload (2000 iterations, 2 images x 3 runs);
# LR_CONFIG2_LITERAL is 1e-3 for positions and 5e-3 for colours read in
# normalised units, with the other planes at 1e-2 / 1e-3.
LR_DEFAULT = (6.25e-5, 6.25e-5, 1e-2, 6.25e-5, 1.25e-3, 1.25e-3, 1.25e-3, 1.5e-2, 1.5e-2, 1.5e-2, 0.0)
LR_CONFIG2_LITERAL = (1e-3, 1e-3, 1e-2, 1e-3, 5e-3, 5e-3, 5e-3, 1e-2, 1e-2, 1e-2, 0.0)


def adam_hparams(lr=None, beta1=0.9, beta2=0.999, eps=1e-8, log_tau_range=(2.0, 20.0),
                 r_range=(1.0, 512.0), a_range=(-2.0, 2.0), b_range=(-8.0, 8.0)):
    """Defaults: Sec. 6.1 clamps; per-plane learning rates (x, y, log_tau, r,
    cr, cg, cb, ux, uy, a, b), LR_DEFAULT unless given."""
    if lr is None:
        lr = LR_DEFAULT
    hp = AdamHparams()
    for i, v in enumerate(lr):
        hp.lr[i] = v
    hp.beta1, hp.beta2, hp.eps = beta1, beta2, eps
    hp.log_tau_min, hp.log_tau_max = log_tau_range
    hp.r_min, hp.r_max = r_range
    hp.a_min, hp.a_max = a_range
    hp.b_min, hp.b_max = b_range
    return hp


def sad_adam_step(params, grads, m, v, H, W, t, hp, stream=None):
    cap = params.shape[1]
    n = N_PARAMS * cap
    _check(lib().sad_adam_step(_ptr(params, torch.float32, "params", n),
                               _ptr(grads, torch.float32, "grads", n),
                               _ptr(m, torch.float32, "m", n), _ptr(v, torch.float32, "v", n),
                               cap, H, W, t, ctypes.byref(hp), _stream(stream)),
           "sad_adam_step")
    return params


# ----------------------------------------------------------------------------
# batched training (many images per launch)
# ----------------------------------------------------------------------------

def batch_table(images):
    """images: list of dicts with H, W, site_offset, capacity, pixel_offset, seed."""
    arr = (BatchImage * len(images))()
    for i, d in enumerate(images):
        arr[i].H, arr[i].W = d["H"], d["W"]
        arr[i].site_offset, arr[i].capacity = d["site_offset"], d["capacity"]
        arr[i].pixel_offset, arr[i].seed = d["pixel_offset"], d["seed"] & ((1 << 64) - 1)
        arr[i].state_index = d.get("state_index", i)
        arr[i].flags = d.get("flags", 0)
    return arr


def step_workspace(table, K, total_cap, total_pixels, max_records=0, device="cuda", tile_w=16):
    n = lib().sad_step_workspace_bytes(ctypes.cast(table, ctypes.c_void_p), len(table), K, tile_w,
                                       total_cap, total_pixels, max_records)
    if n == 0:
        raise ValueError("invalid batch table for sad_step_workspace_bytes")
    # zeroed once: the per-site accumulators must start at zero (each call
    # clears them again after use)
    return torch.zeros(n, dtype=torch.uint8, device=device)


def sad_prepare_batch(table, params, prep, total_pixels, stream=None):
    cap = params.shape[1]
    _check(lib().sad_prepare_batch(ctypes.cast(table, ctypes.c_void_p), len(table),
                                   _ptr(params, torch.float32, "params", N_PARAMS * cap),
                                   _ptr(prep, torch.float32, "prep"), cap, total_pixels,
                                   _stream(stream)), "sad_prepare_batch")


def sad_train_step(table, K, J, params, m, v, prep, map_in, map_out, total_pixels, targets, loss,
                   hp, state, ws, grads_out=None, stream=None, tile_w=16):
    """state: device int32[n_states, 4] per-image rows {t, pass, parity, 0};
    tile_w: 16 (16x16 tiles) or 32 (32x8 tiles)."""
    cap = params.shape[1]
    n = N_PARAMS * cap
    _check(lib().sad_train_step(ctypes.cast(table, ctypes.c_void_p), len(table), K, J, tile_w,
                                _ptr(params, torch.float32, "params", n), _ptr(m, torch.float32, "m", n),
                                _ptr(v, torch.float32, "v", n), _ptr(prep, torch.float32, "prep"), cap,
                                _ptr(map_in, torch.int32, "map_in", total_pixels * K),
                                _ptr(map_out, torch.int32, "map_out", total_pixels * K), total_pixels,
                                _ptr(targets, torch.float32, "targets", total_pixels * 3),
                                _ptr(loss[:len(table)] if loss is not None else None, torch.float32,
                                     "loss", len(table)), ctypes.byref(hp),
                                _ptr(state, torch.int32, "state"), state.shape[0],
                                _ptr(grads_out, torch.float32, "grads_out", n),
                                _ptr(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)),
           "sad_train_step")


class TrainStepCall:
    """A prepared sad_train_step: the arguments are marshalled once, so a
    call (eager or while being captured into a graph) is one ctypes call."""

    def __init__(self, table, K, J, params, m, v, prep, map_in, map_out, total_pixels, targets, loss,
                 hp, state, ws, grads_out=None, tile_w=16):
        cap = params.shape[1]
        n = N_PARAMS * cap
        self.table = table
        self.hp = hp
        self.keep = (params, m, v, prep, map_in, map_out, targets, loss, state, ws, grads_out)
        self.args = [ctypes.cast(table, ctypes.c_void_p), len(table), K, J, tile_w,
                     _ptr(params, torch.float32, "params", n), _ptr(m, torch.float32, "m", n),
                     _ptr(v, torch.float32, "v", n), _ptr(prep, torch.float32, "prep"), cap,
                     _ptr(map_in, torch.int32, "map_in", total_pixels * K),
                     _ptr(map_out, torch.int32, "map_out", total_pixels * K), total_pixels,
                     _ptr(targets, torch.float32, "targets", total_pixels * 3),
                     _ptr(loss[:len(table)] if loss is not None else None, torch.float32, "loss",
                          len(table)), ctypes.byref(hp),
                     _ptr(state, torch.int32, "state"), state.shape[0],
                     _ptr(grads_out, torch.float32, "grads_out", n),
                     _ptr(ws, torch.uint8, "workspace"), ws.numel()]
        self.fn = lib().sad_train_step

    def __call__(self, stream=None):
        _check(self.fn(*self.args, _stream(stream)), "sad_train_step")


def sad_decode_batch(table, K, prep, total_cap, map_in, total_pixels, xy, qimg, rgb, stream=None):
    n = xy.shape[0]
    _check(lib().sad_decode_batch(ctypes.cast(table, ctypes.c_void_p), len(table), K,
                                  _ptr(prep, torch.float32, "prep"), total_cap,
                                  _ptr(map_in, torch.int32, "map", total_pixels * K), total_pixels,
                                  _ptr(xy, torch.float32, "xy", 2 * n), _ptr(qimg, torch.int32, "qimg", n),
                                  n, _ptr(rgb, torch.float32, "rgb", 3 * n), _stream(stream)),
           "sad_decode_batch")
    return rgb


def sad_batch_insert(entry, K, src_params, src_map, src_target, params, m, v, map_out, targets,
                     total_pixels, stream=None):
    """entry: one-element batch_table (the image's ranges)."""
    n, P = entry[0].capacity, entry[0].H * entry[0].W
    total_cap = params.shape[1]
    _check(lib().sad_batch_insert(ctypes.cast(entry, ctypes.c_void_p), K,
                                  _ptr(src_params, torch.float32, "src_params") if n else None,
                                  src_params.shape[1] if src_params is not None else 0,
                                  _ptr(src_map, torch.int32, "src_map", P * K),
                                  _ptr(src_target, torch.float32, "src_target", 3 * P)
                                  if src_target is not None else None,
                                  _ptr(params, torch.float32, "params"), _ptr(m, torch.float32, "m"),
                                  _ptr(v, torch.float32, "v"), total_cap,
                                  _ptr(map_out, torch.int32, "map", total_pixels * K),
                                  _ptr(targets, torch.float32, "targets", 3 * total_pixels),
                                  total_pixels, _stream(stream)),
           "sad_batch_insert")


def sad_trace_enable(on=True):
    """Switch kernel stage tracing on or off; returns the previous setting."""
    return bool(lib().sad_trace_enable(1 if on else 0))


def sad_trace_collect():
    """{kernel name: (launches, total device ms)} since the last collect."""
    arr = (TraceEntry * 128)()
    n = ctypes.c_int32(0)
    _check(lib().sad_trace_collect(ctypes.cast(arr, ctypes.c_void_p), 128, ctypes.byref(n)),
           "sad_trace_collect")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
            for i in range(min(n.value, 128))}


def sad_batch_update(table, K, J, prep, total_cap, map_in, map_out, total_pixels, state, stream=None):
    """One propagation pass of every image of the table (state rows advance)."""
    _check(lib().sad_batch_update(ctypes.cast(table, ctypes.c_void_p), len(table), K, J,
                                  _ptr(prep, torch.float32, "prep"), total_cap,
                                  _ptr(map_in, torch.int32, "map_in", total_pixels * K),
                                  _ptr(map_out, torch.int32, "map_out", total_pixels * K), total_pixels,
                                  _ptr(state, torch.int32, "state"), state.shape[0], _stream(stream)),
           "sad_batch_update")


def sad_pack_sites(params, H, W, packed=None, q=None, stream=None):
    """Packed 16-byte evaluation records: (int32[cap, 4] words, float32[10] q) on the device."""
    cap = params.shape[1]
    if packed is None:
        packed = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=params.device)
    if q is None:
        q = torch.empty(10, dtype=torch.float32, device=params.device)
    _check(lib().sad_pack_sites(_ptr(params, torch.float32, "params", N_PARAMS * cap), cap, H, W,
                                _ptr(packed, torch.int32, "packed"), _ptr(q, torch.float32, "q", 10),
                                _stream(stream)), "sad_pack_sites")
    return packed, q


def sad_unpack_sites(packed, q, cap, H, W, params=None, stream=None):
    if params is None:
        params = torch.empty((N_PARAMS, cap), dtype=torch.float32, device=packed.device)
    _check(lib().sad_unpack_sites(_ptr(packed, torch.int32, "packed"), _ptr(q, torch.float32, "q", 10), cap,
                                  H, W, _ptr(params, torch.float32, "params", N_PARAMS * cap),
                                  _stream(stream)), "sad_unpack_sites")
    return params


def sad_decode_packed(packed, q, cap, H, W, K, map_in, xy, rgb, stream=None):
    """q: the 10 range floats (a host sequence or tensor; read on the host)."""
    qh = (ctypes.c_float * 10)(*[float(v) for v in (q.tolist() if hasattr(q, "tolist") else q)])
    n = xy.shape[0]
    _check(lib().sad_decode_packed(_ptr(packed, torch.int32, "packed"), ctypes.cast(qh, ctypes.c_void_p), cap,
                                   H, W, K, _ptr(map_in, torch.int32, "map", H * W * K),
                                   _ptr(xy, torch.float32, "xy", 2 * n), n,
                                   _ptr(rgb, torch.float32, "rgb", 3 * n), _stream(stream)),
           "sad_decode_packed")
    return rgb


def sad_render_packed(packed, q, cap, H, W, K, map_in, rgb, stream=None):
    qh = (ctypes.c_float * 10)(*[float(v) for v in (q.tolist() if hasattr(q, "tolist") else q)])
    _check(lib().sad_render_packed(_ptr(packed, torch.int32, "packed"), ctypes.cast(qh, ctypes.c_void_p), cap,
                                   H, W, K, _ptr(map_in, torch.int32, "map", H * W * K),
                                   _ptr(rgb, torch.float32, "rgb", H * W * 3), _stream(stream)),
           "sad_render_packed")
    return rgb


def sad_jfa_flood(prep, cap, H, W, K, map_in, map_out, step_code, stream=None):
    _check(lib().sad_jfa_flood(_ptr(prep, torch.float32, "prep"), cap, H, W, K,
                               _ptr(map_in, torch.int32, "map_in", H * W * K),
                               _ptr(map_out, torch.int32, "map_out", H * W * K), step_code & 0xFFFFFFFF,
                               _stream(stream)), "sad_jfa_flood")
    return map_out


def grid_dims(H, W, s_grid):
    return (H + s_grid - 1) // s_grid, (W + s_grid - 1) // s_grid


def sad_grid_seed(prep, cap, H, W, s_grid, K, map_grid, stream=None):
    Hc, Wc = grid_dims(H, W, s_grid)
    _check(lib().sad_grid_seed(_ptr(prep, torch.float32, "prep"), cap, H, W, s_grid, K,
                               _ptr(map_grid, torch.int32, "map", Hc * Wc * K), _stream(stream)),
           "sad_grid_seed")
    return map_grid


def sad_grid_update(prep, cap, H, W, s_grid, K, map_in, map_out, step_code, n_inject, seed, stream=None):
    Hc, Wc = grid_dims(H, W, s_grid)
    _check(lib().sad_grid_update(_ptr(prep, torch.float32, "prep"), cap, H, W, s_grid, K,
                                 _ptr(map_in, torch.int32, "map_in", Hc * Wc * K),
                                 _ptr(map_out, torch.int32, "map_out", Hc * Wc * K), step_code & 0xFFFFFFFF,
                                 n_inject, seed & ((1 << 64) - 1), _stream(stream)), "sad_grid_update")
    return map_out


def sad_grid_expand(map_grid, H, W, s_grid, K, map_pixels, stream=None):
    Hc, Wc = grid_dims(H, W, s_grid)
    _check(lib().sad_grid_expand(_ptr(map_grid, torch.int32, "map_grid", Hc * Wc * K), H, W, s_grid, K,
                                 _ptr(map_pixels, torch.int32, "map", H * W * K), _stream(stream)),
           "sad_grid_expand")
    return map_pixels


def sad_tau_diffusion(params, H, W, K, map_in, lam, g_logtau, g_out, stream=None):
    cap = params.shape[1]
    _check(lib().sad_tau_diffusion(_ptr(params, torch.float32, "params", N_PARAMS * cap), cap, H, W, K,
                                   _ptr(map_in, torch.int32, "map", H * W * K), float(lam),
                                   _ptr(g_logtau, torch.float32, "g_logtau", cap),
                                   _ptr(g_out, torch.float32, "g_out", cap), _stream(stream)),
           "sad_tau_diffusion")
    return g_out


# ----------------------------------------------------------------------------
# 1-D SAD (Sec. "1D Signal Fitting")
# ----------------------------------------------------------------------------

SAD1D_LR = (2e-3, 1e-2, 1e-2, 1e-3)   # p, c, log_tau, r


def sad1d_hparams(lr=SAD1D_LR, beta1=0.9, beta2=0.999, eps=1e-8, log_tau_range=(2.0, 20.0)):
    h = Sad1dAdam()
    for j in range(4):
        h.lr[j] = lr[j]
    h.beta1, h.beta2, h.eps = beta1, beta2, eps
    h.log_tau_min, h.log_tau_max = log_tau_range
    return h


def sad1d_render(params, B, N, L, K, values=None, stream=None):
    """Values of B signals (params float32[4, B*N] device): float32[B, L]."""
    if values is None:
        values = torch.empty((B, L), dtype=torch.float32, device=params.device)
    _check(lib().sad1d_render(_ptr(params, torch.float32, "params", 4 * B * N), B, N, L, K,
                              _ptr(values, torch.float32, "values", B * L), _stream(stream)), "sad1d_render")
    return values


def sad1d_train_step(params, m, v, B, N, L, K, target, loss, hp, t, grads_out=None, stream=None):
    """One fused 1-D training iteration of every signal (Adam step t)."""
    _check(lib().sad1d_train_step(_ptr(params, torch.float32, "params", 4 * B * N),
                                  _ptr(m, torch.float32, "m", 4 * B * N),
                                  _ptr(v, torch.float32, "v", 4 * B * N), B, N, L, K,
                                  _ptr(target, torch.float32, "target", B * L),
                                  _ptr(loss, torch.float32, "loss", B), ctypes.byref(hp), t,
                                  _ptr(grads_out, torch.float32, "grads_out", 4 * B * N),
                                  _stream(stream)), "sad1d_train_step")
    return loss
