"""The C-ABI library builds, loads and exports every entry point that
include/sad.h declares; host-side argument checks reject bad input before any
launch (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sad.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sad(?:1d)?_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2604_21984_gb300 import build, capi
    build.build()
    return capi.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    from paper_2604_21984_gb300 import capi
    assert set(names) == set(capi.exported_symbols())


def test_status_strings_and_version(L):
    assert L.sad_abi_version() == 8
    assert L.sad_status_string(0) == b"ok"
    assert L.sad_status_string(1) == b"invalid argument"
    assert L.sad_status_string(99) == b"unknown status"


def test_workspace_size_query(L):
    small = L.sad_backward_workspace_bytes(64, 64, 8, 256, 0)
    big = L.sad_backward_workspace_bytes(2048, 2048, 16, 262144, 0)
    assert 0 < small < big
    assert L.sad_backward_workspace_bytes(64, 64, 5, 256, 0) == 0      # bad K
    assert L.sad_backward_workspace_bytes(0, 64, 8, 256, 0) == 0       # empty image
    more = L.sad_backward_workspace_bytes(64, 64, 8, 256, 10 ** 6)
    assert more > small


def test_backward_record_bound(L):
    # 4 x 4 tiles of 16 x 16; a tile's 256 pixels list at most 256 K distinct sites
    assert L.sad_backward_max_records(64, 64, 8, 256) == 16 * 256            # capped by the sites
    assert L.sad_backward_max_records(64, 64, 8, 10 ** 6) == 16 * 256 * 8    # capped by the lists
    assert L.sad_backward_max_records(65, 48, 4, 10 ** 6) == 5 * 3 * 256 * 4  # ragged edge tiles count whole
    assert L.sad_backward_max_records(64, 64, 8, 0) == 0
    assert L.sad_backward_max_records(64, 64, 5, 256) == -1
    assert L.sad_backward_max_records(0, 64, 8, 256) == -1


def test_bad_arguments_rejected_on_host(L):
    p = ctypes.c_void_p(256)          # never dereferenced: checks fail first
    assert L.sad_render(p, 10, 8, 8, 5, p, p, None) == 1                # K not in {4,8,16}
    assert b"K must be" in L.sad_last_error()
    assert L.sad_render(p, 10, 0, 8, 8, p, p, None) == 1                # empty image
    assert L.sad_update_topk(p, 10, 8, 8, 8, p, p, 0, 17, 0, None) == 1  # too many injections
    assert L.sad_update_topk(p, 10, 8, 8, 8, p, p, 0, 2, 0, None) == 1   # in-place update
    assert b"overlap" in L.sad_last_error()
    assert L.sad_prepare_sites(p, -1, 8, 8, p, None) == 1
    assert L.sad_render(ctypes.c_void_p(260), 10, 8, 8, 8, p, p, None) == 1   # misaligned prep
    assert L.sad_decode_points(p, 10, 8, 8, 8, p, p, -1, p, None) == 1
    assert L.sad_render_backward(p, p, 10, 8, 8, 8, p, p, p, p, 16, None) == 3  # workspace too small
    assert b"at least" in L.sad_last_error()
    assert L.sad_adam_step(p, p, p, p, 10, 8, 8, 0, None, None) == 1


def test_product_path_has_no_oracle_import():
    """The CUDA path never imports the oracle (only tests, smoke and the
    bench's CPU legs may)."""
    pkg = os.path.join(ROOT, "paper_2604_21984_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle|sad_oracle|oracle/", txt, re.M), f


def test_batch_above_the_image_limit_is_rejected(L):
    """A batch descriptor holds at most 64 images (the per-image fixed-point
    scales and the step's image table are sized for that): 65 images are
    refused on the host by the workspace query and by every batched call,
    before any launch."""
    from paper_2604_21984_gb300 import capi
    ims = [dict(H=16, W=16, site_offset=4 * i, capacity=4, pixel_offset=256 * i, seed=i, state_index=i)
           for i in range(65)]
    tab = capi.batch_table(ims)
    tp = ctypes.cast(tab, ctypes.c_void_p)
    assert L.sad_step_workspace_bytes(tp, 65, 16, 16, 260, 65 * 256, 0) == 0
    assert L.sad_step_workspace_bytes(tp, 64, 16, 16, 260, 65 * 256, 0) > 0
    p = ctypes.c_void_p(256)          # never dereferenced: the count check fails first
    st = L.sad_train_step(tp, 65, 16, 4, 16, p, p, p, p, 260, p, p, 65 * 256, p, p, None, p, 128,
                          None, p, 1 << 20, None)
    assert st == 1 and b"B <= 64" in L.sad_last_error()
    st = L.sad_batch_update(tp, 65, 16, 4, p, 260, p, p, 65 * 256, p, 128, None)
    assert st == 1 and b"B <= 64" in L.sad_last_error()
    st = L.sad_train_step(tp, 0, 16, 4, 16, p, p, p, p, 260, p, p, 65 * 256, p, p, None, p, 128,
                          None, p, 1 << 20, None)
    assert st == 1
