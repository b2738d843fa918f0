"""The C-ABI library loads and exports every entry point include/fastatlas.h
declares (no GPU needed: only calls that return before touching CUDA)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastatlas.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fa_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_17712_gb300 import build, fastatlas
    build.build()
    return fastatlas.load()


def test_header_declares_the_boundary():
    names = declared()
    for n in ["fa_create", "fa_destroy", "fa_mesh_register", "fa_visibility", "fa_chartify",
              "fa_parameterize", "fa_pack", "fa_uv", "fa_atlas_frame", "fa_last_device_status"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2502_17712_gb300 import fastatlas
    for n in declared():
        assert hasattr(lib, n), n
    assert sorted(fastatlas.EXPORTS) == declared()


def test_host_side_argument_errors(lib):
    from paper_2502_17712_gb300 import fastatlas as F
    assert lib.fa_version() == 10000
    assert lib.fa_status_string(F.FA_E_PACK_FAILED) == b"FA_E_PACK_FAILED"
    h = ctypes.c_void_p()
    # NULL config / zero maxima are rejected before any CUDA call
    assert lib.fa_create(ctypes.byref(h), None) == F.FA_E_INVALID_ARG
    cfg = F.fa_config(0, 10, 10, 64, 64, 10, 2, 0, 0)
    assert lib.fa_create(ctypes.byref(h), ctypes.byref(cfg)) == F.FA_E_INVALID_ARG
    cfg = F.fa_config(10, 10, 10, 64, 64, 15, 2, 0, 0)  # atlas side 2^15 > 2^14
    assert lib.fa_create(ctypes.byref(h), ctypes.byref(cfg)) == F.FA_E_INVALID_ARG
    cfg = F.fa_config(10, 10, 10, 64, 64, 10, 0, 0, 0)  # min_box 0
    assert lib.fa_create(ctypes.byref(h), ctypes.byref(cfg)) == F.FA_E_INVALID_ARG
    assert h.value is None
    assert lib.fa_launch_count(None) == 0
    assert lib.fa_set_wait_limits(None, 0, 0) == F.FA_E_INVALID_ARG
    assert lib.fa_set_raster_schedule(None, 64, 0) == F.FA_E_INVALID_ARG
    assert lib.fa_set_chart_pack_schedule(None, 1024, 1024) == F.FA_E_INVALID_ARG
    ks = F.fa_kernel_schedule()
    assert lib.fa_get_kernel_schedule(None, ctypes.byref(ks)) == F.FA_E_INVALID_ARG
    assert lib.fa_batch_get_kernel_schedule(None, ctypes.byref(ks)) == F.FA_E_INVALID_ARG
    lib.fa_destroy(None)
    lib.fa_mesh_release(None)
    out = ctypes.c_int32()
    assert lib.fa_last_device_status(None, None, ctypes.byref(out)) == F.FA_E_INVALID_ARG
    # frame entry points reject NULL handles before touching the device
    params = F.frame_params(np.eye(4, dtype=np.float32), 64, 64, 1.0, 10)
    fo = F.fa_frame_out()
    assert lib.fa_atlas_frame(None, None, ctypes.byref(params), ctypes.byref(fo), None) == F.FA_E_INVALID_ARG
    assert lib.fa_atlas_frame_dev_matrix(None, None, ctypes.byref(params), None, ctypes.byref(fo),
                                         None) == F.FA_E_INVALID_ARG
