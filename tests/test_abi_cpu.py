"""The C-ABI library builds, loads and exports every declared symbol; argument
validation fails before any GPU work; without a GPU the library reports an error
instead of falling back to the CPU. No kernel is launched here."""
import ctypes as C
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

needs_nvcc = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mosaicflow.h")).read()
    return sorted(set(re.findall(r"^\s*(?:mf_status|const char\*|int)\s+(mf_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def m():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_14258_gb300 import mosaicflow
    return mosaicflow


@needs_nvcc
def test_exports_every_declared_symbol(m):
    lib = m.load()
    decl = declared_symbols()
    assert len(decl) >= 12
    assert sorted(m.EXPORTS) == decl
    for name in decl:
        assert getattr(lib, name) is not None
    assert lib.mf_version() == 100


@needs_nvcc
def test_validation_before_gpu_work(m):
    lib = m.load()
    h = C.c_void_p()
    w = np.zeros(100, dtype=np.float32)
    assert lib.mf_load_sdnet(None, w.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
    assert lib.mf_load_sdnet(C.byref(m.SDNetDesc(96, 4)), w.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
    assert b"width" in lib.mf_last_error()
    assert lib.mf_load_sdnet(C.byref(m.SDNetDesc(64, 9)), w.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
    bc = np.zeros(1000)
    assert lib.mf_create_grid(C.byref(m.GridDesc(0, 2)), bc.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
    assert lib.mf_create_grid(C.byref(m.GridDesc(2, 200)), bc.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
    assert lib.mf_sweep(None, None, None, None, None) == m.MF_ERR_INVALID_ARG
    assert lib.mf_residual(None, None, None, None) == m.MF_ERR_INVALID_ARG
    assert lib.mf_grid_upload(None, None, 0, None) == m.MF_ERR_INVALID_ARG


@needs_nvcc
def test_no_cpu_fallback_without_gpu(m):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(m.MFError) as e:
        m.Grid(2, 2, np.zeros(4 * 64))
    assert e.value.status == m.MF_ERR_CUDA


def test_missing_library_fails_loudly(tmp_path):
    from paper_2308_14258_gb300 import mosaicflow
    saved = mosaicflow._lib
    mosaicflow._lib = None
    try:
        with pytest.raises(RuntimeError):
            mosaicflow.load(str(tmp_path / "nope.so"))
    finally:
        mosaicflow._lib = saved
