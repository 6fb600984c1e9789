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
    assert lib.mf_version() == 300


@needs_nvcc
def test_validation_before_gpu_work(m):
    lib = m.load()
    h = C.c_void_p()
    w = np.zeros(100, dtype=np.float32)
    assert lib.mf_load_sdnet(None, None, w.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
    assert lib.mf_load_sdnet(None, C.byref(m.SDNetDesc(96, 4)), w.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
    assert b"width" in lib.mf_last_error()
    assert lib.mf_load_sdnet(None, C.byref(m.SDNetDesc(64, 9)), w.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
    bc = np.zeros(1000)
    assert lib.mf_create_grid(None, C.byref(m.GridDesc(0, 2)), bc.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
    assert lib.mf_create_grid(None, C.byref(m.GridDesc(2, 200)), bc.ctypes.data, C.byref(h)) == m.MF_ERR_INVALID_ARG
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


@needs_nvcc
def test_every_entry_point_validates_before_gpu_work(m):
    """Each call the header documents with MF_ERR_INVALID_ARG rejects a bad argument
    without touching the device (this machine has none, so a call that reached CUDA
    would report MF_ERR_CUDA instead)."""
    lib = m.load()
    bad = m.MF_ERR_INVALID_ARG
    h = C.c_void_p()
    w = np.zeros(200000, dtype=np.float32)
    # SDNet variants: activation, embedding channels and kernel size out of range
    ex = m.SDNetDescEx
    assert lib.mf_load_sdnet_ex(None, C.byref(ex(128, 6, 7, 0, 0)), w.ctypes.data, C.byref(h)) == bad
    assert lib.mf_load_sdnet_ex(None, C.byref(ex(128, 6, 1, 17, 5)), w.ctypes.data, C.byref(h)) == bad
    assert lib.mf_load_sdnet_ex(None, C.byref(ex(128, 6, 1, 8, 4)), w.ctypes.data, C.byref(h)) == bad
    assert lib.mf_load_sdnet_ex(None, None, w.ctypes.data, C.byref(h)) == bad
    assert lib.mf_load_sdnet(None, C.byref(m.SDNetDesc(64, 4)), None, C.byref(h)) == bad
    # batches: count, descriptor and sizes
    descs = (m.GridDesc * 2)(m.GridDesc(2, 2), m.GridDesc(0, 2))
    bc = np.zeros(10000)
    assert lib.mf_create_batch(None, 0, descs, bc.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_batch(None, 2, None, bc.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_batch(None, 2, descs, bc.ctypes.data, C.byref(h)) == bad
    nx, ny, off = C.c_int(), C.c_int(), C.c_longlong()
    assert lib.mf_batch_info(None, 0, C.byref(nx), C.byref(ny), C.byref(off)) == bad
    assert lib.mf_batch_upload(None, 0, None, 0, None) == bad
    assert lib.mf_batch_download(None, 0, None, 0, None) == bad
    assert lib.mf_batch_sweep(None, None, None, None, None) == bad
    assert lib.mf_batch_residual(None, 0, None, None, None) == bad
    # single grids
    assert lib.mf_grid_dims(None, C.byref(nx), C.byref(ny)) == bad
    assert lib.mf_grid_download(None, None, 0, None) == bad
    assert lib.mf_create_grid(None, C.byref(m.GridDesc(2, 2)), None, C.byref(h)) == bad
    # allocation-free sweep: null grid, size limits
    d = C.c_double()
    assert lib.mf_sweep_noalloc(None, 2, 2, None, 0, 1, C.byref(d), None) == bad
    u = np.zeros(65 * 65, dtype=np.float32)
    assert lib.mf_sweep_noalloc(u.ctypes.data, 0, 2, None, 0, 1, C.byref(d), None) == bad
    assert lib.mf_sweep_noalloc(u.ctypes.data, 33, 2, None, 0, 1, C.byref(d), None) == bad
    # failure-detection self-test: the limit must lie in (0, 1000] ms
    n = C.c_int()
    assert lib.mf_check_wait_timeout(0.0, C.byref(n)) == bad
    assert lib.mf_check_wait_timeout(2000.0, C.byref(n)) == bad
    # trainer: options, sizes and weights
    td = m.TrainDesc

    def desc(width=128, depth=6, prec=1, opt=1, F=4, P=128, engine=0):
        return td(width, depth, prec, opt, F, P, 0.9, 0.999, 1e-6, 0.0, engine)

    from paper_2308_14258_gb300 import inputs as I
    tw = I.xavier_sdnet(I.SDNetShape(128, 6), 0)
    assert lib.mf_create_trainer(None, None, tw.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_trainer(None, C.byref(desc(width=96)), tw.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_trainer(None, C.byref(desc(depth=9)), tw.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_trainer(None, C.byref(desc(prec=5)), tw.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_trainer(None, C.byref(desc(opt=3)), tw.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_trainer(None, C.byref(desc(P=100)), tw.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_trainer(None, C.byref(desc(F=0)), tw.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_trainer(None, C.byref(desc(F=1 << 20, P=1 << 12)), tw.ctypes.data, C.byref(h)) == bad
    assert lib.mf_create_trainer(None, C.byref(desc()), None, C.byref(h)) == bad
    wn = tw.copy()
    wn[5] = np.nan
    assert lib.mf_create_trainer(None, C.byref(desc()), wn.ctypes.data, C.byref(h)) == bad
    assert b"finite" in lib.mf_last_error() or b"weight" in lib.mf_last_error()
    loss = (C.c_double * 3)()
    assert lib.mf_train_grad(None, 1, 64, 64, None, None, None, None, loss, None) == bad
    assert lib.mf_train_step(None, 1, 64, 64, None, None, None, None, 1e-3, loss, None) == bad
    assert lib.mf_trainer_set_weights(None, None, 0, None) == bad
    assert lib.mf_trainer_get_weights(None, None, 0, None) == bad
    assert lib.mf_trainer_get_grads(None, None, 0, None) == bad


@needs_nvcc
def test_context_calls_validate_and_report_no_device(m):
    """mf_ctx_create rejects a bad index or a null result pointer before touching CUDA;
    on this machine (no GPU) a valid request reports MF_ERR_CUDA. The creating calls
    check their descriptors before they look at the context, and a null context is
    rejected by name."""
    import torch
    lib = m.load()
    bad = m.MF_ERR_INVALID_ARG
    c = C.c_void_p()
    assert lib.mf_ctx_create(-1, C.byref(c)) == bad
    assert lib.mf_ctx_create(0, None) == bad
    assert lib.mf_ctx_create(10**6, C.byref(c)) == bad
    assert lib.mf_ctx_device(None, None, None) == bad
    assert lib.mf_ctx_destroy(None) == m.MF_OK
    if not torch.cuda.is_available():
        assert lib.mf_ctx_create(0, C.byref(c)) == m.MF_ERR_CUDA
        assert not c.value
    h = C.c_void_p()
    w = np.zeros(200000, dtype=np.float32)
    assert lib.mf_load_sdnet(None, C.byref(m.SDNetDesc(96, 4)), w.ctypes.data, C.byref(h)) == bad
    assert b"width" in lib.mf_last_error()
    assert lib.mf_load_sdnet(None, C.byref(m.SDNetDesc(64, 4)), w.ctypes.data, C.byref(h)) == bad
    assert b"context" in lib.mf_last_error()
    bc = np.zeros(1000)
    assert lib.mf_create_grid(None, C.byref(m.GridDesc(2, 2)), bc.ctypes.data, C.byref(h)) == bad
    assert b"context" in lib.mf_last_error()
    descs = (m.GridDesc * 1)(m.GridDesc(2, 2))
    assert lib.mf_create_batch(None, 1, descs, bc.ctypes.data, C.byref(h)) == bad
    assert b"context" in lib.mf_last_error()
    from paper_2308_14258_gb300 import inputs as I
    tw = I.xavier_sdnet(I.SDNetShape(128, 6), 0)
    td = m.TrainDesc(128, 6, 1, 1, 4, 128, 0.9, 0.999, 1e-6, 0.0, 0)
    assert lib.mf_create_trainer(None, C.byref(td), tw.ctypes.data, C.byref(h)) == bad
    assert b"context" in lib.mf_last_error()
    wn = tw.copy()
    wn[7] = np.inf
    assert lib.mf_create_trainer(None, C.byref(td), wn.ctypes.data, C.byref(h)) == bad
    assert b"finite" in lib.mf_last_error()
