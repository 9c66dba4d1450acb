"""The C-ABI library loads and exports every entry point include/afr.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "afr.h")).read()
    return sorted(set(re.findall(r"^AFR_API\s+[\w\s\*]*?\b(afr_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_15876_gb300 import _lib
    from paper_2510_15876_gb300.build import build
    build()
    return _lib.load()


def test_header_declares_the_path():
    names = _declared()
    for n in ("afr_create", "afr_insert_samples", "afr_estimate_gradients", "afr_reproject", "afr_reconstruct",
              "afr_tile_feedback", "afr_reconstruct_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2510_15876_gb300 import _lib
    names = _declared()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_lib.EXPORTED) | set(names)
    assert set(_lib.EXPORTED) == set(names)


def test_invalid_config_is_rejected_on_host(lib):
    from paper_2510_15876_gb300 import _lib as L
    h = ctypes.c_void_p()
    for bad in (L.AfrConfig(0, 8, 4, 32, 4, 0, 1.0, 1e-4, 2.0), L.AfrConfig(8, 8, 33, 32, 4, 0, 1.0, 1e-4, 2.0),
                L.AfrConfig(8, 8, 4, 32, 9, 0, 1.0, 1e-4, 2.0), L.AfrConfig(8, 8, 4, 32, 4, 7, 1.0, 1e-4, 2.0),
                L.AfrConfig(8, 8, 4, 32, 4, 0, 0.0, 1e-4, 2.0)):
        assert lib.afr_create(ctypes.byref(bad), ctypes.byref(h)) == L.AFR_ERR_INVALID_ARG
    assert lib.afr_create(None, ctypes.byref(h)) == L.AFR_ERR_INVALID_ARG
    assert lib.afr_insert_samples(None, None, 0, None) == L.AFR_ERR_INVALID_ARG
    assert lib.afr_last_error(None) == b"null context"


def test_no_device_means_loud_failure(lib):
    """Without a usable GPU the library refuses to create a context (there is
    no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2510_15876_gb300 import _lib as L
    cfg = L.AfrConfig(8, 8, 4, 32, 4, 0, 1.0, 1e-4, 2.0)
    h = ctypes.c_void_p()
    assert lib.afr_create(ctypes.byref(cfg), ctypes.byref(h)) == L.AFR_ERR_CUDA
    from paper_2510_15876_gb300.api import Reconstructor
    with pytest.raises(Exception):
        Reconstructor(8, 8, 4, device="cuda")


def _declared_debug():
    txt = open(os.path.join(ROOT, "include", "afr_debug.h")).read()
    return sorted(set(re.findall(r"^AFR_API\s+[\w\s\*]*?\b(afr_\w+)\s*\(", txt, flags=re.M)))


def test_debug_library_exports_its_hooks(lib):
    """libafr_debug.so (the AFR_DEBUG build) exports the whole ABI plus the
    hooks of include/afr_debug.h; the release library has no hook."""
    from paper_2510_15876_gb300 import _lib
    dbg = _lib.load_debug()
    hooks = _declared_debug()
    assert hooks == sorted(_lib.DEBUG_EXPORTED)
    for n in _declared() + hooks:
        assert hasattr(dbg, n), n
    for n in hooks:
        assert not hasattr(lib, n), n


def test_null_handles_are_rejected_on_host(lib):
    """Every call that takes a context or a batch refuses a null one before
    touching the GPU (no device needed)."""
    from paper_2510_15876_gb300 import _lib as L
    prm = L.AfrParams(1, 0, 3, 1, 0, 1)
    assert lib.afr_insert_samples(None, None, 1, None) == L.AFR_ERR_INVALID_ARG
    assert lib.afr_insert_samples_ex(None, None, 1, 0, None, None) == L.AFR_ERR_INVALID_ARG
    assert lib.afr_insert_samples_ex(None, None, 0, L.AFR_INSERT_RESET, None, None) == L.AFR_ERR_INVALID_ARG
    assert lib.afr_estimate_gradients(None, 1.0, None) == L.AFR_ERR_INVALID_ARG
    assert lib.afr_reproject(None, 1.0, None) == L.AFR_ERR_INVALID_ARG
    assert lib.afr_batch_refresh(None, 1.0, ctypes.byref(prm), None, None) == L.AFR_ERR_INVALID_ARG
    assert lib.afr_batch_reconstruct(None, 1.0, ctypes.byref(prm), None, None) == L.AFR_ERR_INVALID_ARG
