"""CPU checks of the C ABI: the library builds, loads without a GPU and exports
every entry point that include/gbs.h declares; the binding declares them too."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def so_path():
    from paper_2106_01445_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gbs_build_state", "gbs_prob", "gbs_run_host", "gbs_gen_patterns", "gbs_create",
                 "gbs_destroy", "gbs_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(so_path):
    lib = ctypes.CDLL(so_path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol(so_path):
    from paper_2106_01445_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()
    L = _lib.load(so_path)
    assert L.gbs_version() >= 100


def test_create_without_gpu_fails_cleanly(so_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2106_01445_gb300 import _lib
    L = _lib.load(so_path)
    h = ctypes.c_void_p()
    assert L.gbs_create(ctypes.byref(h), 0, None) != 0
    assert not h.value


def test_null_context_is_rejected(so_path):
    from paper_2106_01445_gb300 import _lib
    L = _lib.load(so_path)
    assert L.gbs_prob(None, 4, None, None, None, 1, 0, 0, None, None, None, None) == _lib.GBS_E_INVALID
    assert L.gbs_build_state(None, 4, None, None, 1.0, None, None, None, None) == _lib.GBS_E_INVALID
    assert L.gbs_grad(None, 4, None, None, None, 1, None, None, None, None) == _lib.GBS_E_INVALID
    assert L.gbs_grad_approx(None, 4, None, None, None, 1, 2, None, None, None, None) == _lib.GBS_E_INVALID


def test_missing_library_is_an_error(tmp_path):
    # no fallback: without libgbs.so the binding refuses to load (the loaded-library
    # cache is set aside for the check and put back)
    from paper_2106_01445_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "libgbs.so"))
    finally:
        _lib._lib = saved
