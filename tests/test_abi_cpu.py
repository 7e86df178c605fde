"""The C-ABI library builds, loads and exports every entry point that
include/gs.h declares, and the ctypes mirrors of its structs have the C
layout (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gs_status|int|size_t|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2603_04847_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_path():
    names = _declared()
    for n in ("gs_project", "gs_sort_tiles", "gs_render_fwd", "gs_render_bwd", "track_reproj_fwd_bwd",
              "pose_se3_update"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2603_04847_gb300 import _lib
    names = _declared()
    assert names
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.PROTOTYPES, "binding lacks " + n


def test_struct_layouts_match(lib):
    from paper_2603_04847_gb300 import _lib
    for i, s in enumerate(_lib.STRUCTS):
        assert lib.gs_struct_size(i) == ctypes.sizeof(s), s.__name__
    assert lib.gs_struct_size(99) == 0
    assert lib.gs_abi_version() == 5


def test_argument_errors_without_gpu(lib):
    """Validation happens before any CUDA call: null arguments are
    GS_ERR_ARG with a message, not a crash."""
    from paper_2603_04847_gb300 import _lib
    r = lib.gs_project(None, None, None, None, None, None)
    assert r == _lib.GS_ERR_ARG
    assert b"null" in lib.gs_last_error()
    b = _lib.gs_batch(0, 16, 0, 0, 0, 0, 0, 0)
    ws = ctypes.c_size_t(0)
    assert lib.gs_sort_tiles_workspace(10, ctypes.byref(b), 100, ctypes.byref(ws)) == _lib.GS_ERR_ARG
    b = _lib.gs_batch(1, 8, 1, 1, 1, 0, 0, 0)
    assert lib.gs_sort_tiles_workspace(10, ctypes.byref(b), 100, ctypes.byref(ws)) == _lib.GS_ERR_UNSUPPORTED
    assert lib.gs_step_advance(None, None) == _lib.GS_ERR_ARG
    assert lib.gs_zero(None, 0, None) == _lib.GS_OK


def test_product_raises_without_library(tmp_path):
    from paper_2603_04847_gb300 import _lib
    with pytest.raises(_lib.GsError):
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = None
