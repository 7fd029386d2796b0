"""Host-side checks of the C ABI (no GPU needed): libgi.so loads, exports
every symbol include/gi.h declares, and rejects bad arguments before any
CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gi.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_08551_gb300 import _lib
    return _lib.load()


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^GI_API [^;]*?\b(gi_\w+)\(", src, flags=re.M)))


def test_header_declares_the_path():
    names = declared()
    for want in ("gi_project", "gi_bin_tiles", "gi_render", "gi_render_backward", "gi_vq_decode",
                 "gi_fit_create", "gi_fit_step", "gi_fit_destroy", "gi_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2403_08551_gb300 import _lib
    for name in declared():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"
    assert set(_lib.SIGNATURES) == set(declared())


def test_version_and_status_strings(lib):
    assert lib.gi_abi_version() == 8
    assert lib.gi_status_string(0) == b"GI_OK"
    assert lib.gi_status_string(3) == b"GI_ERR_CAPACITY"


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2403_08551_gb300 import _lib
    img_bad = _lib.GIImage(64, 64, 12)
    rc = lib.gi_project(None, None, None, 10, img_bad, None, None, None, None)
    assert rc == 1 and b"tile" in lib.gi_last_error()
    img = _lib.GIImage(64, 64, 16)
    rc = lib.gi_project(None, None, None, 10, img, None, None, None, None)
    assert rc == 1 and b"NULL" in lib.gi_last_error()
    sz = ctypes.c_size_t(0)
    assert lib.gi_bin_workspace_size(100, img, 0, ctypes.byref(sz)) == 1
    assert lib.gi_bin_workspace_size(100, img, 1 << 30, ctypes.byref(sz)) == 1
    # few tiles: count-matrix binning, scratch sized by chunks x tiles, not by capacity
    assert lib.gi_bin_workspace_size(1000, img, 5000, ctypes.byref(sz)) == 0 and sz.value >= 8 * 16 * 4
    small = sz.value
    assert lib.gi_bin_workspace_size(1000, img, 50000, ctypes.byref(sz)) == 0 and sz.value == small
    # many tiles: radix binning, two key/value buffers of the pair capacity
    big = _lib.GIImage(4096, 4096, 16)
    assert lib.gi_bin_workspace_size(100, big, 5000, ctypes.byref(sz)) == 0 and sz.value > 5000 * 8
    small = sz.value
    assert lib.gi_bin_workspace_size(100, big, 50000, ctypes.byref(sz)) == 0 and sz.value > small
    assert lib.gi_backward_workspace_size(100, img, 5000, ctypes.byref(sz)) == 0 and sz.value >= 5000 * 32
    # n = 0 is a no-op that needs no pointers
    assert lib.gi_project(None, None, None, 0, img, None, None, None, None) == 0
    assert lib.gi_vq_decode(None, None, None, 5, 0, 256, None, None, None, None) == 1
    assert lib.gi_vq_decode(None, None, None, 5, 2, 257, None, None, None, None) == 1
    desc = _lib.GIFitDesc()
    h = ctypes.c_void_p()
    assert lib.gi_fit_create(ctypes.byref(desc), None, ctypes.byref(h)) == 1


def test_product_does_not_import_oracle():
    """The product package never references the oracle (test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2403_08551_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "gi_oracle" not in txt and "gio_" not in txt, f
