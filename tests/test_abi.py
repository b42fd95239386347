"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/gbdart.h declares; calls that need no GPU
return status codes instead of crashing."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2609_09322_gb300 import build as gbuild
from paper_2609_09322_gb300 import gbdart

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gbdart.h")


def declared_in_header():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbd_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_in_header()
    for required in ("gbd_create", "gbd_destroy", "gbd_load_snapshots", "gbd_render", "gbd_render_batch",
                     "gbd_error_string", "gbd_last_error"):
        assert required in names


@pytest.mark.parametrize("checked", [False, True])
def test_library_exports_every_declared_symbol(checked):
    path = gbuild.build(checked=checked)[0]
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gbd_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in declared_in_header() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    lib = ctypes.CDLL(path)
    for n in declared_in_header():
        assert getattr(lib, n) is not None


def test_binding_covers_header():
    assert set(gbdart.declared_symbols()) <= set(declared_in_header())


def test_error_strings():
    lib = gbdart.load_library()
    for code in range(9):
        assert lib.gbd_error_string(code)
    assert lib.gbd_error_string(123) == b"unknown status"


def test_null_arguments_return_status():
    lib = gbdart.load_library()
    assert lib.gbd_create(None, 0, 0) == gbdart.ERR_INVALID
    assert b"NULL" in lib.gbd_last_error()
    assert lib.gbd_destroy(None) == gbdart.OK
    assert lib.gbd_render(None, 1, None, None, None, None) == gbdart.ERR_INVALID
    assert lib.gbd_render_batch(None, 1, None, 1, None, None, None) == gbdart.ERR_INVALID
    assert lib.gbd_load_snapshots(None, None, None, None) == gbdart.ERR_INVALID
    assert lib.gbd_unload(None, 1) == gbdart.ERR_INVALID


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = gbdart.load_library()
    h = ctypes.c_void_p()
    rc = lib.gbd_create(ctypes.byref(h), 0, 0)
    assert rc in (gbdart.ERR_CUDA, gbdart.ERR_INVALID)
    assert not h.value
    assert lib.gbd_last_error()
