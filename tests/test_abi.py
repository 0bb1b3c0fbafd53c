"""Host-only checks of the C-ABI library: it builds, loads without a GPU and
exports every entry point that include/*.h declares (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:[A-Za-z_][\w ]*?[\s\*]+)(kx_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_00755_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("kx_build_kernel", "kx_collision", "kx_step", "kx_solve", "kx_create",
                     "kx_destroy", "kx_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_exports(lib):
    import paper_2607_00755_b300 as kx
    for name in kx.EXPORTS:
        assert hasattr(lib, name)
    assert set(kx.EXPORTS) <= set(declared_functions())


def test_strerror_and_error_paths_without_gpu(lib):
    lib.kx_strerror.restype = ctypes.c_char_p
    assert lib.kx_strerror(0) == b"ok"
    assert b"invalid" in lib.kx_strerror(-1)
    # null arguments are rejected before any CUDA call
    assert lib.kx_create(None, 0, None) == -1
    assert lib.kx_build_kernel(None, None, None) == -1
    assert lib.kx_collision(None, None, 1, None, None, None, 1, None) == -1


def test_struct_layouts_match_header():
    import paper_2607_00755_b300 as kx
    # sizes follow the C declarations (x86-64 ABI)
    assert ctypes.sizeof(kx.GridDesc) == 48
    assert ctypes.sizeof(kx.SolveParams) == 8 * 8 + 4 * 4
    assert ctypes.sizeof(kx.Diag) == 9 * 8 + 2 * 4
    assert ctypes.sizeof(kx.Result) == 6 * 8 + 3 * 8 + 2 * 4
    assert ctypes.sizeof(kx.Source) == 40
