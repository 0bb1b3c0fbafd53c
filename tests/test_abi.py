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
    # the gain-operand setting is host state only: out-of-range values are
    # rejected, 0 (either placement, the default) is accepted
    assert lib.kx_set_gain_operand(3) == -1 and lib.kx_set_gain_operand(-1) == -1
    assert lib.kx_set_gain_operand(0) == 0


def test_struct_layouts_match_header(tmp_path):
    """ctypes layouts of the binding against the C compiler's sizeof and
    offsetof of the header's structs (x86-64)."""
    import subprocess
    import paper_2607_00755_b300 as kx
    structs = {"kx_grid_desc": kx.GridDesc, "kx_solve_params": kx.SolveParams, "kx_diag": kx.Diag,
               "kx_result": kx.Result, "kx_source": kx.Source, "kx_server_config": kx.ServerConfig,
               "kx_server_stats": kx.ServerStats, "kx_expansion": kx.Expansion,
               "kx_expansion_result": kx.ExpansionResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kx.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                               check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)
