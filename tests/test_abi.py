"""The C-ABI library builds, loads and exports every symbol include/pot.h
declares.  Host-only calls run; nothing here launches a kernel."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2601_05765_b300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lgc_compute_cells" in names and "pot_newton_solve" in names and "pot_fluid_step" in names
    for name in names:
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    from paper_2601_05765_b300 import pot
    p = pot.default_params()
    assert p.tol == 1e-4 and p.max_newton == 100 and p.max_halvings == 30
    assert abs(p.gravity[2] + 9.81) < 1e-12 and p.eps == 0.01
    lib.pot_status_string.restype = ctypes.c_char_p
    assert lib.pot_status_string(0) == b"ok"
    assert b"coincident" in lib.pot_status_string(4)
    # invalid arguments are rejected before any device call
    h = ctypes.c_void_p()
    assert lib.pot_create(ctypes.byref(h), 0, ctypes.c_int64(0), 64, 3) == 1
    assert lib.pot_create(ctypes.byref(h), 0, ctypes.c_int64(10), 1025, 3) == 1
    assert lib.pot_create(ctypes.byref(h), 0, ctypes.c_int64(10), 64, 0) == 1
    assert lib.lgc_compute_cells(None, None, ctypes.c_int64(10), None, None, None, None, None, None,
                                 None, None, None, None) == 1
    assert lib.pot_destroy(None) == 0


def test_struct_layouts_match_header(lib, tmp_path):
    """ctypes mirrors of the header's structs: size and every field offset
    agree with what the C compiler makes of include/pot.h."""
    import subprocess

    from paper_2601_05765_b300 import pot
    structs = {"pot_domain": pot.Domain, "pot_csr": pot.Csr, "pot_cell_stats": pot.CellStats,
               "pot_params": pot.Params, "pot_solve_stats": pot.SolveStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pot.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)
