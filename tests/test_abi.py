"""The C ABI loads, exports every function of include/*.h, and rejects bad arguments on the host."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"DWF_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def dw():
    from paper_2004_07732_gb300 import build
    build.build()
    import paper_2004_07732_gb300 as pkg
    return pkg


def test_header_declares_the_paper_calls():
    names = _declared_functions()
    for required in ("dwf_apply", "pv_apply", "dwf_pvdag_apply", "cgne_solve", "dwf_dot",
                     "dwf_convert_links", "dwf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(dw):
    L = ctypes.CDLL(dw._lib.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, f"missing exports: {missing}"


def test_sizes_and_host_side_argument_checks(dw):
    g = dw.make_geom((32, 32), 8)
    assert dw.spinor_size(g) == 32 * 32 * 8 * 2
    assert dw.link_size(g) == 2 * 32 * 32
    g4 = dw.make_geom((4, 4, 4, 8), 6, group="su3")
    assert dw.spinor_size(g4) == 4 * 4 * 4 * 8 * 6 * 12
    assert dw.link_size(g4) == 4 * 512 * 9
    L = dw.lib()
    bad = dw.make_geom((32, 32), 0)                       # Ls = 0
    assert L.dwf_apply(ctypes.byref(bad), None, None, None, 1.0, 0.01, 0, 0, None) == 1
    assert b"Ls" in L.dwf_last_error()
    bad = dw.make_geom((32, 32), 8, group="su3")          # 2-d SU(3) unsupported combination
    assert L.dwf_apply(ctypes.byref(bad), None, None, None, 1.0, 0.01, 0, 0, None) == 1
    g = dw.make_geom((32, 32), 8)
    assert L.dwf_apply(ctypes.byref(g), None, None, None, 1.0, 0.01, 0, 9, None) == 1     # bad precision
    assert L.dwf_apply(ctypes.byref(g), None, None, None, 1.0, 0.01, 0, 0, None) == 1     # NULL pointers
    assert b"NULL" in L.dwf_last_error()
    # aliasing psi and out is rejected before any device work
    fake = ctypes.c_void_p(4096)
    assert L.dwf_apply(ctypes.byref(g), fake, fake, fake, 1.0, 0.01, 0, 0, None) == 1
    assert L.cgne_solve(ctypes.byref(g), fake, fake, ctypes.c_void_p(8192), 1.0, 0.01, 0.0, 10, None, None) == 1
    # an empty lattice is a no-op
    empty = dw.make_geom((0, 4), 4)
    assert L.dwf_apply(ctypes.byref(empty), None, None, None, 1.0, 0.01, 0, 0, None) == 1   # L >= 1 required
    res = (ctypes.c_double * 2)()
    assert L.dwf_dot(None, None, 0, 0, res, None) == 0 and res[0] == 0.0


def test_packed_layout_sizes_and_checks(dw):
    g4 = dw.make_geom((3, 5, 2, 3), 4, group="su3")          # V = 90: three blocks of 32, the last padded
    assert dw.packed_spinor_size(g4) == 4 * 96 * 12
    assert dw.packed_link_size(g4) == 4 * 96 * 9
    g2 = dw.make_geom((32, 32), 8)
    assert dw.packed_spinor_size(g2) == 0 and dw.packed_link_size(g2) == 0
    L = dw.lib()
    fake, fake2 = ctypes.c_void_p(4096), ctypes.c_void_p(8192)
    assert L.dwf_apply_packed(ctypes.byref(g2), fake, fake, fake2, 1.8, 0.01, 0, 2, None) == 6   # 2-d: unsupported
    assert L.dwf_apply_packed(ctypes.byref(g4), None, None, None, 1.8, 0.01, 0, 2, None) == 1    # NULL pointers
    assert L.dwf_apply_packed(ctypes.byref(g4), fake, fake, fake, 1.8, 0.01, 0, 2, None) == 1    # psi == out
    assert L.dwf_apply_packed(ctypes.byref(g4), fake, ctypes.c_void_p(4100), fake2, 1.8, 0.01, 0, 2, None) == 1
    assert b"aligned" in L.dwf_last_error()
    assert L.dwf_pack_links(ctypes.byref(g4), fake, fake2, 0, None) == 1                        # F64 not packed
    assert L.dwf_pack_spinor(ctypes.byref(g4), fake, fake, None) == 1
    assert L.dwf_unpack_spinor(ctypes.byref(g2), fake, fake2, None) == 6


def _struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in include/dwf.h (comments removed)."""
    src = open(os.path.join(ROOT, "include", "dwf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            fields.append(re.sub(r"\[.*?\]", "", part).split()[-1].lstrip("*"))
    return fields


@pytest.mark.parametrize("cname,pyname", [("dwf_mg_params", "MgParams"), ("dwf_solve_stats", "SolveStats"),
                                          ("dwf_mg_level_params", "LevelParams"), ("dwf_geom", "Geom")])
def test_binding_structs_follow_the_header(cname, pyname):
    """The ctypes mirrors of the ABI structs list the header's fields in the header's order."""
    import paper_2004_07732_gb300._lib as L
    assert [f for f, _ in getattr(L, pyname)._fields_] == _struct_fields(cname)
