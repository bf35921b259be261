"""The C ABI library loads and exports every entry point include/amrhydro.h declares,
and the ctypes mirror of its structs has the C layout (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_2411_14631_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(\S+)", out))
    declared = _declared()
    assert len(declared) >= 11
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_scope_entry_points_are_exported(built):
    """The four entry points of the hot path's boundary carry these exact names."""
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(\S+)", out))
    for name in ("amr_build_octree", "hydro_godunov_level", "hydro_courant", "reflux_level"):
        assert name in exported, name
        assert name in _declared(), name


def test_library_loads_and_binding_covers_header(built):
    from paper_2411_14631_gb300 import abi
    L = abi.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(abi.EXPORTS) <= set(_declared())
    assert L.amr_status_string(abi.EUNBALANCED) == b"octree violates the 2:1 rule"


def test_struct_layout_matches_c(tmp_path):
    import ctypes as C
    from paper_2411_14631_gb300 import abi
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "amrhydro.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu\\n", sizeof(amr_tree), sizeof(hydro_params),'
                   ' sizeof(amr_geom), offsetof(amr_tree, tile_slot), offsetof(hydro_params, d_counters));'
                   ' printf("%zu\\n", offsetof(amr_tree, ghost_cell));}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [C.sizeof(abi.AmrTree), C.sizeof(abi.HydroParams), C.sizeof(abi.AmrGeom),
                   abi.AmrTree.tile_slot.offset, abi.HydroParams.d_counters.offset, abi.AmrTree.ghost_cell.offset]


def test_query_is_host_only_and_validates(built):
    import ctypes as C
    import numpy as np
    from paper_2411_14631_gb300 import abi, workloads as W
    lx = W.uniform_tree(4)
    g = abi.AmrGeom(4, (C.c_int32 * 6)(*([1] * 6)))
    tb, wb = C.c_size_t(), C.c_size_t()
    assert abi.lib().amr_build_octree_query(C.byref(g), lx.ctypes.data_as(C.c_void_p), lx.shape[0],
                                            C.byref(tb), C.byref(wb)) == abi.OK
    assert tb.value > 0 and wb.value > 0
    g.levelmin = 1
    assert abi.lib().amr_build_octree_query(C.byref(g), lx.ctypes.data_as(C.c_void_p), lx.shape[0],
                                            C.byref(tb), C.byref(wb)) == abi.EINVAL
    g.levelmin = 4
    g.bc[0] = 0   # periodic on one face of an axis only
    assert abi.lib().amr_build_octree_query(C.byref(g), lx.ctypes.data_as(C.c_void_p), lx.shape[0],
                                            C.byref(tb), C.byref(wb)) == abi.EINVAL
    bad = lx.copy(); bad[0, 0] = 25
    g.bc[0] = 1
    assert abi.lib().amr_build_octree_query(C.byref(g), bad.ctypes.data_as(C.c_void_p), bad.shape[0],
                                            C.byref(tb), C.byref(wb)) == abi.EINVAL


def test_poisson_entry_points_validate_on_host(built, tmp_path):
    """The Poisson calls check their arguments before any CUDA call; the ctypes structs
    have the C layout."""
    import ctypes as C
    from paper_2411_14631_gb300 import abi
    L = abi.lib()
    n = 37 * 21 * 13
    nb = L.ppcg_workspace_bytes(37, 21, 13)
    assert nb >= 8 * n * 8 and L.ppcg_workspace_bytes(0, 21, 13) == 0
    assert L.poisson_apply(37, 21, 13, 5, C.c_void_p(256), C.c_void_p(512), None) == abi.EINVAL
    assert L.poisson_apply(0, 21, 13, abi.OP_A, C.c_void_p(256), C.c_void_p(512), None) == abi.EINVAL
    prm = abi.PpcgParams(37, 21, 13, abi.PRECOND_IP, 1e-4, 10, 0, 0, 0)
    w = C.c_void_p(1 << 20)
    assert L.ppcg_start(C.byref(prm), w, w, C.c_void_p((1 << 20) + 8), nb, None, None) == abi.EINVAL  # misaligned
    assert L.ppcg_start(C.byref(prm), w, w, w, nb - 1, None, None) == abi.ECAPACITY
    for bad in (dict(precond=3), dict(tol=-1.0), dict(max_iter=-1), dict(tile_y=12), dict(seg=2)):
        p2 = abi.PpcgParams(37, 21, 13, abi.PRECOND_IP, 1e-4, 10, 0, 0, 0)
        for k, v in bad.items():
            setattr(p2, k, v)
        assert L.ppcg_iterate(C.byref(p2), w, w, nb, None, 1, None) == abi.EINVAL, bad
    src = tmp_path / "pp.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ppcg.h"\n'
                   'int main(){printf("%zu %zu %zu %zu\\n", sizeof(ppcg_params), sizeof(ppcg_info),'
                   ' offsetof(ppcg_params, seg), offsetof(ppcg_info, eps));}\n')
    exe = tmp_path / "pp"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [C.sizeof(abi.PpcgParams), C.sizeof(abi.PpcgInfo), abi.PpcgParams.seg.offset,
                   abi.PpcgInfo.eps.offset]


def test_every_struct_field_offset_matches_c(tmp_path):
    """Each field of the ctypes mirrors sits at the offset the C compiler gives it (a swap
    of two equal-sized fields keeps the struct size and would pass a size check)."""
    from paper_2411_14631_gb300 import abi
    structs = {"amr_tree": abi.AmrTree, "hydro_params": abi.HydroParams, "amr_geom": abi.AmrGeom,
               "ppcg_params": abi.PpcgParams, "ppcg_info": abi.PpcgInfo}
    lines = []
    for cname, S in structs.items():
        for f in S._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    src = tmp_path / "off.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "amrhydro.h"\n#include "ppcg.h"\n'
                   'int main(){%s}\n' % "\n".join(lines))
    exe = tmp_path / "off"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, S in structs.items():
        for f in S._fields_:
            assert int(got["%s.%s" % (cname, f[0])]) == getattr(S, f[0]).offset, (cname, f[0])
