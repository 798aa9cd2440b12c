"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every entry point declared in include/oasis.h; argument errors are
reported before any device work."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1602_03643_gb300 import build, capi as c
    build.build()
    c.lib()
    return c


def declared_functions():
    src = open(os.path.join(ROOT, "include", "oasis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(oasis_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(capi):
    names = declared_functions()
    assert len(names) >= 18
    lib = capi.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(capi.SIGNATURES) == names


def test_header_constants_match_binding(capi):
    """Every #define the binding mirrors has the header's value; struct sizes agree."""
    import ctypes
    src = open(os.path.join(ROOT, "include", "oasis.h")).read()
    defs = dict(re.findall(r"#define\s+(OASIS_[A-Z0-9_]+)\s+(-?\d+)", src))
    shared = [k for k in defs if hasattr(capi, k)]
    assert len(shared) >= 8
    for k in shared:
        assert getattr(capi, k) == int(defs[k]), k
    assert ctypes.sizeof(capi.oasis_tuning) == 4 * 2 + 6 * 4 * 16 + 8 * 16 + 4 * 2 + 3 * 4 * 8 + 8 * 8 + 4 * 8
    assert ctypes.sizeof(capi.oasis_amg_info) == 8 + 2 * 8 * 16 + 8 + 8 * 16 + 4 * 16
    # C layouts written out by hand: 5 doubles + f[3], 3 int32 (+4 padding), a
    # double, 9 int32 (+4 padding); stats: 8 int32, 7 doubles, res_m[3], it_m, it_c, res_c
    assert ctypes.sizeof(capi.oasis_params) == 8 * 7 + 4 * 3 + 4 + 8 + 4 * 9 + 4
    assert ctypes.sizeof(capi.oasis_step_stats) == 4 * 8 + 8 * 7 + 8 * 3 + 4 + 4 + 8
    # kernel families of oasis_profile_read
    for name, v in capi.PROF_FAMILIES.items():
        assert int(defs["OASIS_PROF_" + name.upper()]) == v, name
    assert len(capi.PROF_FAMILIES) == len([k for k in defs if k.startswith("OASIS_PROF_")])


def test_version_and_error_string(capi):
    assert capi.oasis_version() >= 100
    assert isinstance(capi.lib().oasis_last_error(), bytes)


def test_null_pointer_is_einval(capi):
    import ctypes as C
    out = C.c_void_p()
    rc = capi.lib().oasis_mesh_create(3, 4, None, 1, None, None, 4, None, C.byref(out))
    assert rc == capi.OASIS_EINVAL
    assert b"null" in capi.lib().oasis_last_error()


def test_repeated_dof_is_emesh(capi):
    coords = np.array([[0, 0], [1, 0], [0, 1.0]])
    cells = np.array([[0, 1, 1]], np.int32)
    with pytest.raises(capi.OasisError) as e:
        capi.oasis_mesh_create(2, coords, cells)
    assert e.value.code == capi.OASIS_EMESH


def test_out_of_range_vertex_is_einval(capi):
    coords = np.array([[0, 0], [1, 0], [0, 1.0]])
    cells = np.array([[0, 1, 7]], np.int32)
    with pytest.raises(capi.OasisError) as e:
        capi.oasis_mesh_create(2, coords, cells)
    assert e.value.code == capi.OASIS_EINVAL


def test_bad_dim_is_einval(capi):
    with pytest.raises(capi.OasisError) as e:
        capi.oasis_mesh_create(4, np.zeros((5, 4)), np.zeros((1, 5), np.int32))
    assert e.value.code == capi.OASIS_EINVAL


def test_graft_entry_build():
    import __graft_entry__ as g
    g.build()


def test_struct_layouts_match_c_compiler(tmp_path, capi):
    """Field offsets of the ctypes mirrors equal what a C compiler makes of the header."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"oasis_params": capi.oasis_params, "oasis_step_stats": capi.oasis_step_stats,
               "oasis_tuning": capi.oasis_tuning, "oasis_amg_info": capi.oasis_amg_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "oasis.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert int(out[f"{name}.{f[0]}"]) == getattr(cls, f[0]).offset, (name, f[0])


def test_mesh_create_rejects_bad_input_before_any_device_work(capi):
    """oasis_mesh_create validates on the host first: these fail the same way
    with or without a GPU."""
    import ctypes as C
    lib = capi.lib()
    tri = np.array([[0, 0], [1, 0], [0, 1]], dtype=np.float64)

    def create(dim, cells, dof=None, n_dofs=3, coords=tri, n_cells=None, perm=None):
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        d = None if dof is None else np.ascontiguousarray(dof, dtype=np.int32)
        pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
        out = C.c_void_p()
        rc = lib.oasis_mesh_create(dim, coords.shape[0], coords.ctypes.data,
                                   cells.shape[0] if n_cells is None else n_cells, cells.ctypes.data,
                                   None if d is None else d.ctypes.data, n_dofs,
                                   None if pm is None else pm.ctypes.data, C.byref(out))
        return rc, lib.oasis_last_error().decode()

    assert create(4, [[0, 1, 2]])[0] == capi.OASIS_EINVAL                      # dimension
    assert create(2, [[0, 1, 2]], n_cells=0)[0] == capi.OASIS_EINVAL           # empty
    assert create(2, [[0, 1, 5]])[0] == capi.OASIS_EINVAL                      # vertex index
    assert create(2, [[0, 1, -1]])[0] == capi.OASIS_EINVAL
    assert create(2, [[0, 1, 2]], dof=[0, 1, 7])[0] == capi.OASIS_EINVAL       # dof map entry
    assert create(2, [[0, 1, 2]], dof=[0, 1, 2], n_dofs=4)[0] == capi.OASIS_EINVAL   # n_dofs > vertices
    rc, msg = create(2, [[0, 1, 1]])                                            # repeated vertex
    assert rc == capi.OASIS_EMESH and "repeated" in msg
    rc, msg = create(2, [[0, 1, 2]], dof=[0, 1, 1], n_dofs=2)                   # repeated dof (periodic map)
    assert rc == capi.OASIS_EMESH and "repeated" in msg
    # the dof renumbering must be a permutation of 0 .. n_dofs-1
    rc, msg = create(2, [[0, 1, 2]], perm=[0, 1, 3])
    assert rc == capi.OASIS_EINVAL and "perm" in msg
    rc, msg = create(2, [[0, 1, 2]], perm=[0, -1, 2])
    assert rc == capi.OASIS_EINVAL and "perm" in msg
    rc, msg = create(2, [[0, 1, 2]], perm=[2, 0, 2])
    assert rc == capi.OASIS_EINVAL and "permutation" in msg
    # a renumbered periodic map: perm has one entry per dof, not per vertex
    rc, msg = create(2, [[0, 1, 2]], dof=[0, 1, 1], n_dofs=2, perm=[1, 0])
    assert rc == capi.OASIS_EMESH and "repeated" in msg
