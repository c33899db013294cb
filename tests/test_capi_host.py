"""CPU checks of the C ABI: the library builds, loads and exports every
symbol include/rt.h declares, and rt_create's host-side validation rejects
bad meshes before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from paper_2002_08377_gb300.inputs import build_mesh, level_symmetric

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rt.h")


@pytest.fixture(scope="module")
def lib():
    rtbuild.build()
    return capi.load()


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", txt)))


def test_header_symbols_exported(lib):
    names = header_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(capi.EXPORTS) == sorted(n for n in names if n in capi.EXPORTS)
    assert set(names) <= set(capi.EXPORTS) | set(getattr(capi, "EXTRA_EXPORTS", []))


def _desc(mesh, dirs, w, keep):
    def p(a, dt):
        a = np.ascontiguousarray(np.asarray(a, dt))
        keep.append(a)
        return a.ctypes.data

    d = capi.MeshDesc()
    d.n_cells, d.n_faces, d.n_angles = mesh.n_cells, mesh.n_faces, dirs.shape[0]
    d.cell_volume = p(mesh.cell_volume, np.float64)
    d.cell_centroid = p(mesh.cell_centroid, np.float64)
    d.face_cells = p(mesh.face_cells, np.int32)
    d.face_area = p(mesh.face_area, np.float64)
    d.face_normal = p(mesh.face_normal, np.float64)
    d.face_centroid = p(mesh.face_centroid, np.float64)
    d.face_w = None
    d.cell_face_ptr = p(mesh.cell_face_ptr, np.int64)
    d.cell_face_idx = p(mesh.cell_face_idx, np.int32)
    d.angle_dir = p(dirs, np.float64)
    d.angle_w = p(w, np.float64)
    return d


def _create(lib, mesh, dirs, w):
    keep = []
    d = _desc(mesh, dirs, w, keep)
    pr = capi.Params(10.0, 10.0, 1.0, 5.0 / 3.0, 1.0, 0.3, capi.RT_FP64, 64)
    st = ctypes.c_void_p()
    return lib.rt_create(ctypes.byref(d), ctypes.byref(pr), None, ctypes.byref(st)), st


def test_create_rejects_bad_meshes(lib):
    mesh = build_mesh((3, 3, 3), seed=1)
    dirs, w = level_symmetric(4)
    # open cell: drop one face's area
    m2 = build_mesh((3, 3, 3), seed=1)
    m2.face_area = m2.face_area.copy()
    m2.face_area[5] *= 0.5
    code, st = _create(lib, m2, dirs, w)
    assert code == capi.RT_ERR_MESH and not st.value
    # face index out of range
    m3 = build_mesh((3, 3, 3), seed=1)
    m3.face_cells = m3.face_cells.copy()
    m3.face_cells[0, 1] = 10 ** 6
    assert _create(lib, m3, dirs, w)[0] == capi.RT_ERR_MESH
    # CSR entry on the wrong side
    m4 = build_mesh((3, 3, 3), seed=1)
    m4.cell_face_idx = m4.cell_face_idx.copy()
    m4.cell_face_idx[0] = -m4.cell_face_idx[0] - 1
    assert _create(lib, m4, dirs, w)[0] == capi.RT_ERR_MESH
    # angle set without the antipodal ordering
    d2 = dirs.copy()
    d2[[0, 1]] = d2[[1, 0]]
    assert _create(lib, mesh, d2, w)[0] == capi.RT_ERR_ARG
    # weights not normalised
    assert _create(lib, mesh, dirs, w * 2)[0] == capi.RT_ERR_ARG


def test_create_rejects_degenerate_sizes_and_values(lib):
    """The degenerate inputs: no cells, an odd or too large angle count, a
    non-positive or non-finite cell volume, a NaN face area.  Each is refused
    before any device work, with no state returned."""
    import dataclasses
    mesh = build_mesh((3, 3, 3), seed=1)
    dirs, w = level_symmetric(4)
    keep = []
    d = _desc(mesh, dirs, w, keep)
    d.n_cells = 0
    pr = capi.Params(10.0, 10.0, 1.0, 5.0 / 3.0, 1.0, 0.3, capi.RT_FP64, 64)
    st = ctypes.c_void_p()
    assert lib.rt_create(ctypes.byref(d), ctypes.byref(pr), None, ctypes.byref(st)) == capi.RT_ERR_ARG
    assert not st.value
    d = _desc(mesh, dirs, w, keep)
    d.n_angles = dirs.shape[0] - 1
    assert lib.rt_create(ctypes.byref(d), ctypes.byref(pr), None, ctypes.byref(st)) == capi.RT_ERR_ARG
    big = np.concatenate([dirs] * 6)[:130]
    assert _create(lib, mesh, big, np.full(130, 1.0 / 130))[0] == capi.RT_ERR_ARG
    for bad in (0.0, -1.0, np.nan, np.inf):
        vol = mesh.cell_volume.copy()
        vol[4] = bad
        m2 = dataclasses.replace(mesh, cell_volume=vol)
        assert _create(lib, m2, dirs, w)[0] == capi.RT_ERR_MESH, bad
    area = mesh.face_area.copy()
    area[3] = np.nan
    assert _create(lib, dataclasses.replace(mesh, face_area=area), dirs, w)[0] == capi.RT_ERR_MESH


def test_create_rejects_bad_params(lib):
    """Flags outside {0, 1}, van Leer with the GCL, non-finite or too negative
    opacity exponents and T_ref <= 0 with an exponent are refused before any
    device work."""
    mesh = build_mesh((3, 3, 3), seed=1)
    dirs, w = level_symmetric(4)

    def code(**kw):
        keep = []
        d = _desc(mesh, dirs, w, keep)
        offs = np.ascontiguousarray(mesh.face_offset(), np.float64)  # van Leer's input, present
        keep.append(offs)
        d.face_offset = offs.ctypes.data
        pr = capi.Params(10.0, 10.0, 1.0, 5.0 / 3.0, 1.0, 0.3, capi.RT_FP64, 64)
        pr.T_ref = 1.0
        for k, v in kw.items():
            setattr(pr, k, v)
        st = ctypes.c_void_p()
        c = lib.rt_create(ctypes.byref(d), ctypes.byref(pr), None, ctypes.byref(st))
        assert not st.value
        return c

    for kw in ({"plain_launches": 2}, {"boost": -1}, {"gcl": 2}, {"integrator": 5},
               {"gcl": 1, "integrator": capi.RT_VAN_LEER}, {"beta_P": float("nan")},
               {"beta_P": -3.5}, {"beta_J": 1.0, "T_ref": 0.0}, {"precision": 7}, {"cfl": 0.0},
               {"float_quartic": 2}, {"hydro": 2}, {"hydro": 1, "gcl": 1}):
        assert code(**kw) == capi.RT_ERR_ARG, kw


def test_fp32_state_outside_float_range_refused(lib):
    """A float state of a mesh in physical units whose cbar A (or volume)
    leaves float range is refused by rt_create with RT_ERR_ARG before any
    device work; the same mesh is accepted up to that check in FP64 (it then
    needs a device, absent here)."""
    mesh = build_mesh((3, 3, 3), seed=1)
    dirs, w = level_symmetric(4)
    L = 3.0856775814913673e18  # one parsec in cm
    for arr, k in (("cell_volume", 3), ("face_area", 2)):
        setattr(mesh, arr, getattr(mesh, arr) * L ** k)
    keep = []
    d = _desc(mesh, dirs, w, keep)
    pr = capi.Params(2.99792458e10, 2.99792458e10, 7.565733e-15, 5.0 / 3.0, 8.25e7, 0.3,
                     capi.RT_FP32, 64)
    st = ctypes.c_void_p()
    assert lib.rt_create(ctypes.byref(d), ctypes.byref(pr), None, ctypes.byref(st)) == capi.RT_ERR_ARG
    assert not st.value


def test_null_arguments(lib):
    st = ctypes.c_void_p()
    assert lib.rt_create(None, None, None, ctypes.byref(st)) == capi.RT_ERR_ARG
    assert lib.rt_step(None, 0.0, None) == capi.RT_ERR_ARG
    assert lib.rt_step_io(None, 0.0, None, None) == capi.RT_ERR_ARG
    assert lib.rt_sync(None) == capi.RT_ERR_ARG
    assert lib.rt_totals(None, None) == capi.RT_ERR_ARG
    assert lib.rt_adjoint_step(None, 0.0, None, None, None, None, None, None, None, None, None,
                               None, None, 0) == capi.RT_ERR_ARG
    assert lib.rt_launch_count(None) == -1
    lib.rt_destroy(None)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of rt_mesh_desc and rt_params have the header's
    size and field offsets (compiled with the host C compiler)."""
    import subprocess
    inc = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rt.h"', "int main(void) {"]
    for cname, py in (("rt_mesh_desc", capi.MeshDesc), ("rt_params", capi.Params)):
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", inc, str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in (("rt_mesh_desc", capi.MeshDesc), ("rt_params", capi.Params)):
        assert int(got[cname]) == ctypes.sizeof(py)
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f
