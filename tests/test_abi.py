"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every symbol include/cloth.h declares, the ctypes mirror of every struct has
the C layout, and argument validation answers without touching a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cloth.h")


@pytest.fixture(scope="module")
def capi():
    from paper_2507_11794_gb300 import build as B
    B.build()
    from paper_2507_11794_gb300 import capi as A
    A.lib()
    return A


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cloth_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("cloth_create", "cloth_set_mesh", "cloth_step", "cloth_read", "cloth_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(capi):
    out = subprocess.run(["nm", "-D", "--defined-only", capi.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (cloth_\w+)", out))
    declared = set(header_functions())
    assert declared <= exported, declared - exported
    assert set(capi.EXPORTS) == declared


def test_struct_layout_matches_c(capi, tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "cloth.h"
#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("ClothDesc %zu\nClothWind %zu\nClothInfo %zu\nClothGridParams %zu\n", sizeof(ClothDesc), sizeof(ClothWind), sizeof(ClothInfo), sizeof(ClothGridParams));
  F(ClothDesc, ks_spring); F(ClothDesc, pinned); F(ClothDesc, gravity); F(ClothDesc, dt);
  F(ClothDesc, substeps); F(ClothDesc, mt_t_min); F(ClothDesc, wind); F(ClothDesc, flags); F(ClothDesc, pin_velocity);
  F(ClothInfo, substeps_done); F(ClothInfo, pos_planes); F(ClothInfo, vel_planes); F(ClothInfo, ntris);
  F(ClothInfo, grid_h); F(ClothInfo, grid_entries); F(ClothInfo, has_per_spring); F(ClothInfo, row_pitch);
  F(ClothGridParams, origin); F(ClothGridParams, dims); F(ClothGridParams, ncells); F(ClothGridParams, nentries);
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.rsplit(" ", 1) for l in lines if l)
    assert int(got["ClothDesc"]) == C.sizeof(capi.ClothDesc)
    assert int(got["ClothWind"]) == C.sizeof(capi.ClothWind)
    assert int(got["ClothInfo"]) == C.sizeof(capi.ClothInfo)
    assert int(got["ClothGridParams"]) == C.sizeof(capi.ClothGridParams)
    for key, val in got.items():
        if "." in key:
            T, m = key.split(".")
            assert int(val) == getattr(getattr(capi, T), m).offset, key


def _desc(capi, **kw):
    d = capi.ClothDesc()
    d.nx, d.ny = kw.get("nx", 4), kw.get("ny", 4)
    d.du[0], d.dv[2] = 0.1, 0.1
    d.total_mass = kw.get("total_mass", 1.0)
    d.dt = kw.get("dt", 1e-3)
    d.substeps = kw.get("substeps", 1)
    d.mt_eps = 1e-7
    d.restitution = -0.5
    return d


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", -3), ("substeps", 0), ("dt", 0.0), ("dt", float("nan")),
                                         ("total_mass", 0.0)])
def test_create_rejects_bad_desc_without_gpu(capi, field, value):
    # validation happens on the host before any CUDA call
    d = _desc(capi, **{field: value})
    h = C.c_void_p()
    rc = capi.lib().cloth_create(C.byref(d), None, C.byref(h))
    assert rc == capi.CLOTH_ERR_INVALID_ARG
    assert h.value is None
    assert capi.lib().cloth_last_error()


def test_null_arguments_are_rejected(capi):
    L = capi.lib()
    h = C.c_void_p()
    assert L.cloth_create(None, None, C.byref(h)) == capi.CLOTH_ERR_INVALID_ARG
    assert L.cloth_create(C.byref(_desc(capi)), None, None) == capi.CLOTH_ERR_INVALID_ARG
    assert L.cloth_step(None, 1) == capi.CLOTH_ERR_INVALID_ARG
    assert L.cloth_read(None, None, None) == capi.CLOTH_ERR_INVALID_ARG
    assert L.cloth_set_mesh(None, None, 0, None, 0) == capi.CLOTH_ERR_INVALID_ARG
    assert L.cloth_sync(None) == capi.CLOTH_ERR_INVALID_ARG
    L.cloth_destroy(None)  # NULL-safe


def test_batch_rejects_the_atomic_spring_flag_without_gpu(capi):
    d = (type(_desc(capi)) * 2)(_desc(capi), _desc(capi))
    d[1].flags = capi.CLOTH_FLAG_ATOMIC_SPRINGS
    b = C.c_void_p()
    assert capi.lib().cloth_batch_create(d, 2, None, C.byref(b)) == capi.CLOTH_ERR_INVALID_ARG
    assert b.value is None
    assert b"ATOMIC" in capi.lib().cloth_last_error()


def test_profile_entry_rejects_bad_arguments(capi):
    w = C.c_float()
    assert capi.lib().cloth_profile_substeps(None, 4, C.byref(w), None) == capi.CLOTH_ERR_INVALID_ARG


def test_nonfinite_parameters_are_rejected(capi):
    d = _desc(capi)
    d.gravity[1] = float("inf")
    h = C.c_void_p()
    assert capi.lib().cloth_create(C.byref(d), None, C.byref(h)) == capi.CLOTH_ERR_INVALID_ARG
    assert b"non-finite" in capi.lib().cloth_last_error()


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2507_11794_gb300 import capi as A
    monkeypatch.setattr(A, "_lib", None)
    monkeypatch.setattr(A, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        A.lib()


@pytest.mark.parametrize("nx,ny,what", [(1, 1 << 30, b"plane"), (1 << 16, 1 << 15, b"too many nodes"),
                                        (4, 1 << 28, b"32-bit state offsets")])
def test_create_rejects_the_largest_grids_without_gpu(capi, nx, ny, what):
    # kernels index a plane with 32-bit offsets: a padded plane of 2^31 floats
    # or more, six planes of 2^32 floats or more, or more than 2^30 nodes, are
    # refused before any allocation
    d = _desc(capi, nx=nx, ny=ny)
    h = C.c_void_p()
    assert capi.lib().cloth_create(C.byref(d), None, C.byref(h)) == capi.CLOTH_ERR_INVALID_ARG
    assert h.value is None
    assert what in capi.lib().cloth_last_error()


def test_rollout_entry_points_reject_null_arguments(capi):
    L = capi.lib()
    r = C.c_void_p()
    assert L.cloth_rollout_create(None, 8, 2, C.byref(r)) == capi.CLOTH_ERR_INVALID_ARG
    assert r.value is None
    assert L.cloth_rollout_create(None, 8, 2, None) == capi.CLOTH_ERR_INVALID_ARG
    assert L.cloth_rollout_forward(None, None, None, None, None, None) == capi.CLOTH_ERR_INVALID_ARG
    assert L.cloth_rollout_backward(None, None, None, None, None, None) == capi.CLOTH_ERR_INVALID_ARG
    L.cloth_rollout_destroy(None)  # NULL-safe


def _static_reject(capi, verts, tris):
    # limits are checked on the host before any CUDA call (no GPU needed)
    rc, prm = capi.cloth_grid_build_static(verts, tris, 0, 0, 0, 0, 0, 0)
    return rc, prm, capi.lib().cloth_last_error()


def test_static_grid_rejects_too_many_vertices_alone(capi):
    import numpy as np
    nv = 131073  # one over the vertex limit, with a single triangle
    verts = np.zeros((nv, 3), np.float32)
    verts[1, 0] = verts[2, 1] = 1.0
    tris = np.array([[0, 1, 2]], np.int32)
    rc, _, msg = _static_reject(capi, verts, tris)
    assert rc == capi.CLOTH_ERR_INVALID_ARG and b"static limits" in msg and b"131073 vertices" in msg


def test_static_grid_rejects_too_many_triangles_alone(capi):
    import numpy as np
    nt = 131073
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    tris = np.tile(np.array([0, 1, 2], np.int32), (nt, 1))
    rc, _, msg = _static_reject(capi, verts, tris)
    assert rc == capi.CLOTH_ERR_INVALID_ARG and b"131073 triangles" in msg


def test_static_grid_rejects_a_grid_over_the_cell_limit(capi):
    import numpy as np
    # two triangles of side 5 mm at opposite corners of a unit cube: the cell
    # is twice the mean longest side (1 cm), so the grid has about 104^3 cells
    s = 0.005
    verts = np.array([[0, 0, 0], [s, 0, 0], [0, s, 0], [1, 1, 1], [1 - s, 1, 1], [1, 1 - s, 1]], np.float32)
    tris = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    rc, prm, msg = _static_reject(capi, verts, tris)
    assert rc == capi.CLOTH_ERR_INVALID_ARG and b"cells exceeds the static limit" in msg
    assert prm.ncells > 262144 and prm.ncells == prm.dims[0] * prm.dims[1] * prm.dims[2]


def test_status_codes_match_the_header(capi):
    src = open(HEADER).read()
    codes = dict((n, int(v)) for n, v in re.findall(r"\bCLOTH_(OK|ERR_\w+)\s*=\s*(-?\d+)", src))
    assert codes["OK"] == 0 and len(codes) >= 8
    for name, val in codes.items():
        assert getattr(capi, "CLOTH_" + name) == val, name
