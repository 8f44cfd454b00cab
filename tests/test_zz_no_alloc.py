"""The allocation-free grid build (cloth_grid_build_static) against the grid
that cloth_set_mesh builds for the same mesh.

cloth_grid_build_static serves callers that must not allocate device memory
(hosts under a fixed-budget allocator, or that forbid cudaMalloc once
start-up is over): its temporaries live in a fixed device array of the
library and the caller passes the output buffers.  Here the test is the
caller: it sizes and allocates the outputs with torch, calls the entry point
through the C ABI, and compares every output with the existing path bit for
bit (the grid is integer data).  Two meshes are built back to back so that
the second call runs on scratch memory left over from the first, and a
repeated call must leave the device's free memory unchanged.
"""
import numpy as np
import pytest

import cloth_scenes as cs
from helpers import make_scene

pytestmark = pytest.mark.gpu


def _static_grid(P, torch, verts, tris):
    A = P.capi
    stream = int(torch.cuda.current_stream().cuda_stream)
    rec = torch.empty(12 * len(tris), dtype=torch.float32, device="cuda")
    # size the outputs from the entry point's own answers (zero capacities)
    rc, prm = A.cloth_grid_build_static(verts, tris, stream, rec.data_ptr(), 0, 0, 0, 0)
    assert rc == A.CLOTH_ERR_INVALID_ARG and prm.ncells > 0
    cell_start = torch.empty(prm.ncells + 1, dtype=torch.int32, device="cuda")
    rc, prm = A.cloth_grid_build_static(verts, tris, stream, rec.data_ptr(), cell_start.data_ptr(),
                                        cell_start.numel(), 0, 0)
    assert rc == A.CLOTH_ERR_INVALID_ARG and prm.nentries > 0
    tri_ids = torch.empty(prm.nentries, dtype=torch.int32, device="cuda")
    rc, prm = A.cloth_grid_build_static(verts, tris, stream, rec.data_ptr(), cell_start.data_ptr(),
                                        cell_start.numel(), tri_ids.data_ptr(), tri_ids.numel())
    assert rc == A.CLOTH_OK, A.lib().cloth_last_error()
    torch.cuda.synchronize()
    return prm, cell_start.cpu().numpy(), tri_ids.cpu().numpy(), rec.cpu().numpy().reshape(-1, 3, 4)


def test_static_grid_build_matches_set_mesh_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11794_gb300 import build as B
    B.build()
    import paper_2507_11794_gb300 as P

    meshes = [(cs.config3("l6", n=8).mesh_verts, cs.config3("l6", n=8).mesh_tris),
              cs.sphere_mesh(2, 0.3, (0.0, -0.5, 0.0))]
    for verts, tris in meshes:
        prm, cs_static, ids_static, rec = _static_grid(P, torch, verts, tris)
        with P.Cloth(make_scene(4, 4, mesh=(verts, tris))) as cl:
            info = cl.info()
            cs_ref, ids_ref = cl.grid()
        assert prm.h == info.grid_h and prm.inv == info.grid_inv
        assert tuple(prm.origin) == tuple(info.grid_origin) and tuple(prm.dims) == tuple(info.grid_dims)
        assert prm.nentries == info.grid_entries
        assert np.array_equal(cs_static, cs_ref)
        assert np.array_equal(ids_static, ids_ref)
        # triangle records: first vertex and edge vectors of every triangle
        v = verts.astype(np.float32)
        np.testing.assert_array_equal(rec[:, 0, :3], v[tris[:, 0]])
        np.testing.assert_array_equal(rec[:, 1, :3], v[tris[:, 1]] - v[tris[:, 0]])
        np.testing.assert_array_equal(rec[:, 2, :3], v[tris[:, 2]] - v[tris[:, 0]])


def test_static_grid_build_allocates_nothing():
    """Once the first call on the device has loaded the library's module, a
    call changes the device's free memory by nothing."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11794_gb300 import build as B
    B.build()
    import paper_2507_11794_gb300 as P

    verts, tris = cs.sphere_mesh(3, 0.3, (0.0, 0.0, 0.0))
    first = _static_grid(P, torch, verts, tris)
    A = P.capi
    stream = int(torch.cuda.current_stream().cuda_stream)
    prm0 = first[0]
    rec = torch.empty(12 * len(tris), dtype=torch.float32, device="cuda")
    cell_start = torch.empty(prm0.ncells + 1, dtype=torch.int32, device="cuda")
    tri_ids = torch.empty(prm0.nentries, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        rc, prm = A.cloth_grid_build_static(verts, tris, stream, rec.data_ptr(), cell_start.data_ptr(),
                                            cell_start.numel(), tri_ids.data_ptr(), tri_ids.numel())
        assert rc == A.CLOTH_OK, A.lib().cloth_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(cell_start.cpu().numpy(), first[1])
    assert np.array_equal(tri_ids.cpu().numpy(), first[2])
