"""Kinematic pins and the paper's pulling scene (its second experiment) on the
GPU against the oracle."""
import numpy as np
import pytest

import cloth_scenes as cs
from test_gpu_parity import TOL_1, TOL_100, max_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mesh", ["sphere", "l6"])
def test_pulling_scene_parity(cloth_lib, oracle_lib, mesh):
    sc = cs.pulling_scene(48, mesh)
    p, _ = run_gpu(cloth_lib, sc, 1)
    x, _ = run_oracle(oracle_lib, sc, 1)
    assert max_err(p, x) <= TOL_1
    # the cloth reaches the model after about 120 steps
    p, v = run_gpu(cloth_lib, sc, 100)
    x, _ = run_oracle(oracle_lib, sc, 100)
    assert np.all(np.isfinite(p)) and max_err(p, x) <= TOL_100
    pin = sc.pinned.astype(bool)
    np.testing.assert_allclose(v[pin], np.broadcast_to(np.float32(sc.pin_velocity), v[pin].shape), rtol=0, atol=0)


def test_pulling_scene_contact_replay(cloth_lib, oracle_lib):
    # one step from oracle states while the cloth slides over the sphere
    sc = cs.pulling_scene(48, "sphere")
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    x, v = sc.init_pos, sc.init_vel
    done, contacts = 0, 0
    with cloth_lib.Cloth(sc) as g:
        for s in (160, 200, 240):
            x, v = oracle_lib.step(cl, x, v, done * sc.substeps, (s - done) * sc.substeps, grid)
            done = s
            x0, v0 = x.astype(np.float32), v.astype(np.float32)
            xo, _, hits = oracle_lib.step(cl, x0, v0, 0, sc.substeps, grid, want_hits=True)
            contacts += int((hits > 0).sum())
            g.set_state(x0, v0)
            g.step(1)
            p, _ = g.read()
            err = np.abs(p.astype(np.float64) - xo).max(axis=1)
            path = np.linalg.norm(xo - x0, axis=1) + np.linalg.norm(p.astype(np.float64) - x0, axis=1)
            assert np.all(err <= np.maximum(1e-5, 1.01 * path + 1e-7)), s
            assert (err > 1e-5).mean() <= 0.02, s
    assert contacts > 20


@pytest.mark.parametrize("flags", ["atomic", "edges"])
def test_kinematic_pins_in_the_other_paths(cloth_lib, oracle_lib, flags):
    sc = cs.pulling_scene(32, "sphere")
    f = {"atomic": cloth_lib.capi.CLOTH_FLAG_ATOMIC_SPRINGS, "edges": cloth_lib.capi.CLOTH_FLAG_EDGE_COLLISION}[flags]
    p, v = run_gpu(cloth_lib, sc, 20, flags=f)
    x, _ = run_oracle(oracle_lib, sc, 20)
    assert max_err(p, x) <= TOL_100
    pin = sc.pinned.astype(bool)
    assert np.all(v[pin][:, 0] == np.float32(sc.pin_velocity[0]))
