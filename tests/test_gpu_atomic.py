"""The atomic spring path (Algorithm 1 as printed: one thread per spring,
FP32 atomic adds) against the FP64 oracle and the default fused walk.

Its additions happen in a run-dependent order, so it is held to the same
tolerances as the default path rather than to bitwise equality: <= 1e-5 m
after 1 step, <= 1e-3 m after 100 steps while no contact is sustained.
"""
import numpy as np
import pytest

import cloth_scenes as cs
from test_gpu_parity import SCENES, TOL_1, TOL_100, max_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _atomic(P):
    return P.capi.CLOTH_FLAG_ATOMIC_SPRINGS


@pytest.mark.parametrize("name", ["config1", "config3_small_wind", "config4", "ragged_45x19_floor", "contact24"])
def test_atomic_path_one_step_parity(cloth_lib, oracle_lib, name):
    sc = SCENES[name]()
    p, v = run_gpu(cloth_lib, sc, 1, flags=_atomic(cloth_lib))
    x, _ = run_oracle(oracle_lib, sc, 1)
    assert max_err(p, x) <= TOL_1


@pytest.mark.parametrize("name", ["config1", "config3_small_wind"])
def test_atomic_path_hundred_steps_parity(cloth_lib, oracle_lib, name):
    # no contact within the first 100 steps of these scenes
    sc = SCENES[name]()
    p, v = run_gpu(cloth_lib, sc, 100, flags=_atomic(cloth_lib))
    x, _ = run_oracle(oracle_lib, sc, 100)
    assert np.all(np.isfinite(p)) and np.all(np.isfinite(v))
    assert max_err(p, x) <= TOL_100


def test_atomic_path_matches_fused_walk_and_keeps_pins(cloth_lib):
    sc = cs.config3("l5", n=96)
    a = run_gpu(cloth_lib, sc, 1)
    b = run_gpu(cloth_lib, sc, 1, flags=_atomic(cloth_lib))
    assert max_err(a[0], b[0]) <= 1e-6 and max_err(a[1], b[1]) <= 1e-4
    p, v = run_gpu(cloth_lib, sc, 20, flags=_atomic(cloth_lib))
    pin = sc.pinned.astype(bool)
    assert np.array_equal(p[pin], sc.init_pos[pin]) and np.all(v[pin] == 0)


def test_atomic_path_contact_replay(cloth_lib, oracle_lib):
    # one step from oracle states in contact: the bound of the default path's
    # replay test (every node within max(1e-5, its path), <= 2% beyond 1e-5)
    sc = SCENES["contact_l4"]()
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    x, v = sc.init_pos, sc.init_vel
    done, contacts = 0, 0
    with cloth_lib.Cloth(sc, flags=_atomic(cloth_lib)) as g:
        for s in (5, 20, 40, 60, 80):
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


def test_atomic_path_profiles_and_rollout_forward(cloth_lib):
    sc = cs.small_collision_scene(24, level=2, gap=0.004, seed=5)
    with cloth_lib.Cloth(sc, flags=_atomic(cloth_lib)) as a, cloth_lib.Cloth(sc) as b:
        w, c = a.profile_substeps(2 * sc.substeps)
        b.step(2)
        assert w > 0 and c > 0
        assert max_err(a.read()[0], b.read()[0]) <= 1e-5


def test_atomic_path_is_rejected_by_the_rollout(cloth_lib):
    import ctypes as C
    sc = cs.small_collision_scene(n=12, level=2, gap=0.01)
    with cloth_lib.Cloth(sc, flags=_atomic(cloth_lib)) as cl:
        ro = C.c_void_p()
        rc = cloth_lib.capi.lib().cloth_rollout_create(C.c_void_p(cl.h), 4, 2, C.byref(ro))
        assert rc == cloth_lib.capi.CLOTH_ERR_INVALID_ARG
