"""The edge-triangle narrow phase (CLOTH_FLAG_EDGE_COLLISION, the paper's own
detection) on the GPU against the oracle's reading of it.

Contact through edges is as chaotic as through node paths, so it is checked
by one-step replays from oracle states: both sides start from the same
float32 state.  A hit decided within float32 rounding of its threshold may
go either (valid) way; such a flip moves a node by at most the distance
between its previous position and the response, so: every node within
max(1e-5, |x_gpu - S| + |x_oracle - S|), and at most 2% of nodes beyond 1e-5.
"""
import numpy as np
import pytest

import cloth_scenes as cs
from helpers import floor_mesh, make_scene

pytestmark = pytest.mark.gpu


def _edge(P):
    return P.capi.CLOTH_FLAG_EDGE_COLLISION


def _replay(cloth_lib, oracle_lib, sc, steps):
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    x, v = sc.init_pos, sc.init_vel
    done, contacts = 0, 0
    with cloth_lib.Cloth(sc, flags=_edge(cloth_lib)) as g:
        for s in steps:
            x, v = oracle_lib.step_edges(cl, x, v, done * sc.substeps, (s - done) * sc.substeps, grid)
            done = s
            x0, v0 = x.astype(np.float32), v.astype(np.float32)
            xo, vo, hits = oracle_lib.step_edges(cl, x0, v0, 0, 1, grid, want_hits=True)
            contacts += int((hits > 0).sum())
            g.set_state(x0, v0)
            g.profile_substeps(1)  # one substep, as the oracle call above
            p, _ = g.read()
            S = x0.astype(np.float64)
            err = np.abs(p.astype(np.float64) - xo).max(axis=1)
            bound = np.linalg.norm(xo - S, axis=1) + np.linalg.norm(p.astype(np.float64) - S, axis=1)
            assert np.all(err <= np.maximum(1e-5, 1.01 * bound + 1e-7)), s
            assert (err > 1e-5).mean() <= 0.02, s
    return contacts


def test_edge_phase_replay_on_a_sphere(cloth_lib, oracle_lib):
    sc = cs.small_collision_scene(n=24, level=2, gap=0.002)
    assert _replay(cloth_lib, oracle_lib, sc, [3, 10, 20, 40, 60]) > 20


def test_edge_phase_replay_tilted_sheet_on_a_floor(cloth_lib, oracle_lib):
    # a sheet tilted against the floor, so its edges cross the floor plane
    nx, ny = 20, 16
    rng = np.random.default_rng(5)
    X0 = cs.flat_grid(nx, ny, (0.2, 0.004, 0.2), (0.02, 0.0, 0.0), (0.0, 0.0015, 0.025))
    pos = (X0 + rng.uniform(-5e-4, 5e-4, X0.shape)).astype(np.float32)
    vel = np.zeros_like(pos)
    vel[:, 1] = -1.5
    sc = make_scene(nx, ny, origin=(0.2, 0.004, 0.2), du=(0.02, 0, 0), dv=(0, 0.0015, 0.025), total_mass=0.3,
                    ks=(200.0, 100.0, 40.0), kd=(0.2, 0.1, 0.05), gravity=(0, -9.81, 0), dt=1 / 1200, substeps=4,
                    pos=pos, vel=vel, mesh=floor_mesh())
    assert _replay(cloth_lib, oracle_lib, sc, [1, 3, 6, 10]) > 20


def test_edge_mode_without_contact_equals_default(cloth_lib):
    sc = cs.config3("l5", n=96)  # falls for 20 steps without reaching the sphere
    with cloth_lib.Cloth(sc) as a, cloth_lib.Cloth(sc, flags=_edge(cloth_lib)) as b:
        a.step(20)
        b.step(20)
        pa, va = a.read()
        pb, vb = b.read()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)


def test_edge_mode_is_rejected_by_the_rollout(cloth_lib):
    sc = cs.small_collision_scene(n=12, level=2, gap=0.01)
    with cloth_lib.Cloth(sc, flags=_edge(cloth_lib)) as cl:
        import ctypes as C
        ro = C.c_void_p()
        rc = cloth_lib.capi.lib().cloth_rollout_create(C.c_void_p(cl.h), 4, 2, C.byref(ro))
        assert rc == cloth_lib.capi.CLOTH_ERR_INVALID_ARG


def test_edge_phase_lists_the_nodes_of_stretched_edges(cloth_lib, oracle_lib):
    # The paper's response moves a node towards a hit point on another edge of
    # its triangles, so in contact the cloth's edges can stretch to several
    # rest diagonals (up to 7 in the FP64 oracle on the sphere scene).  Here
    # one node sits 0.3 m below a floor and its neighbours 0.3 m above, far
    # outside any fixed margin around the floor, with the edges between them
    # crossing it.  The listing from the updated positions must still find
    # every node a hit affects: one substep matches the oracle, which tests
    # every edge of the cloth.
    # (placed so that no edge crosses the floor near the diagonal its two
    # triangles share, where a float32 and a double test can differ)
    nx = ny = 9
    sc = make_scene(nx, ny, origin=(0.213, 0.3, 0.2), du=(0.02, 0, 0), dv=(0, 0, 0.02), total_mass=0.2,
                    ks=(20.0, 10.0, 4.0), kd=(0.02, 0.02, 0.01), gravity=(0, -9.81, 0), dt=1 / 4800, substeps=1,
                    mesh=floor_mesh(), delta=1e-4)
    pos = sc.init_pos.copy()
    pos[4 * nx + 4, 1] = -0.3
    vel = np.zeros_like(pos)
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    xo, _, hits = oracle_lib.step_edges(cl, pos, vel, 0, 1, grid, want_hits=True)
    affected = np.nonzero(hits > 0)[0]
    assert len(affected) >= 4  # the neighbours of the low node
    far = affected[affected != 4 * nx + 4]
    assert np.all(pos[far, 1] > 0.25)  # 0.25 m or more above the floor
    with cloth_lib.Cloth(sc, flags=_edge(cloth_lib)) as g:
        g.set_state(pos, vel)
        g.step(1)
        p, _ = g.read()
    err = np.abs(p.astype(np.float64) - xo).max()
    assert err <= 1e-5, err
