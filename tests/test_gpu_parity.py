"""GPU (CUDA, FP32) vs FP64 oracle parity through the C ABI.

Tolerances (the workloads' accuracy targets, cloth extent 1 m):
  max |x_gpu - x_oracle| <= 1e-5 m after 1 step and <= 1e-3 m after 100 steps.
Integer work is compared bit for bit: the grid (cell_start, tri_ids and its
parameters) and every broad-phase candidate set on identical float32 inputs.
"""
import dataclasses

import numpy as np
import pytest

import cloth_scenes as cs
from helpers import floor_mesh, make_scene, ray_parity_inside

pytestmark = pytest.mark.gpu

TOL_1 = 1e-5
TOL_100 = 1e-3


def run_gpu(P, sc, steps, **kw):
    with P.Cloth(sc, **kw) as cl:
        cl.step(steps)
        return cl.read()


def run_oracle(oracle_lib, sc, steps):
    return oracle_lib.run(sc, steps)


def max_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))))


SCENES = {
    "config1": lambda: cs.config1(),
    "contact24": lambda: cs.small_collision_scene(n=24, level=2, gap=0.002),
    "contact_l4": lambda: cs.small_collision_scene(n=64, level=4, gap=0.001, seed=7),
    "config4": lambda: cs.config4(),
    "config3_small_wind": lambda: cs.config3("l5", n=96),
    "contact37_l3": lambda: cs.small_collision_scene(n=37, level=3, gap=0.003),
}


def _ragged_scene():
    # non-square, ragged tiles in both directions, pins, wind, a floor
    nx, ny = 45, 19
    w = cs.Wind(1.5, (0.3, 0.0, 0.9), (0.6, 0.0, 0.8), 2.0, 9.0, 0.7)
    rng = np.random.default_rng(17)
    X0 = cs.flat_grid(nx, ny, (0.05, 0.01, 0.05), (0.02, 0.0, 0.0), (0.0, 0.0, 0.045))
    pos = X0 + rng.uniform(-1e-3, 1e-3, X0.shape)
    vel = np.zeros_like(pos)
    vel[:, 1] = -0.8
    pinned = np.zeros(nx * ny, np.uint8)
    pinned[[0, nx - 1, 5 * nx + 7]] = 1
    return make_scene(nx, ny, origin=(0.05, 0.01, 0.05), du=(0.02, 0, 0), dv=(0, 0, 0.045), ks=(300.0, 150.0, 60.0),
                      kd=(0.3, 0.2, 0.1), gravity=(0, -9.81, 0), dt=1 / 1200, substeps=4, pos=pos, vel=vel,
                      pinned=pinned, mesh=floor_mesh(), wind=w, name="ragged")


SCENES["ragged_45x19_floor"] = _ragged_scene


@pytest.mark.parametrize("name", sorted(SCENES))
def test_parity_one_and_hundred_steps(cloth_lib, oracle_lib, name):
    sc = SCENES[name]()
    p1, v1 = run_gpu(cloth_lib, sc, 1)
    x1, _ = run_oracle(oracle_lib, sc, 1)
    e1 = max_err(p1, x1)
    assert e1 <= TOL_1
    p, v = run_gpu(cloth_lib, sc, 100)
    x, vo = run_oracle(oracle_lib, sc, 100)
    err = max_err(p, x)
    print(f"{name}: max position error {e1:.2e} m after 1 step, {err:.2e} m after 100 steps")
    assert np.all(np.isfinite(p)) and np.all(np.isfinite(v))
    assert err <= TOL_100, f"{name}: max position error {err:.3e} m after 100 steps"


def _oracle_states(oracle_lib, sc, steps_list):
    """Oracle (FP64) states of a scene at the given steps, as float32."""
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    x, v = sc.init_pos, sc.init_vel
    done = 0
    out = {}
    for s in sorted(steps_list):
        x, v = oracle_lib.step(cl, x, v, done * sc.substeps, (s - done) * sc.substeps, grid)
        done = s
        out[s] = (x.astype(np.float32), v.astype(np.float32))
    return out


def _substep_scene(sc):
    """The scene stepped one substep per step: dt is the float32 substep the
    library derives from the scene (float32(dt / substeps)), so a GPU step of
    this scene is exactly one substep of the original."""
    dts = float(np.float32(float(np.float32(sc.dt)) / sc.substeps))
    return dataclasses.replace(sc, dt=dts, substeps=1)


def _explained_by_rounding(oracle_lib, clo, grid, x0, v0, i, target, tol):
    """Whether a float32-sized change of node i's start state makes the FP64
    oracle's substep put node i within tol of `target`: the start position
    moved by 1 or 4 float32 ulps of 1 m (1.19e-7 m) along an axis, or the
    start velocity by the same amounts in m/s."""
    for which in (0, 1):
        for ax in range(3):
            for d in (1.19e-7, -1.19e-7, 4.77e-7, -4.77e-7):
                x = np.array(x0, np.float64)
                v = np.array(v0, np.float64)
                (x if which == 0 else v)[i, ax] += d
                xo, _ = oracle_lib.step(clo, x, v, 0, 1, grid)
                if np.max(np.abs(xo[i] - target)) <= tol:
                    return True
    return False


@pytest.mark.parametrize("scene", ["config1", "contact_l4"])
def test_contact_replay_substeps(cloth_lib, oracle_lib, scene):
    # Through sustained contact the trajectory is chaotic (a 3e-8 m change of
    # the FP64 oracle's input grows to ~4e-3 m in 100 steps), so contact is
    # checked substep by substep: both sides start from the same float32
    # state (the FP64 oracle's trajectory rounded to float32) and take one
    # substep.  Every node must land within 1e-5 m of the oracle, except a
    # node whose hit/miss decision lies within float32 rounding of an MT
    # threshold: for such a node the test shows that the FP64 oracle takes the
    # GPU's branch, landing within 1e-5 m of the GPU result, once the node's
    # start position or velocity moves by at most 4 float32 ulps of 1 m
    # (4.8e-7).  No node is accepted on a distance bound alone.
    sc = SCENES[scene]()
    sub = _substep_scene(sc)
    steps = [120, 140, 160, 180, 200, 240] if scene == "config1" else [5, 20, 40, 60, 80]
    states = _oracle_states(oracle_lib, sc, steps)
    clo = oracle_lib.Cloth(sc)
    clo1 = oracle_lib.Cloth(sub)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    contacts = flips = replays = 0
    with cloth_lib.Cloth(sub) as cl:
        for s in steps:
            x, v = (a.astype(np.float64) for a in states[s])
            for j in range(sc.substeps):
                x0, v0 = x.astype(np.float32), v.astype(np.float32)
                cl.set_state(x0, v0)
                cl.step(1)
                p, _ = cl.read()
                xo, _, hits = oracle_lib.step(clo1, x0, v0, 0, 1, grid, want_hits=True)
                contacts += int((hits > 0).sum())
                replays += 1
                err = np.abs(p.astype(np.float64) - xo).max(axis=1)
                for i in np.nonzero(err > TOL_1)[0]:
                    assert _explained_by_rounding(oracle_lib, clo1, grid, x0, v0, i, p[i].astype(np.float64),
                                                  TOL_1), (s, j, int(i), float(err[i]))
                    flips += 1
                x, v = oracle_lib.step(clo, x, v, s * sc.substeps + j, 1, grid)
    print(f"{scene}: {replays} substep replays, {contacts} node contacts, {flips} branch flips explained")
    assert contacts > 20


def test_full_size_config2(cloth_lib, oracle_lib):
    sc = cs.config2()
    p, _ = run_gpu(cloth_lib, sc, 1)
    x, _ = run_oracle(oracle_lib, sc, 1)
    e1 = max_err(p, x)
    assert e1 <= TOL_1
    p, _ = run_gpu(cloth_lib, sc, 100)
    x, _ = run_oracle(oracle_lib, sc, 100)
    e100 = max_err(p, x)
    print(f"config2: max position error {e1:.2e} m after 1 step, {e100:.2e} m after 100 steps")
    assert e100 <= TOL_100


def test_full_size_config3_metric_workload(cloth_lib, oracle_lib):
    # 800x800 cloth, 81,920-triangle mesh, wind: the benchmarked workload
    sc = cs.config3("l6")
    p, _ = run_gpu(cloth_lib, sc, 1)
    x, _ = run_oracle(oracle_lib, sc, 1)
    e1 = max_err(p, x)
    assert e1 <= TOL_1
    p, v = run_gpu(cloth_lib, sc, 100)
    x, _ = run_oracle(oracle_lib, sc, 100)
    e100 = max_err(p, x)
    print(f"config3 (L6): max position error {e1:.2e} m after 1 step, {e100:.2e} m after 100 steps")
    assert e100 <= TOL_100
    pin = sc.pinned.astype(bool)
    assert np.array_equal(p[pin], sc.init_pos[pin])


def test_pinned_nodes_bitwise_unchanged(cloth_lib):
    sc = cs.config1()
    p, v = run_gpu(cloth_lib, sc, 50)
    pin = sc.pinned.astype(bool)
    assert np.array_equal(p[pin], sc.init_pos[pin])
    assert np.all(v[pin] == 0)


def test_deterministic_and_graph_equals_plain_launches(cloth_lib):
    sc = cs.small_collision_scene(n=40, level=3, gap=0.002)
    a = run_gpu(cloth_lib, sc, 30)
    b = run_gpu(cloth_lib, sc, 30)
    c = run_gpu(cloth_lib, sc, 30, flags=cloth_lib.capi.CLOTH_FLAG_NO_GRAPH)
    for x, y in ((a, b), (a, c)):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])


def test_step_in_pieces_equals_one_call(cloth_lib):
    sc = cs.config3("l5", n=64)
    a = run_gpu(cloth_lib, sc, 12)
    with cloth_lib.Cloth(sc) as cl:
        for n in (1, 5, 0, 6):
            cl.step(n)
        b = cl.read()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("mesh", ["l2", "l5", "l6d", "floor"])
def test_grid_bit_exact_vs_oracle(cloth_lib, oracle_lib, mesh):
    mv, mt = {"l2": lambda: cs.sphere_mesh(2, 0.3, (0, -0.5, 0)),
              "l5": lambda: cs.sphere_mesh(5, 0.25, (0, -0.6, 0.3)),
              "l6d": lambda: (cs.config3("l6", n=8).mesh_verts, cs.config3("l6", n=8).mesh_tris),
              "floor": floor_mesh}[mesh]()
    sc = make_scene(4, 4, mesh=(mv, mt))
    g = oracle_lib.Grid(mv, mt)
    with cloth_lib.Cloth(sc) as cl:
        info = cl.info()
        gp = g.params
        assert info.grid_h == gp["h"] and info.grid_inv == gp["inv"]
        assert tuple(info.grid_origin) == gp["origin"] and tuple(info.grid_dims) == gp["dims"]
        cs_gpu, ids_gpu = cl.grid()
        assert np.array_equal(cs_gpu, g.cell_start())
        assert np.array_equal(ids_gpu, g.tri_ids())
        # candidate sets of random segments (plus degenerate ones) on identical float32 inputs
        rng = np.random.default_rng(3)
        V = mv.astype(np.float64)
        lo, hi = V.min(0) - 0.1, V.max(0) + 0.1
        S = rng.uniform(lo, hi, (3000, 3)).astype(np.float32)
        E = (S + rng.normal(0, 0.02, (3000, 3))).astype(np.float32)
        E[:50] = S[:50]                                   # zero-length
        S[50:60] = E[50:60] = np.float32(1e30)            # far outside (clamped to the empty border)
        S[60:70] = E[60:70] = np.float32(-1e30)
        counts, ids = cl.query_candidates(S, E)
        for i in range(len(S)):
            ref = g.candidates_f32(S[i], E[i])
            got = np.sort(ids[i, :counts[i]])
            assert np.array_equal(got, ref), i
        assert np.all(counts[50:70] == 0)
        # a few long segments that leave the grid (large candidate sets)
        S2 = rng.uniform(lo, hi, (4, 3)).astype(np.float32)
        E2 = (S2 + np.float32(5.0)).astype(np.float32)
        counts, ids = cl.query_candidates(S2, E2)
        for i in range(len(S2)):
            assert np.array_equal(np.sort(ids[i, :counts[i]]), g.candidates_f32(S2[i], E2[i]))


def test_candidates_of_the_gpu_trajectory_bit_exact(cloth_lib, oracle_lib):
    # replay one substep's (x, x*) segments of the GPU state through both grids
    sc = cs.config1()
    with cloth_lib.Cloth(sc) as cl:
        cl.step(140)
        pos, vel = cl.read()
        E = (pos + np.float32(sc.dt / sc.substeps) * vel).astype(np.float32)
        counts, ids = cl.query_candidates(pos, E)
    g = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    nonempty = 0
    for i in range(len(pos)):
        ref = g.candidates_f32(pos[i], E[i])
        nonempty += len(ref) > 0
        assert np.array_equal(np.sort(ids[i, :counts[i]]), ref)
    assert nonempty > 50


def test_set_state_read_roundtrip_and_nonfinite_flag(cloth_lib):
    sc = cs.config3("none", n=33)
    with cloth_lib.Cloth(sc) as cl:
        rng = np.random.default_rng(0)
        p = rng.normal(size=(sc.n, 3)).astype(np.float32)
        v = rng.normal(size=(sc.n, 3)).astype(np.float32)
        cl.set_state(p, v)
        a, b = cl.read()
        assert np.array_equal(a, p) and np.array_equal(b, v)
        cl.step(3)
        cl.set_state(p, None)
        a, b = cl.read()
        assert np.array_equal(a, p)
        bad = p.copy()
        bad[7, 1] = np.nan
        cl.set_state(bad, v)
        cl.step(1)
        with pytest.raises(cloth_lib.ClothError) as ei:
            cl.read()
        assert ei.value.code == cloth_lib.capi.CLOTH_ERR_NONFINITE
        cl.set_state(p, v)  # clears the flag
        cl.step(1)
        cl.read()
        # a non-finite velocity alone: the walk checks the positions it
        # stores, and x = x0 + dt v carries it (node 500 is not pinned)
        assert not sc.pinned[500]
        badv = v.copy()
        badv[500, 2] = np.inf
        cl.set_state(p, badv)
        cl.step(1)
        with pytest.raises(cloth_lib.ClothError) as ei:
            cl.read()
        assert ei.value.code == cloth_lib.capi.CLOTH_ERR_NONFINITE
        cl.set_state(p, v)
        cl.step(1)
        cl.read()


def test_bad_mesh_is_rejected_and_previous_mesh_kept(cloth_lib):
    sc = cs.small_collision_scene(n=16, level=1, gap=0.002)
    with cloth_lib.Cloth(sc) as cl:
        ntris = cl.info().ntris
        bad = sc.mesh_tris.copy()
        bad[3, 1] = len(sc.mesh_verts)
        with pytest.raises(cloth_lib.ClothError) as ei:
            cl.set_mesh(sc.mesh_verts, bad)
        assert ei.value.code == cloth_lib.capi.CLOTH_ERR_BAD_MESH
        assert cl.info().ntris == ntris
        cl.set_mesh(None, None)  # clear
        assert cl.info().ntris == 0
        cl.step(2)
        cl.read()


def test_empty_and_minimal_cloths(cloth_lib, oracle_lib):
    for nx, ny in [(1, 1), (1, 2), (2, 1), (3, 1), (1, 5)]:
        sc = make_scene(nx, ny, ks=(50.0, 20.0, 10.0), kd=(0.1, 0.1, 0.1), gravity=(0, -9.81, 0), dt=1e-3,
                        substeps=2, mesh=floor_mesh(), origin=(0.3, 0.01, 0.3), du=(0.05, 0, 0), dv=(0, 0, 0.05))
        p, v = run_gpu(cloth_lib, sc, 40)
        x, vo = run_oracle(oracle_lib, sc, 40)
        assert max_err(p, x) <= TOL_100


def test_penetration_bounded_gpu_config1(cloth_lib):
    # The FP64 oracle keeps every node of config 1 outside the sphere (CPU
    # test).  In float32 a node that ends a substep within ~1e-8 m of the
    # surface can miss the crossing in the next one (the hit distance carries
    # that rounding), and the two-sided test then keeps it inside.  Bound: at
    # most 1% of the nodes inside at any checked step, none deeper than 1 cm
    # (a tenth of an L2 triangle edge) below the nearest face plane of the
    # (convex) icosphere.
    sc = cs.config1()
    V = sc.mesh_verts.astype(np.float64)
    T = sc.mesh_tris
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    off = np.einsum("ij,ij->i", n, V[T[:, 0]])
    with cloth_lib.Cloth(sc) as cl:
        for _ in range(12):
            cl.step(25)
            p, _ = cl.read()
            inside = ray_parity_inside(p, sc.mesh_verts, sc.mesh_tris)
            assert inside.mean() <= 0.01
            if inside.any():
                depth = -np.max(p[inside].astype(np.float64) @ n.T - off[None, :], axis=1)
                assert np.all(depth <= 1e-2), depth


@pytest.mark.parametrize("mode", ["atomic", "edges"])
def test_minimal_cloths_in_the_alternative_paths(cloth_lib, oracle_lib, mode):
    # ragged and degenerate grids through the atomic spring path and the edge
    # narrow phase: the same tolerances as the default path (edge mode against
    # the oracle's edge reading)
    flag = {"atomic": cloth_lib.capi.CLOTH_FLAG_ATOMIC_SPRINGS, "edges": cloth_lib.capi.CLOTH_FLAG_EDGE_COLLISION}[mode]
    for nx, ny in [(1, 1), (1, 2), (2, 1), (3, 1), (1, 5), (2, 2), (5, 3), (61, 2)]:
        sc = make_scene(nx, ny, ks=(50.0, 20.0, 10.0), kd=(0.1, 0.1, 0.1), gravity=(0, -9.81, 0), dt=1e-3,
                        substeps=2, mesh=floor_mesh(), origin=(0.3, 0.012, 0.3), du=(0.007, 0, 0),
                        dv=(0, 0.004, 0.005))
        p, v = run_gpu(cloth_lib, sc, 1, flags=flag)
        if mode == "edges":
            cl = oracle_lib.Cloth(sc)
            x, _ = oracle_lib.step_edges(cl, sc.init_pos, sc.init_vel, 0, sc.substeps,
                                         oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris))
        else:
            x, _ = run_oracle(oracle_lib, sc, 1)
        assert np.all(np.isfinite(p)) and max_err(p, x) <= TOL_1, (nx, ny)
