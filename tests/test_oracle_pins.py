"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each checks a closed form, an
invariant, a constructed ground truth, a hand-derived fixture
(tests/golden/) or brute force on tiny inputs, chosen so that a dropped term,
a wrong sign or index, or a transposed operand in the oracle fails one of
them.
"""
import math
import os

import numpy as np
import pytest

import cloth_scenes as cs
from helpers import (GOLDEN, floor_mesh, make_scene, pair_type, ray_parity_inside, spring_energy,
                     stencil_pairs)


# ------------------------------------------------------------ spring layout

@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 2), (2, 1), (3, 3), (4, 7), (6, 5)])
def test_spring_enumeration_matches_brute_force_pairs(oracle_lib, nx, ny):
    a, b, t = oracle_lib.springs(nx, ny)
    got = {(min(i, j), max(i, j)) for i, j in zip(a.tolist(), b.tolist())}
    assert len(got) == len(a), "duplicate spring"
    assert got == stencil_pairs(nx, ny)
    assert len(a) == cs.spring_count(nx, ny)
    for i, j, ty in zip(a.tolist(), b.tolist(), t.tolist()):
        assert ty == pair_type(nx, i, j)
    # canonical order: node1 row-major ascending
    assert np.all(np.diff(a) >= 0)


def test_spring_counts_of_the_workloads():
    # structural 2n(n-1), shear 2(n-1)^2, bend 2n(n-2)
    for n, S in [(32, 5826), (128, 97026), (256, 390658), (800, 3832002)]:
        assert cs.spring_count(n, n) == S == 2 * n * (n - 1) + 2 * (n - 1) ** 2 + 2 * n * (n - 2)


# ------------------------------------------------------------ force law (Alg. 1)

def test_zero_force_at_rest_length(oracle_lib):
    # dyadic spacing: every rest length and current length is computed from
    # identical exact differences, so Hooke's term is exactly zero; a uniform
    # velocity makes every damping term exactly zero too.
    sc = make_scene(9, 7, du=(0.125, 0.0, 0.0), dv=(0.0, 0.0, 0.125), ks=(500, 250, 100), kd=(0.5, 0.3, 0.2))
    cl = oracle_lib.Cloth(sc)
    x = sc.init_pos.astype(np.float64)
    v = np.tile([0.5, -1.25, 2.0], (sc.n, 1))
    F = oracle_lib.spring_forces(cl, x, v)
    assert np.all(F == 0.0)


def test_momentum_internal_forces_sum_to_zero(oracle_lib):
    rng = np.random.default_rng(11)
    sc = make_scene(12, 9, ks=(500, 250, 100), kd=(0.5, 0.3, 0.2))
    cl = oracle_lib.Cloth(sc)
    x = sc.init_pos + rng.normal(0, 0.02, (sc.n, 3))
    v = rng.normal(0, 1.0, (sc.n, 3))
    F = oracle_lib.spring_forces(cl, x, v)
    tot = np.abs(F).sum()
    assert tot > 1.0
    assert np.all(np.abs(F.sum(axis=0)) <= 1e-12 * tot)
    # angular momentum: central forces exert no net torque
    tau = np.cross(x, F).sum(axis=0)
    assert np.all(np.abs(tau) <= 1e-12 * (np.abs(np.cross(x, F)).sum()))


def test_spring_force_is_minus_energy_gradient(oracle_lib):
    # kd = 0: F_i = -dE/dx_i for E = sum 1/2 k (l - L0)^2 over the brute-force
    # pair list (central finite differences).
    rng = np.random.default_rng(3)
    nx, ny = 5, 4
    ks = (500.0, 250.0, 100.0)
    sc = make_scene(nx, ny, ks=ks)
    X0 = cs.flat_grid(nx, ny, sc.origin, sc.du, sc.dv)
    x = X0 + rng.normal(0, 0.01, X0.shape)
    cl = oracle_lib.Cloth(sc)
    F = oracle_lib.spring_forces(cl, x, np.zeros_like(x))
    kof = lambda i, j: ks[pair_type(nx, i, j)]
    h = 1e-6
    for i in range(sc.n):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            g = (spring_energy(nx, ny, X0, xp, kof) - spring_energy(nx, ny, X0, xm, kof)) / (2 * h)
            assert abs(F[i, k] + g) <= 1e-6 * max(1.0, abs(g)), (i, k, F[i, k], -g)


def test_damping_is_dissipative(oracle_lib):
    # ks = 0: the power of the damping forces, sum F_i . v_i, is never positive
    rng = np.random.default_rng(5)
    sc = make_scene(7, 6, kd=(0.5, 0.3, 0.2))
    cl = oracle_lib.Cloth(sc)
    for _ in range(5):
        x = sc.init_pos + rng.normal(0, 0.02, (sc.n, 3))
        v = rng.normal(0, 1.0, (sc.n, 3))
        F = oracle_lib.spring_forces(cl, x, v)
        assert np.sum(F * v) < 0.0


def test_two_node_damping_closed_form(oracle_lib):
    # Two nodes on one structural spring, ks = 0, velocities along the spring:
    # symplectic Euler gives dv_n = (1 - 2 kd dt / m)^n dv_0 exactly.
    kd, m, dt, u = 0.3, 0.05, 1e-3, 0.75  # u exact in float32
    sc = make_scene(2, 1, du=(0.1, 0.0, 0.0), total_mass=2 * m, kd=(kd, 0, 0), dt=dt,
                    vel=[[-u, 0, 0], [u, 0, 0]])
    cl = oracle_lib.Cloth(sc)
    n = 37
    x, v = oracle_lib.step(cl, sc.init_pos, sc.init_vel, 0, n)
    dv = v[1, 0] - v[0, 0]
    assert dv == pytest.approx(2 * u * (1 - 2 * kd * dt / m) ** n, rel=1e-12)
    assert np.all(v[:, 1:] == 0)
    # momentum conserved
    assert abs(v[0, 0] + v[1, 0]) < 1e-15


# ------------------------------------------------------------ integrator

def test_free_fall_discrete_closed_form(oracle_lib):
    # No springs: symplectic Euler gives v_n = v0 + n dt g and
    # x_n = x0 + n dt v0 + dt^2 g n(n+1)/2 (explicit Euler would give n(n-1)/2).
    g = np.array([0.3, -9.81, 0.2])
    v0 = np.array([1.0, 2.0, -0.5])
    x0 = np.array([0.1, 0.2, 0.3])
    dt = 1.0 / 4800
    sc = make_scene(1, 1, origin=x0, gravity=g, dt=dt, vel=[v0])
    cl = oracle_lib.Cloth(sc)
    n = 250
    x, v = oracle_lib.step(cl, sc.init_pos, sc.init_vel, 0, n)
    x0f = sc.init_pos[0].astype(np.float64)
    v0f = sc.init_vel[0].astype(np.float64)
    np.testing.assert_allclose(v[0], v0f + n * dt * g, rtol=0, atol=1e-12)
    np.testing.assert_allclose(x[0], x0f + n * dt * v0f + dt * dt * g * n * (n + 1) / 2, rtol=0, atol=1e-12)


def test_hanging_spring_static_extension(oracle_lib):
    # One pinned node, one free node of mass m below it on a damped spring:
    # converges to l = L0 + m g / k.
    m, k, kd, L0 = 0.05, 50.0, 1.0, 0.1
    sc = make_scene(1, 2, dv=(0.0, -L0, 0.0), total_mass=2 * m, ks=(k, 0, 0), kd=(kd, 0, 0),
                    gravity=(0, -9.81, 0), dt=1e-3, pinned=[1, 0])
    cl = oracle_lib.Cloth(sc)
    x, v = oracle_lib.step(cl, sc.init_pos, sc.init_vel, 0, 6000)
    ell = np.linalg.norm(x[1] - x[0])
    assert ell == pytest.approx(L0 + m * 9.81 / k, rel=1e-9)
    assert np.all(x[0] == sc.init_pos[0].astype(np.float64))


def _energy(oracle_lib, sc, x, v):
    m = sc.total_mass / sc.n
    X0 = cs.flat_grid(sc.nx, sc.ny, sc.origin, sc.du, sc.dv)
    kof = lambda i, j: sc.ks[pair_type(sc.nx, i, j)]
    return 0.5 * m * np.sum(v * v) + spring_energy(sc.nx, sc.ny, X0, x, kof)


def test_energy_drift_first_order(oracle_lib):
    # kd = 0, no gravity or pins, jittered start: symplectic Euler keeps the
    # energy error bounded and first order in dt (halves when dt halves).
    nx = ny = 6
    base = make_scene(nx, ny, du=(0.1, 0, 0), dv=(0, 0, 0.1), total_mass=0.36, ks=(40.0, 20.0, 8.0))
    rng = np.random.default_rng(9)
    x0 = base.init_pos + rng.uniform(-0.01, 0.01, base.init_pos.shape).astype(np.float32)
    drifts = []
    T = 0.1
    for dt in (2e-4, 1e-4, 5e-5):
        sc = make_scene(nx, ny, du=(0.1, 0, 0), dv=(0, 0, 0.1), total_mass=0.36, ks=(40.0, 20.0, 8.0),
                        dt=dt, pos=x0)
        cl = oracle_lib.Cloth(sc)
        x, v = x0.astype(np.float64), np.zeros_like(x0, dtype=np.float64)
        E0 = _energy(oracle_lib, sc, x, v)
        n = int(round(T / dt))
        chunk = n // 20
        worst = 0.0
        for s in range(20):
            x, v = oracle_lib.step(cl, x, v, s * chunk, chunk)
            worst = max(worst, abs(_energy(oracle_lib, sc, x, v) - E0) / E0)
        drifts.append(worst)
    assert drifts[0] < 0.2
    r1, r2 = drifts[0] / drifts[1], drifts[1] / drifts[2]
    assert 1.6 < r1 < 2.5 and 1.6 < r2 < 2.5, drifts


def test_pinned_nodes_hold_position_and_zero_velocity(oracle_lib):
    sc = cs.config1()
    cl = oracle_lib.Cloth(sc)
    x, v = oracle_lib.step(cl, sc.init_pos, sc.init_vel + 0.1, 0, 40)
    pin = sc.pinned.astype(bool)
    assert np.all(x[pin] == sc.init_pos[pin].astype(np.float64))
    assert np.all(v[pin] == 0.0)
    assert np.all(x[~pin] != sc.init_pos[~pin].astype(np.float64))


def test_wind_matches_integrated_sinusoid(oracle_lib):
    # One free node under wind only: the discrete velocity is a left Riemann
    # sum of w(t), within T*max|w'|*dt/2 of the exact integral
    # -A/(2 pi f) [cos(2 pi f T + c) - cos(c)], c = kappa (udir . X0) + phase.
    w = cs.wind_config3()
    X0 = np.array([0.3, -0.7, 0.1])
    dt = 1.0 / 4800
    n = 2400
    sc = make_scene(1, 1, origin=X0, dt=dt, wind=w)
    cl = oracle_lib.Cloth(sc)
    x, v = oracle_lib.step(cl, sc.init_pos, sc.init_vel, 0, n)
    c = w.kappa * float(np.dot(w.udir, X0)) + w.phase
    T = n * dt
    om = 2 * math.pi * w.freq
    exact = -w.amp / om * (math.cos(om * T + c) - math.cos(c))
    bound = T * w.amp * om * dt / 2
    assert abs(v[0, 2] - exact) <= bound
    assert abs(exact) > 50 * bound
    assert v[0, 0] == 0.0 and v[0, 1] == 0.0
    # the node at a different rest position sees a different phase
    sc2 = make_scene(1, 1, origin=X0 + np.array([0.125, 0.0, 0.0]), dt=dt, wind=w)
    x2, v2 = oracle_lib.step(oracle_lib.Cloth(sc2), sc2.init_pos, sc2.init_vel, 0, n)
    c2 = c + w.kappa * w.udir[0] * 0.125
    exact2 = -w.amp / om * (math.cos(om * T + c2) - math.cos(c2))
    assert abs(v2[0, 2] - exact2) <= bound


# ------------------------------------------------------------ MT test

def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                p = line.split()
                rows.append((p[0], [float(z) for z in p[1:]]))
    return rows


@pytest.mark.parametrize("name,vals", _golden("mt_cases.txt"))
def test_mt_golden_cases(oracle_lib, name, vals):
    S, E = vals[0:3], vals[3:6]
    hit, t = int(vals[6]), vals[7]
    V0, V1, V2 = [0, 0, 0], [1, 0, 0], [0, 1, 0]
    got = oracle_lib.mt(S, E, V0, V1, V2, 1e-7)
    if hit:
        assert got is not None and got == pytest.approx(t, rel=1e-15, abs=1e-15)
    else:
        assert got is None


def test_mt_constructed_hits_and_misses(oracle_lib):
    # Ground truth by construction: P = V0 + u e1 + v e2 inside the triangle,
    # S = P - t0 r; the segment S -> S + L r hits at t0 iff L > t0.
    rng = np.random.default_rng(21)
    nhit = nmiss = 0
    for _ in range(3000):
        V = rng.normal(0, 1, (3, 3))
        e1, e2 = V[1] - V[0], V[2] - V[0]
        n = np.cross(e1, e2)
        if np.linalg.norm(n) < 0.1:
            continue
        r = rng.normal(0, 1, 3)
        r /= np.linalg.norm(r)
        if abs(np.dot(r, n)) / np.linalg.norm(n) < 0.2:
            continue
        u, v = rng.uniform(0, 1, 2)
        t0 = rng.uniform(0.01, 1.0)
        inside = rng.uniform() < 0.5
        if inside:
            if u + v > 1:
                u, v = 1 - u, 1 - v
            u, v = 0.02 + 0.96 * u, 0.02 + 0.96 * v
            if u + v > 0.98:
                continue
        else:
            # clearly outside: one barycentric coordinate negative or sum > 1
            choice = rng.integers(3)
            if choice == 0:
                u = -0.05 - u
            elif choice == 1:
                v = -0.05 - v
            else:
                u, v = u + 0.6, v + 0.6
        P = V[0] + u * e1 + v * e2
        S = P - t0 * r
        long_ = rng.uniform() < 0.5
        L = t0 * (1.05 + rng.uniform()) if long_ else t0 * rng.uniform(0.1, 0.95)
        E = S + L * r
        got = oracle_lib.mt(S, E, V[0], V[1], V[2], 1e-7)
        if inside and long_:
            assert got is not None and got == pytest.approx(t0, rel=1e-9, abs=1e-12)
            nhit += 1
        else:
            assert got is None
            nmiss += 1
    assert nhit > 300 and nmiss > 1000


def _det3(a, b, c):
    return (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
            + a[2] * (b[0] * c[1] - b[1] * c[0]))


def test_mt_matches_exact_rational_segment_triangle_intersection(oracle_lib):
    # Ground truth in exact rational arithmetic from the definition: solve
    # S + s d = V0 + u e1 + v e2 (d = E - S) by Cramer's rule and apply the
    # test's conditions (reading C6): |a| >= eps with a = r . (e2 x e1),
    # r = d/|d|, i.e. (d . (e1 x e2))^2 >= eps^2 |d|^2; u in [0, 1], v >= 0,
    # u + v <= 1; t = s |d| in (eps, |d|).  Squares keep |d| out of it, so
    # everything stays rational.  Pairs within 1e-9 of a threshold are
    # skipped (away from ties, where double rounding may decide either way).
    from fractions import Fraction as Fr
    rng = np.random.default_rng(23)
    eps = 1e-7
    fe = Fr(eps)
    nhit = nmiss = nskip = 0
    reasons = set()
    for it in range(10000):
        V = rng.normal(0, 1, (3, 3))
        e1, e2 = V[1] - V[0], V[2] - V[0]
        u0, v0 = rng.uniform(-0.3, 1.3, 2)
        P = V[0] + u0 * e1 + v0 * e2
        kind = it % 4
        r = rng.normal(0, 1, 3)
        if kind == 1:  # nearly parallel to the triangle's plane
            n = np.cross(e1, e2)
            n /= np.linalg.norm(n)
            r = r - np.dot(r, n) * n + rng.choice([1e-12, 1e-9, 1e-6, 1e-3]) * n
        r /= np.linalg.norm(r)
        t0 = rng.uniform(-0.5, 1.5) if kind != 2 else rng.choice([1e-9, 5e-8, 2e-7, 1e-6])
        L = rng.uniform(0.05, 2.0)
        S = P - t0 * r
        E = S + L * r
        # exact decision
        FS, FE = [Fr(float(x)) for x in S], [Fr(float(x)) for x in E]
        FV = [[Fr(float(x)) for x in row] for row in V]
        d = [FE[k] - FS[k] for k in range(3)]
        f1 = [FV[1][k] - FV[0][k] for k in range(3)]
        f2 = [FV[2][k] - FV[0][k] for k in range(3)]
        b = [FV[0][k] - FS[k] for k in range(3)]
        m1 = [-x for x in f1]
        m2 = [-x for x in f2]
        L2 = sum(x * x for x in d)
        det = _det3(d, m1, m2)
        margins = []
        if det == 0:
            exact_hit, why = False, "parallel"
        else:
            par = det * det - fe * fe * L2  # |a| >= eps  <=>  par >= 0
            sc = _det3(b, m1, m2) / det
            u = _det3(d, b, m2) / det
            v = _det3(d, m1, b) / det
            tl = sc * sc * L2 - fe * fe  # t > eps  <=>  s > 0 and tl > 0
            margins = [float(par) / max(float(fe * fe * L2), 1e-300), float(u), float(1 - u), float(v),
                       float(1 - u - v), float(sc - 1), float(sc)]
            if float(L2) > 0:
                margins.append(float(tl) / float(fe * fe))
            if par < 0:
                exact_hit, why = False, "parallel"
            elif not (0 <= u <= 1 and v >= 0 and u + v <= 1):
                exact_hit, why = False, "outside"
            elif not (sc > 0 and tl > 0):
                exact_hit, why = False, "behind or within eps"
            elif not sc < 1:
                exact_hit, why = False, "beyond the end"
            else:
                exact_hit, why = True, "hit"
        if any(abs(m) < 1e-9 for m in margins):
            nskip += 1
            continue
        got = oracle_lib.mt(S, E, V[0], V[1], V[2], eps)
        assert (got is not None) == exact_hit, (it, why, got)
        reasons.add(why)
        if exact_hit:
            t_exact = float(sc) * float(np.sqrt(float(L2)))
            assert got == pytest.approx(t_exact, rel=1e-8, abs=1e-12)
            nhit += 1
        else:
            nmiss += 1
    assert nhit > 500 and nmiss > 5000 and nskip < 500, (nhit, nmiss, nskip)
    assert reasons == {"hit", "parallel", "outside", "behind or within eps", "beyond the end"}


# ------------------------------------------------------------ response (Alg. 2)

@pytest.mark.parametrize("name,vals", _golden("response_cases.txt"))
def test_response_golden_cases(oracle_lib, name, vals):
    S, V, K = vals[0:3], vals[3:6], int(vals[6])
    X, W = vals[7:10], vals[10:13]
    sc = make_scene(1, 1, origin=S, dt=2.0 ** -10, vel=[V], mesh=floor_mesh(), delta=1e-4)
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(*floor_mesh())
    for brute in (False, True):
        x, v, hits = oracle_lib.step(cl, sc.init_pos, sc.init_vel, 0, 1, grid, brute=brute, want_hits=True)
        assert hits[0] == K
        np.testing.assert_allclose(x[0], X, rtol=0, atol=1e-15)
        np.testing.assert_allclose(v[0], W, rtol=0, atol=0)


@pytest.mark.parametrize("y0", [0.05, 0.0507])
def test_falling_node_lands_on_plane_closed_form(oracle_lib, y0):
    # Gravity only, node released at height y0 above the floor: free fall in
    # closed form until the substep whose segment crosses y = 0, where the
    # node stops delta before the crossing (or stays put when it started
    # closer than delta) and its velocity flips by -0.5.
    g, dt, delta = -9.81, 1.0 / 4800, 1e-4
    sc = make_scene(1, 1, origin=(0.3, y0, 0.6), gravity=(0, g, 0), dt=dt, mesh=floor_mesh(), delta=delta)
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(*floor_mesh())
    y0f = float(sc.init_pos[0, 1])
    ypos = lambda n: y0f + dt * dt * g * n * (n + 1) / 2
    n_hit = next(n for n in range(1, 100000) if ypos(n) < 0)
    x, v = oracle_lib.step(cl, sc.init_pos, sc.init_vel, 0, n_hit - 1, grid)
    assert x[0, 1] == pytest.approx(ypos(n_hit - 1), abs=1e-12)
    x, v, hits = oracle_lib.step(cl, x, v, n_hit - 1, 1, grid, want_hits=True)
    assert hits[0] == 1
    assert x[0, 1] == pytest.approx(min(ypos(n_hit - 1), delta), abs=1e-12)
    assert v[0, 1] == pytest.approx(-0.5 * dt * g * n_hit, rel=1e-12)
    assert x[0, 0] == float(sc.init_pos[0, 0]) and x[0, 2] == float(sc.init_pos[0, 2])


# ------------------------------------------------------------ broad phase

def _tiny_meshes():
    yield cs.sphere_mesh(0, 0.3)
    yield cs.sphere_mesh(1, 0.25, (0.1, -0.05, 0.02))
    yield cs.sphere_mesh(2, 0.3, (0.0, -0.5, 0.0), 0.05, 4)
    yield floor_mesh()


@pytest.mark.parametrize("mi", range(4))
def test_grid_lists_exactly_the_overlapped_cells(oracle_lib, mi):
    verts, tris = list(_tiny_meshes())[mi]
    g = oracle_lib.Grid(verts, tris)
    p = g.params
    h, o, dims = float(p["h"]), np.array(p["origin"], np.float64), p["dims"]
    cs_, ids = g.cell_start(), g.tri_ids()
    assert cs_[0] == 0 and cs_[-1] == len(ids) and np.all(np.diff(cs_) >= 0)
    lists = [ids[cs_[c]:cs_[c + 1]] for c in range(len(cs_) - 1)]
    for L in lists:
        assert np.all(np.diff(L) > 0), "ascending, unique"
    # no spurious entries: each listed triangle's AABB touches the cell box
    V = verts.astype(np.float64)
    for c, L in enumerate(lists):
        cx, cy, cz = c % dims[0], (c // dims[0]) % dims[1], c // (dims[0] * dims[1])
        lo = o + h * np.array([cx, cy, cz]) - 1e-6
        hi = lo + h + 2e-6
        for t in L:
            tl, th = V[tris[t]].min(axis=0), V[tris[t]].max(axis=0)
            assert np.all(tl <= hi) and np.all(th >= lo)
    # no missing entries: sample points on each triangle; the (FP64) cell of
    # each point, when the point is not near a cell face, lists the triangle
    rng = np.random.default_rng(mi)
    for t in range(len(tris)):
        A = V[tris[t]]
        for _ in range(20):
            a, b = rng.uniform(0, 1, 2)
            if a + b > 1:
                a, b = 1 - a, 1 - b
            q = A[0] + a * (A[1] - A[0]) + b * (A[2] - A[0])
            f = (q - o) / h
            if np.any(np.abs(f - np.rint(f)) < 1e-4):
                continue
            cc = np.floor(f).astype(int)
            c = (cc[2] * dims[1] + cc[1]) * dims[0] + cc[0]
            assert t in set(lists[c].tolist())
    # the border cells are empty (origin = min - 1.5h, dims = floor(ext/h) + 4)
    for c, L in enumerate(lists):
        cx, cy, cz = c % dims[0], (c // dims[0]) % dims[1], c // (dims[0] * dims[1])
        if min(cx, cy, cz) == 0 or cx == dims[0] - 1 or cy == dims[1] - 1 or cz == dims[2] - 1:
            assert len(L) == 0


@pytest.mark.parametrize("mi", range(4))
def test_candidates_contain_every_brute_force_hit(oracle_lib, mi):
    verts, tris = list(_tiny_meshes())[mi]
    g = oracle_lib.Grid(verts, tris)
    V = verts.astype(np.float64)
    rng = np.random.default_rng(100 + mi)
    lo, hi = V.min(axis=0) - 0.05, V.max(axis=0) + 0.05
    nhits = 0
    for _ in range(1500):
        S = rng.uniform(lo, hi).astype(np.float32)
        E = (S + rng.normal(0, 0.03, 3)).astype(np.float32)
        cand = set(g.candidates_f32(S, E).tolist())
        for t in range(len(tris)):
            if oracle_lib.mt(S, E, *V[tris[t]], 1e-7) is not None:
                nhits += 1
                assert t in cand
    assert nhits > 20


def test_broad_phase_step_equals_all_pairs_step(oracle_lib):
    sc = cs.small_collision_scene(n=32, level=2, gap=0.002)
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    xa, va = xb, vb = sc.init_pos, sc.init_vel
    contacts = 0
    for k in range(150):
        xa, va, ha = oracle_lib.step(cl, xa, va, k, 1, grid, want_hits=True)
        xb, vb, hb = oracle_lib.step(cl, xb, vb, k, 1, grid, brute=True, want_hits=True)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ha, hb)
        contacts += int((ha > 0).sum())
    assert contacts > 30


def test_no_penetration_config1(oracle_lib):
    # The paper's qualitative claim (Section 4.2): the response keeps the cloth
    # out of the surface model.  Ray-parity point-in-mesh at several steps.
    sc = cs.config1()
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    x, v = sc.init_pos.astype(np.float64), sc.init_vel.astype(np.float64)
    contacts = 0
    for blk in range(12):
        x, v, h = oracle_lib.step(cl, x, v, blk * 25 * sc.substeps, 25 * sc.substeps, grid, want_hits=True)
        contacts += int((h > 0).sum())
        inside = ray_parity_inside(x, sc.mesh_verts, sc.mesh_tris)
        assert not inside.any(), np.nonzero(inside)
    assert contacts > 50


def test_hit_distance_lower_bound_reading(oracle_lib):
    # A node 5e-8 m above the floor moving down: the literal bound eps < t
    # (eps = 1e-7) misses the crossing, the default reading 0 < t catches it.
    S, E = [0.25, 5e-8, 0.75], [0.25, -1e-5, 0.75]
    V = floor_mesh()[0].astype(np.float64)
    assert oracle_lib.mt(S, E, V[0], V[2], V[3], 1e-7) is None
    t = oracle_lib.mt(S, E, V[0], V[2], V[3], 1e-7, t_min=0.0)
    assert t == pytest.approx(5e-8, rel=1e-6)


def test_literal_lower_bound_lets_resting_nodes_through(oracle_lib):
    # Why the default reading drops eps from the lower bound: with eps < t a
    # node that ends a substep within eps of the surface crosses it unseen in
    # the next one, and resting nodes do so within 300 steps of config 1.
    import dataclasses
    sc = dataclasses.replace(cs.config1(), mt_t_min=1e-7)
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    x, v = oracle_lib.step(cl, sc.init_pos, sc.init_vel, 0, 300 * sc.substeps, grid)
    assert ray_parity_inside(x, sc.mesh_verts, sc.mesh_tris).sum() > 0


# ------------------------------------------------------------- vertex normals
# Pins of the normal update (Section 3's last step before rendering) against
# geometry with known normals, not against the oracle's own formula.

def test_normals_of_a_flat_grid_are_the_plane_normal(oracle_lib):
    # grid along u, v: the face normals are (dv x du)/|.| oriented, every vertex the same
    nx, ny = 7, 5
    du, dv = np.array([0.1, 0.0, 0.0]), np.array([0.0, -0.1, 0.0])
    X = cs.flat_grid(nx, ny, (0.2, 0.3, -0.1), tuple(du), tuple(dv))
    n = oracle_lib.normals(X, nx, ny)
    expect = np.cross(dv, du) / np.linalg.norm(np.cross(dv, du))
    np.testing.assert_allclose(n, np.broadcast_to(expect, n.shape), atol=1e-12)


def _surface_errors(oracle_lib, surf, sizes):
    errs = []
    for n in sizes:
        X, exact = surf(n)
        got = oracle_lib.normals(X, n, n)
        sgn = np.sign(np.sum(got * exact, axis=1))[:, None]  # orientation is the grid's, not outward
        inner = np.zeros((n, n), bool)
        inner[1:-1, 1:-1] = True
        errs.append(float(np.max(np.linalg.norm(got * sgn - exact, axis=1)[inner.ravel()])))
    return errs


def _cylinder(n, power=1.0):
    u = np.linspace(0.0, 1.0, n)
    th = 0.2 + 1.8 * u ** power                # columns: angle
    z = np.linspace(0.0, 0.5, n)               # rows: height
    T, Z = np.meshgrid(th, z)
    X = np.stack([np.cos(T), np.sin(T), Z], -1).reshape(-1, 3)
    return X, np.stack([np.cos(T), np.sin(T), 0 * T], -1).reshape(-1, 3)


def _sphere(n):
    th = np.linspace(0.4, 1.2, n)              # polar
    ph = np.linspace(0.3, 1.3, n)              # azimuth
    TH, PH = np.meshgrid(th, ph)
    X = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    return X, X.copy()


def test_normals_of_a_uniform_cylinder_are_radial(oracle_lib):
    # uniform sampling in angle and height: the two triangles on either side of
    # a vertex mirror each other, so the area-weighted normal is exactly radial
    assert max(_surface_errors(oracle_lib, _cylinder, (9, 17))) < 1e-12


def test_normals_converge_on_curved_surfaces(oracle_lib):
    # a sphere: second order (error / 4 per halving of the spacing); a cylinder
    # sampled non-uniformly in angle: order 1.5 (error / 2.83)
    e = _surface_errors(oracle_lib, _sphere, (9, 17, 33))
    assert e[0] < 0.01 and e[0] / e[1] > 3.5 and e[1] / e[2] > 3.5, e
    e = _surface_errors(oracle_lib, lambda n: _cylinder(n, 1.5), (9, 17, 33))
    assert e[0] < 0.05 and e[0] / e[1] > 2.6 and e[1] / e[2] > 2.6, e


def test_normals_rotate_with_the_cloth_and_ignore_scale(oracle_lib):
    rng = np.random.default_rng(21)
    nx, ny = 6, 8
    X = rng.normal(0, 1, (nx * ny, 3))
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    n0 = oracle_lib.normals(X, nx, ny)
    np.testing.assert_allclose(oracle_lib.normals(X @ q.T, nx, ny), n0 @ q.T, atol=1e-12)
    np.testing.assert_allclose(oracle_lib.normals(3.7 * X + 1.0, nx, ny), n0, atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(n0, axis=1), 1.0, atol=1e-12)


def test_normals_triangle_list_covers_each_quad_once(oracle_lib):
    nx, ny = 5, 4
    t = oracle_lib.grid_triangles(nx, ny)
    assert t.shape == (2 * (nx - 1) * (ny - 1), 3)
    # every interior vertex belongs to six triangles, corners to one or two
    deg = np.bincount(t.ravel(), minlength=nx * ny).reshape(ny, nx)
    assert np.all(deg[1:-1, 1:-1] == 6)
    assert deg[0, 0] == 2 and deg[-1, -1] == 2 and deg[0, -1] == 1 and deg[-1, 0] == 1


# ------------------------------------------- edge-triangle narrow phase (f1)
# Pins of the oracle's reading of the paper's own narrow phase: cloth
# triangle edges at the updated positions against the surface triangles.

def test_edge_affected_sets_are_the_vertices_of_the_triangles_sharing_the_edge(oracle_lib):
    nx, ny = 5, 4
    tris = oracle_lib.grid_triangles(nx, ny)
    from collections import defaultdict
    by_edge = defaultdict(set)
    for t in tris:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[0], t[2])):
            by_edge[(min(a, b), max(a, b))].update(int(u) for u in t)
    seen = 0
    for r in range(ny):
        for c in range(nx):
            for q, (dr, dc) in enumerate(((0, 1), (1, 0), (1, 1))):
                aff = oracle_lib.edge_affected(nx, ny, r, c, q)
                r2, c2 = r + dr, c + dc
                if r2 >= ny or c2 >= nx:
                    assert aff == []
                    continue
                e = (r * nx + c, r2 * nx + c2)
                assert aff == sorted(by_edge[e]), (r, c, q)
                seen += 1
    assert seen == len(by_edge)  # every edge of the triangulation, once


def _edge_scene(nx, ny, pos, vel, **kw):
    return make_scene(nx, ny, pos=pos, vel=vel, mesh=floor_mesh(), dt=1e-3, substeps=1, **kw)


def test_edge_phase_closed_form_single_edge_through_a_floor(oracle_lib):
    # two free nodes, no forces: the edge A*->B* crosses y = 0 at its midpoint
    # P; each node moves from its previous position towards P, stopping delta
    # short, and its velocity is scaled by -0.5 (Algorithm 2)
    pos = np.array([[0.3, 0.003, 0.3], [0.35, 0.003, 0.3]], np.float32)
    vel = np.array([[0.0, -2.0, 0.0], [0.0, -4.0, 0.0]], np.float32)
    sc = _edge_scene(2, 1, pos, vel)
    grid = oracle_lib.Grid(*floor_mesh())
    x, v, hits = oracle_lib.step_edges(oracle_lib.Cloth(sc), pos, vel, 0, 1, grid, want_hits=True)
    X = pos.astype(np.float64)
    Es = X + 1e-3 * vel.astype(np.float64)
    P = Es[0] + (Es[1] - Es[0]) * (Es[0, 1] / (Es[0, 1] - Es[1, 1]))
    for i in range(2):
        w = P - X[i]
        lw = np.linalg.norm(w)
        np.testing.assert_allclose(x[i], X[i] + (lw - 1e-4) / lw * w, rtol=0, atol=1e-12)
        np.testing.assert_allclose(v[i], -0.5 * vel[i].astype(np.float64), rtol=0, atol=1e-12)
    assert list(hits) == [1, 1]


def test_edge_phase_grid_equals_all_pairs_and_no_mesh_equals_plain_step(oracle_lib):
    rng = np.random.default_rng(31)
    nx, ny = 9, 7
    X0 = cs.flat_grid(nx, ny, (0.2, 0.004, 0.25), (0.05, 0.0, 0.0), (0.0, 0.0, 0.06))
    pos = (X0 + rng.uniform(-0.003, 0.003, X0.shape)).astype(np.float32)
    vel = rng.normal(0.0, 3.0, X0.shape).astype(np.float32)
    vel[:, 1] -= 5.0
    sc = _edge_scene(nx, ny, pos, vel, ks=(50.0, 30.0, 10.0), kd=(0.1, 0.1, 0.1), gravity=(0, -9.81, 0))
    grid = oracle_lib.Grid(*floor_mesh())
    cl = oracle_lib.Cloth(sc)
    a = oracle_lib.step_edges(cl, pos, vel, 0, 1, grid, want_hits=True)
    b = oracle_lib.step_edges(cl, pos, vel, 0, 1, grid, brute=True, want_hits=True)
    assert int(a[2].sum()) > 10
    for u, w in zip(a, b):
        assert np.array_equal(u, w)
    c = oracle_lib.step_edges(cl, pos, vel, 0, 3, None)
    d = oracle_lib.step(cl, pos, vel, 0, 3, None)
    for u, w in zip(c, d):
        assert np.array_equal(u, w)


def test_edge_phase_does_not_see_edges_parallel_to_the_surface(oracle_lib):
    # the method's blind spot (extended MT rejects |a| < eps): a flat cloth
    # that crosses a floor parallel to it keeps every edge parallel to the
    # floor, so no hit is found and the cloth passes through
    nx = ny = 3
    pos = cs.flat_grid(nx, ny, (0.3, 0.001, 0.3), (0.05, 0.0, 0.0), (0.0, 0.0, 0.05)).astype(np.float32)
    vel = np.zeros_like(pos)
    vel[:, 1] = -2.0
    sc = _edge_scene(nx, ny, pos, vel)
    x, _, hits = oracle_lib.step_edges(oracle_lib.Cloth(sc), pos, vel, 0, 1, oracle_lib.Grid(*floor_mesh()),
                                       want_hits=True)
    assert hits.sum() == 0 and np.all(x[:, 1] < 0.0)


# --------------------------------------------------- kinematic pins (f3)

@pytest.mark.parametrize("edges", [False, True])
def test_pinned_nodes_move_at_the_prescribed_velocity(oracle_lib, edges):
    # a pinned node under any force moves exactly x0 + k dt_s u with v = u;
    # its free neighbour is pulled along by the spring
    u = (0.4, -0.1, 0.25)
    pos = np.array([[0.2, 0.5, 0.3], [0.3, 0.5, 0.3]], np.float32)
    pinned = np.array([1, 0], np.uint8)
    sc = make_scene(2, 1, pos=pos, du=(0.1, 0, 0), dv=(0, 0, 0.1), ks=(50.0, 0, 0), kd=(0.1, 0, 0),
                    total_mass=0.02, gravity=(0, -9.81, 0), dt=1e-3, substeps=4, pinned=pinned, mesh=floor_mesh())
    sc.pin_velocity = u
    cl = oracle_lib.Cloth(sc)
    grid = oracle_lib.Grid(*floor_mesh())
    f = oracle_lib.step_edges if edges else oracle_lib.step
    k = 200
    x, v = f(cl, pos, np.zeros_like(pos), 0, k, grid)
    np.testing.assert_allclose(x[0], pos[0].astype(np.float64) + k * (1e-3 / 4) * np.array(u), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(v[0], np.array(u))
    assert x[1, 0] > pos[1, 0] + 0.005  # the free node follows (the pin moved 0.02 m)


def test_pulling_scene_is_the_hanging_model_with_moving_pins(oracle_lib):
    # zero pin velocity reduces the pulling scene's integrator to fixed pins
    sc = cs.pulling_scene(12, "sphere")
    x0 = oracle_lib.run(sc, 3)
    sc.pin_velocity = (0.0, 0.0, 0.0)
    x1 = oracle_lib.run(sc, 3)
    pin = sc.pinned.astype(bool)
    np.testing.assert_array_equal(x1[0][pin], sc.init_pos[pin].astype(np.float64))
    np.testing.assert_allclose(x0[0][pin][:, 0] - x1[0][pin][:, 0], 3 * (1 / 1200) * 0.5, rtol=0, atol=1e-12)
