"""Pins of the oracle's reverse-mode step against FP64 central finite
differences of the oracle's own (independently pinned) forward step.

Gradients of L = mean |x_T - target|^2 w.r.t. per-spring ks, kd and the
initial velocities.  rel err = |g - g_fd| / max(|g_fd|, 1e-3 max_k |g_fd,k|)
<= 1e-3; a parameter whose +-h runs change the contact set is re-drawn.
"""
import numpy as np
import pytest

import cloth_scenes as cs
from helpers import floor_mesh, make_scene


def _loss(oracle_lib, sc, ks, kd, v0, tgt, nsub, grid):
    cl = oracle_lib.Cloth(sc, ks_spring=ks, kd_spring=kd)
    x, v, sig = oracle_lib.step_signature(cl, sc.init_pos, v0, 0, nsub, grid)
    return float(np.sum((x - tgt) ** 2) / len(x)), x, sig


def _check(oracle_lib, sc, nsub, grid, rng, nparam=24, h=1e-6):
    N = sc.n
    S = cs.spring_count(sc.nx, sc.ny)
    ks = np.asarray(sc.ks_spring, np.float64)
    kd = np.asarray(sc.kd_spring, np.float64)
    v0 = sc.init_vel.astype(np.float64)
    tgt = sc.init_pos.astype(np.float64) + rng.normal(0, 0.01, (N, 3))
    L0, x, sig0 = _loss(oracle_lib, sc, ks, kd, v0, tgt, nsub, grid)
    cl = oracle_lib.Cloth(sc, ks_spring=ks, kd_spring=kd)
    _, lv0, gks, gkd = oracle_lib.adjoint(cl, sc.init_pos, v0, 0, nsub, 2 * (x - tgt) / N, np.zeros_like(x), grid)
    got, fds, redraws = [], [], 0
    while len(got) < nparam:
        kind = rng.integers(3)
        if kind == 2:
            i, k = int(rng.integers(N)), int(rng.integers(3))
            vp, vm = v0.copy(), v0.copy()
            vp[i, k] += h
            vm[i, k] -= h
            Lp, _, sp = _loss(oracle_lib, sc, ks, kd, vp, tgt, nsub, grid)
            Lm, _, sm = _loss(oracle_lib, sc, ks, kd, vm, tgt, nsub, grid)
            g = lv0[i, k]
        else:
            s = int(rng.integers(S))
            base = ks if kind == 0 else kd
            p, m = base.copy(), base.copy()
            p[s] += h
            m[s] -= h
            args_p = (p, kd) if kind == 0 else (ks, p)
            args_m = (m, kd) if kind == 0 else (ks, m)
            Lp, _, sp = _loss(oracle_lib, sc, *args_p, v0, tgt, nsub, grid)
            Lm, _, sm = _loss(oracle_lib, sc, *args_m, v0, tgt, nsub, grid)
            g = (gks if kind == 0 else gkd)[s]
        if sp != sig0 or sm != sig0:
            redraws += 1
            assert redraws < 4 * nparam, "contact set too fragile for finite differences"
            continue
        got.append(g)
        fds.append((Lp - Lm) / (2 * h))
    got, fds = np.array(got), np.array(fds)
    scale = np.maximum(np.abs(fds), 1e-3 * np.max(np.abs(fds)))
    rel = np.abs(got - fds) / scale
    assert np.max(rel) <= 1e-3, (rel, got, fds)
    return redraws


def test_adjoint_matches_fd_without_contact(oracle_lib):
    rng = np.random.default_rng(1)
    n = 6
    S = cs.spring_count(n, n)
    sc = make_scene(n, n, du=(0.05, 0, 0), dv=(0, 0, 0.05), total_mass=0.2, ks=(30, 20, 10), kd=(0.02, 0.02, 0.02),
                    gravity=(0, -9.81, 0), dt=2e-3, substeps=4, vel=rng.normal(0, 0.3, (n * n, 3)))
    sc.ks_spring = rng.uniform(20, 40, S)
    sc.kd_spring = rng.uniform(0.01, 0.05, S)
    _check(oracle_lib, sc, 40, None, rng)


def test_adjoint_matches_fd_with_pins_and_wind(oracle_lib):
    rng = np.random.default_rng(2)
    nx, ny = 7, 5
    S = cs.spring_count(nx, ny)
    pinned = np.zeros(nx * ny, np.uint8)
    pinned[[0, nx - 1]] = 1
    w = cs.Wind(2.0, (0.0, 0.0, 1.0), (0.7, 0.7, 0.0), 3.0, 9.0, 0.4)
    sc = make_scene(nx, ny, du=(0.05, 0, 0), dv=(0, -0.05, 0), total_mass=0.2, gravity=(0, -9.81, 0), dt=2e-3,
                    substeps=4, pinned=pinned, wind=w, vel=rng.normal(0, 0.2, (nx * ny, 3)))
    sc.ks_spring = rng.uniform(20, 40, S)
    sc.kd_spring = rng.uniform(0.01, 0.05, S)
    _check(oracle_lib, sc, 48, None, rng)


def test_adjoint_matches_fd_through_contact(oracle_lib):
    # a cloth pressed onto a floor: many substeps with active contacts
    rng = np.random.default_rng(3)
    n = 6
    S = cs.spring_count(n, n)
    vel = np.zeros((n * n, 3))
    vel[:, 1] = -0.6
    vel += rng.normal(0, 0.05, vel.shape)
    sc = make_scene(n, n, origin=(0.3, 0.0015, 0.3), du=(0.05, 0, 0), dv=(0, 0, 0.05), total_mass=0.2,
                    gravity=(0, -9.81, 0), dt=2e-3, substeps=4, vel=vel, mesh=floor_mesh(), delta=1e-4)
    sc.ks_spring = rng.uniform(20, 40, S)
    sc.kd_spring = rng.uniform(0.01, 0.05, S)
    grid = oracle_lib.Grid(*floor_mesh())
    cl = oracle_lib.Cloth(sc)
    hits_total = 0
    x, v = sc.init_pos, sc.init_vel
    for s in range(32):
        x, v, h = oracle_lib.step(cl, x, v, s, 1, grid, want_hits=True)
        hits_total += int((h > 0).sum())
    assert hits_total > 20
    _check(oracle_lib, sc, 32, grid, rng)


def test_adjoint_of_a_single_contact_substep_closed_form(oracle_lib):
    # One free node, no springs, one substep onto the floor from height y0
    # with velocity (ux, -w, uz): the hit stops it delta short along the path,
    # x' = S + (t - delta) r with t = y0 / (w/|v|), so
    # d x'_y / d y0 = 1 - (w/|v|)^{-1} (w/|v|) = 0 (it stops at delta|r_y|),
    # and d x'_x / d y0 = r_x / (w/|v|) = ux / w.
    ux, w, uz, y0, dt = 0.3, 2.0, -0.2, 0.0015, 1e-3
    sc = make_scene(1, 1, origin=(0.4, y0, 0.6), vel=[[ux, -w, uz]], dt=dt, mesh=floor_mesh(), delta=1e-4)
    grid = oracle_lib.Grid(*floor_mesh())
    cl = oracle_lib.Cloth(sc)
    for comp, expect in ((0, [1.0, float(sc.init_vel[0, 0]) / float(-sc.init_vel[0, 1]), 0.0]),
                         (1, [0.0, 0.0, 0.0])):
        lx = np.zeros((1, 3))
        lx[0, comp] = 1.0
        lx0, lv0, _, _ = oracle_lib.adjoint(cl, sc.init_pos, sc.init_vel, 0, 1, lx, np.zeros((1, 3)), grid)
        # dL/dS where L = x'_comp
        np.testing.assert_allclose(lx0[0], expect, atol=1e-12)
