"""GPU reverse pass (cloth_rollout_*, torch.autograd.Function) against the
FP64 oracle's adjoint, and the FP64 adjoint against FP64 central finite
differences at the full differentiation workload.

Elementwise metric: rel err = |g - g_ref| / max(|g_ref|, 1e-3 max_k |g_ref,k|);
each test states its bound and why.
"""
import dataclasses

import numpy as np
import pytest

import cloth_scenes as cs
from helpers import config4_segment_fd, f32_segment_grads, floor_mesh, make_scene
from helpers import config4_target as config4_target_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(g, ref):
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
    return np.abs(g - ref) / scale


def _gpu_grads(P, sc, ks, kd, v0, tgt, nsteps, every):
    from paper_2507_11794_gb300.rollout import Rollout
    with P.Cloth(sc) as cl:
        ro = Rollout(cl, nsteps, every)
        k = torch.tensor(ks, dtype=torch.float32, device="cuda", requires_grad=True)
        d = torch.tensor(kd, dtype=torch.float32, device="cuda", requires_grad=True)
        v = torch.tensor(v0, dtype=torch.float32, device="cuda", requires_grad=True)
        pos, vel = ro(k, d, v)
        t = torch.tensor(tgt, dtype=torch.float32, device="cuda")
        loss = ((pos - t) ** 2).sum(1).mean()
        loss.backward()
        out = (k.grad.cpu().numpy(), d.grad.cpu().numpy(), v.grad.cpu().numpy(), pos.detach().cpu().numpy())
        ro.close()
    return out


def _oracle_grads(oracle_lib, sc, ks, kd, v0, tgt, nsteps, grid):
    cl = oracle_lib.Cloth(sc, ks_spring=ks, kd_spring=kd)
    nsub = nsteps * sc.substeps
    x, v = oracle_lib.step(cl, sc.init_pos, v0, 0, nsub, grid)
    N = sc.n
    _, lv0, gks, gkd = oracle_lib.adjoint(cl, sc.init_pos, v0, 0, nsub, 2 * (x - tgt) / N, np.zeros_like(x), grid)
    return gks, gkd, lv0, x


def _scene(kind, rng):
    n = 6
    if kind == "free":
        sc = make_scene(n, n, du=(0.05, 0, 0), dv=(0, 0, 0.05), total_mass=0.2, gravity=(0, -9.81, 0), dt=2e-3,
                        substeps=4, vel=rng.normal(0, 0.3, (n * n, 3)))
        grid = None
    elif kind == "pins_wind":
        pinned = np.zeros(35, np.uint8)
        pinned[[0, 6]] = 1
        sc = make_scene(7, 5, du=(0.05, 0, 0), dv=(0, -0.05, 0), total_mass=0.2, gravity=(0, -9.81, 0), dt=2e-3,
                        substeps=4, pinned=pinned, wind=cs.Wind(2.0, (0, 0, 1), (0.7, 0.7, 0), 3.0, 9.0, 0.4),
                        vel=rng.normal(0, 0.2, (35, 3)))
        grid = None
    else:
        vel = np.zeros((n * n, 3))
        vel[:, 1] = -0.6
        vel += rng.normal(0, 0.05, vel.shape)
        sc = make_scene(n, n, origin=(0.3, 0.0015, 0.3), du=(0.05, 0, 0), dv=(0, 0, 0.05), total_mass=0.2,
                        gravity=(0, -9.81, 0), dt=2e-3, substeps=4, vel=vel, mesh=floor_mesh(), delta=1e-4)
        grid = "floor"
    S = cs.spring_count(sc.nx, sc.ny)
    sc.ks_spring = rng.uniform(20, 40, S).astype(np.float32)
    sc.kd_spring = rng.uniform(0.01, 0.05, S).astype(np.float32)
    return sc, grid


def _l2(g, ref):
    g, ref = np.asarray(g, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    return float(np.linalg.norm(g - ref) / np.linalg.norm(ref))


def _cos(g, ref):
    g, ref = np.asarray(g, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    return float(np.dot(g, ref) / np.linalg.norm(g) / np.linalg.norm(ref))


@pytest.mark.parametrize("kind,every", [("free", 3), ("pins_wind", 4), ("contact", 2), ("contact", 100)])
def test_gpu_adjoint_matches_oracle_adjoint(cloth_lib, oracle_lib, kind, every):
    # Same float32 inputs; the GPU propagates the adjoints in float32 (per-spring
    # sums over substeps in double), the oracle in double.  Smooth cases: L2
    # rel err <= 1e-4 and every entry within 1e-2 of the floored metric (an
    # entry at 1e-3 of the largest carries ~40 substeps x 1e-7 x 1e3 of float32
    # error).  Contact: after a hit a node rests delta short of the surface, so
    # its next substep's t - delta sits at the kink of max(t - delta, 0), where
    # float32 and double may take opposite sides; L2 rel err <= 2e-3.
    rng = np.random.default_rng(11)
    sc, g = _scene(kind, rng)
    grid = oracle_lib.Grid(*floor_mesh()) if g else None
    nsteps = 10
    v0 = sc.init_vel.astype(np.float32)
    tgt = sc.init_pos + rng.normal(0, 0.01, sc.init_pos.shape)
    gks, gkd, gv0, pos = _gpu_grads(cloth_lib, sc, sc.ks_spring, sc.kd_spring, v0, tgt, nsteps, every)
    oks, okd, ov0, x = _oracle_grads(oracle_lib, sc, sc.ks_spring.astype(np.float64), sc.kd_spring.astype(np.float64),
                                     v0.astype(np.float64), tgt, nsteps, grid)
    assert np.max(np.abs(pos - x)) < 1e-5
    for got, ref in ((gks, oks), (gkd, okd), (gv0, ov0)):
        if kind == "contact":
            assert _l2(got, ref) <= 2e-3
        else:
            assert _l2(got, ref) <= 1e-4
            assert np.max(_rel(got, ref)) <= 1e-2


def test_gpu_adjoint_checkpointing_invariant(cloth_lib):
    rng = np.random.default_rng(12)
    sc, _ = _scene("contact", rng)
    v0 = sc.init_vel.astype(np.float32)
    tgt = sc.init_pos + rng.normal(0, 0.01, sc.init_pos.shape)
    a = _gpu_grads(cloth_lib, sc, sc.ks_spring, sc.kd_spring, v0, tgt, 12, 1)
    b = _gpu_grads(cloth_lib, sc, sc.ks_spring, sc.kd_spring, v0, tgt, 12, 5)
    c = _gpu_grads(cloth_lib, sc, sc.ks_spring, sc.kd_spring, v0, tgt, 12, 12)
    for x, y in ((a, b), (a, c)):
        for u, w in zip(x, y):
            assert np.array_equal(u, w)


def _config4_final(args):
    """Final FP64 oracle positions and contact signature of config 4 (worker
    of a spawned process pool)."""
    import oracle
    ks, kd, v0, nsteps = args
    sc = cs.config4()
    grid = oracle.Grid(sc.mesh_verts, sc.mesh_tris)
    cl = oracle.Cloth(sc, ks_spring=ks, kd_spring=kd)
    x, _, sig = oracle.step_signature(cl, sc.init_pos, v0, 0, nsteps * sc.substeps, grid)
    return x, sig


def test_config4_gradients(cloth_lib, oracle_lib):
    # 128x128 cloth over a 5,120-triangle icosphere, 256 steps, checkpoints
    # every 16; loss = mean squared distance to the target run (per-spring ks
    # * U(0.8,1.2), seed 3); 32 random parameters (seed 4).
    #  * the FP64 adjoint against FP64 central differences (h = 1e-6): every
    #    parameter within rel err 1e-3.  From step 121 on the cloth rests on
    #    the sphere and the trajectory is chaotic, so a parameter is re-drawn
    #    when its +-h or +-h/10 runs change the contact set (or which hits are
    #    active), or when the differences at h and h/10 disagree by more than
    #    1e-3 (the difference quotient has not converged).  The loss
    #    difference is summed as (x+ - x-).(x+ + x- - 2 target)/N, free of the
    #    cancellation of two separate sums.
    #  * the GPU gradient against the FP64 adjoint: the float32 trajectory
    #    parts from the double one in the chaotic stretch (a 1e-9 m change of
    #    the input moves the final state by ~3e-6 m), so direction (cosine >=
    #    0.99) and size (L2 rel err <= 0.2) are checked.
    import multiprocessing as mp
    sc = cs.config4()
    nsteps = sc.steps
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    target_ks = cs.config4_target_ks(sc)
    cl_t = oracle_lib.Cloth(sc, ks_spring=target_ks.astype(np.float64), kd_spring=sc.kd_spring.astype(np.float64))
    tgt, _ = oracle_lib.step(cl_t, sc.init_pos, sc.init_vel, 0, nsteps * sc.substeps, grid)
    ks = sc.ks_spring.astype(np.float64)
    kd = sc.kd_spring.astype(np.float64)
    v0 = sc.init_vel.astype(np.float64)
    gks, gkd, gv0, _ = _gpu_grads(cloth_lib, sc, sc.ks_spring, sc.kd_spring, sc.init_vel, tgt, nsteps, 16)
    oks, okd, ov0, _ = _oracle_grads(oracle_lib, sc, ks, kd, v0, tgt, nsteps, grid)
    for got, ref in ((gks, oks), (gkd, okd), (gv0, ov0)):
        assert _cos(got, ref) >= 0.99 and _l2(got, ref) <= 0.2, (_cos(got, ref), _l2(got, ref))

    rng = np.random.default_rng(4)
    h = 1e-6

    def perturbed(kind, idx, hh):
        if kind == "v0":
            i, c = idx
            vp, vm = v0.copy(), v0.copy()
            vp[i, c] += hh
            vm[i, c] -= hh
            return [(ks, kd, vp, nsteps), (ks, kd, vm, nsteps)]
        base = ks if kind == "ks" else kd
        p, m = base.copy(), base.copy()
        p[idx] += hh
        m[idx] -= hh
        return [(p, kd, v0, nsteps), (m, kd, v0, nsteps)] if kind == "ks" else \
               [(ks, p, v0, nsteps), (ks, m, v0, nsteps)]

    jobs, meta = [(ks, kd, v0, nsteps)], []
    for _ in range(64):  # candidates; 32 are kept
        kind = int(rng.integers(3))
        if kind == 2:
            idx = (int(rng.integers(sc.n)), int(rng.integers(3)))
            meta.append(("v0", idx, ov0[idx]))
        else:
            idx = int(rng.integers(len(ks)))
            meta.append(("ks" if kind == 0 else "kd", idx, (oks if kind == 0 else okd)[idx]))
        jobs += perturbed(meta[-1][0], idx, h) + perturbed(meta[-1][0], idx, h / 10)
    with mp.get_context("spawn").Pool(min(16, max(2, mp.cpu_count() or 2))) as pool:
        res = pool.map(_config4_final, jobs)
    sig0 = res[0][1]

    def quotient(a, b, hh):
        (xp, sp), (xm, sm) = a, b
        dL = float(np.sum((xp - xm) * (xp + xm - 2.0 * tgt)) / len(xp))
        return dL / (2.0 * hh), sp == sig0 and sm == sig0

    rows = []
    for j, (kind, idx, g) in enumerate(meta):
        f1, ok1 = quotient(res[1 + 4 * j], res[2 + 4 * j], h)
        f2, ok2 = quotient(res[3 + 4 * j], res[4 + 4 * j], h / 10)
        rows.append((kind, idx, g, f1, f2, ok1 and ok2))
    same_contacts = [r for r in rows if r[5]]
    assert len(same_contacts) >= 32
    floor = 1e-3 * max(abs(r[3]) for r in same_contacts[:32])
    got, fds, redrawn = [], [], []
    for kind, idx, g, f1, f2, ok in rows:
        if not ok or abs(f1 - f2) > 1e-3 * max(abs(f1), floor):
            redrawn.append((kind, idx))
            continue
        got.append(g)
        fds.append(f1)
        if len(got) == 32:
            break
    print(f"config4 FD: {len(got)} parameters kept, re-drawn: {redrawn}")
    assert len(got) == 32
    rel = np.abs(np.array(got) - np.array(fds)) / np.maximum(np.abs(fds), floor)
    assert np.max(rel) <= 1e-3, rel


def _grads_twice(P, sc, tgt, nsteps, every, flags=0, swap_mesh=None):
    """Two forward/backward passes of one rollout (the second replays any
    cached graphs); optionally replaces the cloth's mesh between them."""
    from paper_2507_11794_gb300.rollout import Rollout
    outs = []
    with P.Cloth(sc, flags=flags) as cl:
        ro = Rollout(cl, nsteps, every)
        for it in range(2):
            if it == 1 and swap_mesh is not None:
                cl.set_mesh(*swap_mesh)
            k = torch.tensor(sc.ks_spring, dtype=torch.float32, device="cuda", requires_grad=True)
            d = torch.tensor(sc.kd_spring, dtype=torch.float32, device="cuda", requires_grad=True)
            v = torch.tensor(sc.init_vel.astype(np.float32), device="cuda", requires_grad=True)
            pos, vel = ro(k, d, v)
            loss = ((pos - torch.tensor(tgt, dtype=torch.float32, device="cuda")) ** 2).sum(1).mean()
            loss.backward()
            outs.append((k.grad.cpu().numpy(), d.grad.cpu().numpy(), v.grad.cpu().numpy(),
                         pos.detach().cpu().numpy()))
        ro.close()
    return outs


def test_rollout_graphs_match_direct_launches(cloth_lib):
    # The forward chain and the reverse pass replayed from CUDA graphs give
    # the same bits as the same launches issued one by one
    # (CLOTH_FLAG_NO_GRAPH), on the first call and on replays; a segment
    # shorter than the others (10 steps, checkpoints every 4) is covered.
    P = cloth_lib
    rng = np.random.default_rng(13)
    sc, _ = _scene("contact", rng)
    tgt = sc.init_pos + rng.normal(0, 0.01, sc.init_pos.shape)
    a = _grads_twice(P, sc, tgt, 10, 4)
    b = _grads_twice(P, sc, tgt, 10, 4, flags=P.capi.CLOTH_FLAG_NO_GRAPH)
    for x in (a[0], a[1], b[1]):
        for u, w in zip(x, b[0]):
            assert np.array_equal(u, w)


def test_rollout_follows_a_mesh_change(cloth_lib):
    # Replacing the mesh after the rollout captured its graphs rebuilds them:
    # the second pass matches a fresh rollout over the new mesh (here: no
    # mesh, so the falling cloth meets nothing).
    P = cloth_lib
    rng = np.random.default_rng(14)
    sc, _ = _scene("contact", rng)
    tgt = sc.init_pos + rng.normal(0, 0.01, sc.init_pos.shape)
    a = _grads_twice(P, sc, tgt, 10, 4, swap_mesh=(None, None))
    free = dataclasses.replace(sc, mesh_verts=None, mesh_tris=None)
    b = _grads_twice(P, free, tgt, 10, 4)
    assert not np.array_equal(a[0][3], a[1][3])  # the contact changed the result
    for u, w in zip(a[1], b[0]):
        assert np.array_equal(u, w)


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 1), (1, 3), (3, 2)])
def test_rollout_on_minimal_cloths(cloth_lib, oracle_lib, nx, ny):
    # Cloths with no springs (1x1), only structural ones (1x3) and the smallest
    # with shear springs, falling onto the floor: the GPU gradients match the
    # FP64 adjoint; a spring-less cloth returns empty per-spring gradients.
    # Bound: L2 rel err <= 1e-2.  These springs stay within about 1e-6 of
    # their rest length, so dL/dks ~ (l - L0) carries the float32 cancellation
    # of l - L0, about 1e-7 l / |l - L0| ~ 5e-3 relative (measured 2.3e-3 at
    # 3x2), on top of the contact kink of the test above.
    rng = np.random.default_rng(15 + nx * 7 + ny)
    n = nx * ny
    vel = np.zeros((n, 3))
    vel[:, 1] = -0.6
    vel += rng.normal(0, 0.05, vel.shape)
    sc = make_scene(nx, ny, origin=(0.3, 0.0015, 0.3), du=(0.05, 0, 0), dv=(0, 0, 0.05), total_mass=0.2,
                    gravity=(0, -9.81, 0), dt=2e-3, substeps=4, vel=vel, mesh=floor_mesh(), delta=1e-4)
    S = cs.spring_count(nx, ny)
    sc.ks_spring = rng.uniform(20, 40, S).astype(np.float32)
    sc.kd_spring = rng.uniform(0.01, 0.05, S).astype(np.float32)
    v0 = sc.init_vel.astype(np.float32)
    tgt = sc.init_pos + rng.normal(0, 0.01, sc.init_pos.shape)
    gks, gkd, gv0, pos = _gpu_grads(cloth_lib, sc, sc.ks_spring, sc.kd_spring, v0, tgt, 8, 3)
    oks, okd, ov0, x = _oracle_grads(oracle_lib, sc, sc.ks_spring.astype(np.float64),
                                     sc.kd_spring.astype(np.float64), v0.astype(np.float64), tgt, 8,
                                     oracle_lib.Grid(*floor_mesh()))
    assert np.max(np.abs(pos - x)) < 1e-5
    assert gks.shape == (S,) and gkd.shape == (S,)
    pairs = [(gv0, ov0)] + ([(gks, oks), (gkd, okd)] if S else [])
    for got, ref in pairs:
        assert _l2(got, ref) <= 1e-2


@pytest.fixture(scope="module")
def config4_target(oracle_lib):
    return config4_target_state(oracle_lib)


# bounds of the GPU gradient in the segment check (see the test): entries at
# >= 1e-2 of the largest, and all 32 (the float32 floor of the smallest)
GPU_BIG = {60: 1e-3, 121: 1e-3, 240: 5e-3}
GPU_FLOOR = {60: 2e-3, 121: 5e-3, 240: 2e-2}


@pytest.mark.parametrize("start", [60, 121, 240])
def test_config4_segment_gradients_match_fd(cloth_lib, oracle_lib, config4_target, start):
    # The differentiation workload's gradient check with the chaos taken out:
    # the GPU steps config 4 to `start` (before contact, at contact onset,
    # resting on the sphere) and its float32 state starts one checkpoint
    # segment (16 steps) on the GPU and in the FP64 oracle.  Loss = mean
    # squared distance of the segment's final positions to the workload's
    # target state.  32 seeded parameters (ks, kd of a spring or a component
    # of the segment's initial velocity), FP64 central differences at
    # h = 1e-6 of the oracle from the same float32 start; a parameter is
    # re-drawn when its +-h or +-h/10 runs change the contact set or the
    # active hits, or when the two quotients disagree by more than 1e-3.
    # Bounds (rel err floored at 1e-3 of the largest |g_fd|):
    #  * the oracle's FP64 adjoint: <= 1e-3 on every parameter;
    #  * the GPU's float32 gradient, on every parameter whose |g_fd| is at
    #    least 1e-2 of the largest: <= 1e-3 before contact and at its onset
    #    (measured 4e-6); resting on the sphere, <= 5e-3 (measured 4.0e-3 on
    #    v0 entries of resting nodes, whose substep paths end at the kink of
    #    max(t - delta, 0), where float32 and double can take opposite sides
    #    on some substeps while the FP64 adjoint matches the differences to
    #    1e-9);
    #  * the GPU on all 32: within 1e-3, or within twice the error of the
    #    float32 restatement of the oracle (oracle.f32: the same algorithm
    #    in the same order with every intermediate rounded to float32) from
    #    the same float32 start, on the same parameters.  The smallest
    #    entries sit at that float32 floor: kd gradients of springs with
    #    almost no stretch rate (1e-6 of the largest gradient, where the
    #    float32 rounding of the node velocities, 6e-8 m/s, exceeds the
    #    relative velocity the gradient measures).  Measured, GPU against
    #    the restatement: 1.1e-3 / 1.7e-3 (step 60), 3.8e-3 / 2.0e-2 (121),
    #    4.0e-3 / 5.1e-3 (240); on the large entries 5.1e-6 / 4.8e-6,
    #    6.2e-6 / 6.1e-6, 4.0e-3 / 3.5e-3.  GPU_FLOOR caps the measured GPU
    #    levels against regressions.
    P = cloth_lib
    sc = cs.config4()
    seg = 16
    tgt = config4_target
    with P.Cloth(sc) as cl:
        cl.step(start)
        x_s, v_s = cl.read()
    seg_sc = dataclasses.replace(sc, init_pos=x_s.astype(np.float32), init_vel=v_s.astype(np.float32))
    k0 = start * sc.substeps
    nsub = seg * sc.substeps
    # GPU: one rollout segment from the float32 state (config 4 has no wind,
    # so a segment does not depend on its start time)
    gks, gkd, gv0, gpos = _gpu_grads(P, seg_sc, sc.ks_spring, sc.kd_spring, v_s.astype(np.float32), tgt, seg, 16)
    ks = sc.ks_spring.astype(np.float64)
    kd = sc.kd_spring.astype(np.float64)
    x0 = x_s.astype(np.float64)
    v0 = v_s.astype(np.float64)
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    cl_o = oracle_lib.Cloth(sc, ks_spring=ks, kd_spring=kd)
    x_end, _ = oracle_lib.step(cl_o, x0, v0, k0, nsub, grid)
    dx = float(np.max(np.abs(gpos - x_end)))
    assert dx < 1e-3, dx  # the 100-step position gate over these 16 steps
    _, ov0, oks, okd = oracle_lib.adjoint(cl_o, x0, v0, k0, nsub, 2 * (x_end - tgt) / sc.n, np.zeros_like(x_end), grid)
    fks, fkd, fv0, _ = f32_segment_grads(x_s, v_s, k0, nsub, tgt)

    rel, kept, fds, redrawn = config4_segment_fd(
        x0, v0, k0, nsub, tgt, {"gpu": (gks, gkd, gv0), "oracle": (oks, okd, ov0), "f32": (fks, fkd, fv0)},
        seed=4 + start)
    rel_gpu, rel_ora, rel_f32 = rel["gpu"], rel["oracle"], rel["f32"]
    big = np.abs(fds) >= 1e-2 * np.max(np.abs(fds))
    print(f"config4 segment from step {start}: max |dx| {dx:.2e} m, re-drawn {redrawn}; max rel err GPU "
          f"{rel_gpu.max():.2e}, float32 restatement {rel_f32.max():.2e}, oracle adjoint {rel_ora.max():.2e}")
    for j in np.argsort(-rel_gpu)[:4]:
        print(f"  {kept[j]} fd {fds[j]:.6e} rel GPU {rel_gpu[j]:.2e} float32 restatement {rel_f32[j]:.2e}")
    print(f"  on the {int(big.sum())} entries at >= 1e-2 of the largest: GPU {rel_gpu[big].max():.2e}, "
          f"float32 restatement {rel_f32[big].max():.2e}")
    assert rel_ora.max() <= 1e-3, rel_ora
    assert rel_gpu[big].max() <= GPU_BIG[start], rel_gpu[big]
    assert rel_gpu.max() <= max(1e-3, 2.0 * rel_f32.max()), (rel_gpu, rel_f32)
    assert rel_gpu.max() <= GPU_FLOOR[start], rel_gpu
