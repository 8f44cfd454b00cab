"""Batched stepping (many cloths, one persistent launch per substep) against
the same cloths stepped one by one, and against the FP64 oracle."""
import numpy as np
import pytest

import cloth_scenes as cs
from helpers import floor_mesh, make_scene

pytestmark = pytest.mark.gpu


def _mixed_batch():
    # uneven sizes, odd shapes, pins, wind, per-spring constants, no mesh,
    # a floor, spheres of several levels; one dt / substep count for all
    sc = cs.config5(count=9, steps=10)
    w = cs.Wind(1.0, (0.0, 0.0, 1.0), (0.7, 0.0, 0.7), 1.5, 6.0, 0.3)
    pinned = np.zeros(37 * 23, np.uint8)
    pinned[:37] = 1
    extra = [
        make_scene(37, 23, origin=(0.1, 0.02, 0.1), du=(0.02, 0, 0), dv=(0, 0, 0.03), ks=(40.0, 20.0, 8.0),
                   kd=(0.05, 0.05, 0.02), gravity=(0, -9.81, 0), dt=1 / 1200, substeps=10, pinned=pinned,
                   mesh=floor_mesh(), wind=w),
        make_scene(1, 1, origin=(0.5, 0.2, 0.5), gravity=(0, -9.81, 0), dt=1 / 1200, substeps=10, mesh=floor_mesh()),
        make_scene(70, 3, du=(0.01, 0, 0), dv=(0, 0, 0.01), ks=(5.0, 2.0, 1.0), kd=(0.01, 0.01, 0.01),
                   gravity=(0, -9.81, 0), dt=1 / 1200, substeps=10),
    ]
    c4 = cs.config4()
    n4 = 48
    per = make_scene(n4, n4, du=(1 / 47, 0, 0), dv=(0, 0, 1 / 47), ks=c4.ks, kd=c4.kd, gravity=(0, -9.81, 0),
                     dt=1 / 1200, substeps=10)
    rng = np.random.default_rng(8)
    S = cs.spring_count(n4, n4)
    per.ks_spring = (rng.uniform(0.5, 1.5, S) * 20.0).astype(np.float32)
    per.kd_spring = (rng.uniform(0.5, 1.5, S) * 0.02).astype(np.float32)
    return sc + extra + [per]


def test_batch_equals_cloths_stepped_alone(cloth_lib):
    scenes = _mixed_batch()
    steps = 12
    with cloth_lib.ClothBatch(scenes) as b:
        b.step(steps)
        got = [b.read(i) for i in range(len(scenes))]
    for i, sc in enumerate(scenes):
        with cloth_lib.Cloth(sc) as cl:
            cl.step(steps)
            ref = cl.read()
        assert np.array_equal(got[i][0], ref[0]) and np.array_equal(got[i][1], ref[1]), sc.name


def test_batch_collision_statistics_equal_the_cloths_alone(cloth_lib):
    """Cloths starting 2-4 mm above their meshes: the batch lists, tests and
    hits exactly what the cloths do alone (its walk decides the listing with
    packed differences, the single walk with comparisons)."""
    scenes = [cs.small_collision_scene(n, level=lv, gap=g, seed=s)
              for n, lv, g, s in ((24, 2, 0.004, 5), (17, 1, 0.002, 6), (31, 2, 0.003, 7))]
    with cloth_lib.ClothBatch(scenes) as b:
        b.step(8)
        got = [b.read(i)[0] for i in range(len(scenes))]
        batch_stats = b.collision_stats()
    single = np.zeros(3, np.int64)
    for i, sc in enumerate(scenes):
        with cloth_lib.Cloth(sc) as cl:
            cl.step(8)
            assert np.array_equal(cl.read()[0], got[i])
            single += np.array(cl.collision_stats(), np.int64)
    assert tuple(int(x) for x in single) == tuple(batch_stats)
    assert batch_stats[0] > 0 and batch_stats[1] > 0 and batch_stats[2] > 0


def test_batch_matches_oracle(cloth_lib, oracle_lib):
    scenes = _mixed_batch()
    with cloth_lib.ClothBatch(scenes) as b:
        b.step(1)
        one = [b.read(i)[0] for i in range(len(scenes))]
        b.step(99)
        hundred = [b.read(i)[0] for i in range(len(scenes))]
    for i in (0, 3, len(scenes) - 4, len(scenes) - 3, len(scenes) - 1):
        sc = scenes[i]
        x1, _ = oracle_lib.run(sc, 1)
        assert np.max(np.abs(one[i] - x1)) <= 1e-5, sc.name
        x, _ = oracle_lib.run(sc, 100)
        assert np.max(np.abs(hundred[i] - x)) <= 1e-3, sc.name


def test_tuning_leaves_the_simulation_unchanged(cloth_lib):
    scenes = cs.config5(count=6, steps=10)
    with cloth_lib.ClothBatch(scenes) as a, cloth_lib.ClothBatch(scenes) as b:
        a.step(3)
        b.step(3)
        t = b.tune(4)
        assert t.candidates >= 7 and 1 <= t.rows_per_warp <= 32 and t.us_per_substep > 0
        assert b.tuning().rows_per_warp == t.rows_per_warp
        a.step(5)
        b.step(5)
        for i in range(len(scenes)):
            pa, va = a.read(i)
            pb, vb = b.read(i)
            assert np.array_equal(pa, pb) and np.array_equal(va, vb)
        # every explicit tuning gives the same bits
        for rows, ctas in ((4, 1), (32, 8), (7, 3)):
            b.set_tuning(rows, ctas)
            a.step(1)
            b.step(1)
            for i in range(len(scenes)):
                assert np.array_equal(a.read(i)[0], b.read(i)[0])


def test_batch_rejects_mixed_time_steps_and_bad_index(cloth_lib):
    s1 = make_scene(4, 4, dt=1e-3, substeps=2)
    s2 = make_scene(4, 4, dt=1e-3, substeps=3)
    with pytest.raises(cloth_lib.ClothError):
        cloth_lib.ClothBatch([s1, s2])
    with cloth_lib.ClothBatch([s1, s1]) as b:
        for bad in (2, -1):
            with pytest.raises(cloth_lib.ClothError) as ei:
                cloth_lib.capi.cloth_batch_read(b.h, bad, 16)
            assert ei.value.code == cloth_lib.capi.CLOTH_ERR_INVALID_ARG
        with pytest.raises(cloth_lib.ClothError):
            b.set_tuning(0, 1)
