"""The float32 floor of the differentiation workload's gradient check.

The gradient target of the 128x128 differentiation workload is rel err
<= 1e-3 against FP64 central differences on 32 seeded parameters, with
rel err = |g - g_fd| / max(|g_fd|, 1e-3 max_k |g_fd,k|).  This file asks how
close ANY float32 evaluation of the method can come: the float32
restatement of the oracle (oracle.f32, the oracle's own steps with every
intermediate rounded to float32) runs one checkpoint segment (16 steps)
from float32 states of the workload before contact (step 60) and at
contact onset (step 121), and its gradients go through the same
finite-difference check as the GPU's.

Measured: on the entries at >= 1e-2 of the largest gradient the float32
restatement is within 1.3e-6 and 6.7e-6; on all 32 it reaches 1.7e-3 and
1.9e-2, on the kd gradients of springs with almost no stretch rate (the
float32 rounding of the node velocities exceeds the relative velocity that
gradient measures).  So 1e-3 on every parameter is below the float32 floor,
while the FP64 adjoint meets it.  The GPU test of the same segments holds the
GPU to 1e-3 or to twice this restatement's error, whichever is larger.
"""
import numpy as np
import pytest

import cloth_scenes as cs
from helpers import config4_segment_fd, config4_target, f32_segment_grads


@pytest.fixture(scope="module")
def target(oracle_lib):
    return config4_target(oracle_lib)


def test_restated_source_is_float_only():
    import oracle.f32 as o32
    import re
    src = o32.restated_source()
    assert not re.search(r"\bdouble\b", src)
    assert not re.search(r"\b(sqrt|fabs|floor|sin)\(", src)
    o32.build()


def test_float32_floor_of_config4_segment_gradients(oracle_lib, target):
    sc = cs.config4()
    grid = oracle_lib.Grid(sc.mesh_verts, sc.mesh_tris)
    ks = sc.ks_spring.astype(np.float64)
    kd = sc.kd_spring.astype(np.float64)
    cl = oracle_lib.Cloth(sc, ks_spring=ks, kd_spring=kd)
    nsub = 16 * sc.substeps
    worst = {}
    for start in (60, 121):
        k0 = start * sc.substeps
        xs, vs = oracle_lib.step(cl, sc.init_pos, sc.init_vel, 0, k0, grid)
        x0, v0 = xs.astype(np.float32), vs.astype(np.float32)
        x_end, _ = oracle_lib.step(cl, x0, v0, k0, nsub, grid)
        _, ov0, oks, okd = oracle_lib.adjoint(cl, x0, v0, k0, nsub, 2 * (x_end - target) / sc.n,
                                              np.zeros_like(x_end), grid)
        fks, fkd, fv0, x32 = f32_segment_grads(x0, v0, k0, nsub, target)
        # the float32 restatement follows the FP64 segment (measured 1.4e-8, 6.0e-8 m)
        assert np.max(np.abs(x32.astype(np.float64) - x_end)) < 1e-6
        rel, kept, fds, redrawn = config4_segment_fd(x0, v0, k0, nsub, target,
                                                     {"oracle": (oks, okd, ov0), "f32": (fks, fkd, fv0)},
                                                     seed=4 + start)
        big = np.abs(fds) >= 1e-2 * np.max(np.abs(fds))
        print(f"step {start}: re-drawn {len(redrawn)}; max rel err FP64 adjoint {rel['oracle'].max():.2e}, "
              f"float32 restatement {rel['f32'].max():.2e} (entries >= 1e-2 of the largest: "
              f"{rel['f32'][big].max():.2e})")
        assert rel["oracle"].max() <= 1e-3
        assert rel["f32"][big].max() <= 1e-4
        worst[start] = rel["f32"].max()
    # 1e-3 on every parameter is out of reach of float32 arithmetic
    assert max(worst.values()) > 1e-3, worst
