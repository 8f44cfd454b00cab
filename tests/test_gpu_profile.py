"""The kernel-timing entry point advances the state exactly like cloth_step."""
import numpy as np
import pytest

import cloth_scenes as cs
from helpers import floor_mesh, make_scene

pytestmark = pytest.mark.gpu


def test_profiled_substeps_match_cloth_step(cloth_lib):
    P = cloth_lib
    sc = cs.small_collision_scene(24, level=2, gap=0.004, seed=5)
    with P.Cloth(sc) as a, P.Cloth(sc) as b:
        a.step(3)
        w, c = b.profile_substeps(3 * sc.substeps)
        pa, va = a.read()
        pb, vb = b.read()
    assert w > 0.0 and c > 0.0
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(va, vb)


def test_profiled_substeps_without_mesh(cloth_lib):
    P = cloth_lib
    sc = make_scene(9, 7, du=(0.05, 0, 0), dv=(0, -0.05, 0), total_mass=0.2, gravity=(0, -9.81, 0), dt=2e-3,
                    substeps=2)
    with P.Cloth(sc) as a, P.Cloth(sc) as b:
        a.step(2)
        w, c = b.profile_substeps(4)
        np.testing.assert_array_equal(a.read()[0], b.read()[0])
    assert w > 0.0 and c == 0.0


@pytest.mark.parametrize("mesh", [False, True])
def test_step_graphs_of_both_parities(cloth_lib, mesh):
    """cloth_step passes each walk its buffer parity; after an odd number of
    profiled substeps the step starts on the other parity (its second cached
    graph, or direct launches without graphs) and must equal the same
    substeps run by the path that reads the parity from the device."""
    P = cloth_lib
    kw = dict(mesh=floor_mesh()) if mesh else {}
    sc = make_scene(29, 17, origin=(0.0, 0.0003, 0.0), du=(0.03, 0, 0), dv=(0, 0, 0.03), total_mass=0.2,
                    gravity=(0, -9.81, 0), dt=2e-3, substeps=2, **kw)
    runs = []
    for flags in (0, P.capi.CLOTH_FLAG_NO_GRAPH):
        with P.Cloth(sc, flags=flags) as a:
            a.step(1)
            a.profile_substeps(3)
            a.step(2)
            a.profile_substeps(1)
            a.step(1)
            runs.append(a.read())
    with P.Cloth(sc) as ref:
        ref.profile_substeps(2 + 3 + 4 + 1 + 2)
        want = ref.read()
    for got in runs:
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])
