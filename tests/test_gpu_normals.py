"""Per-vertex normals on the GPU against the oracle's, on simulated states.

Both sides take the same float32 positions (read back from the GPU), the
oracle in double.  Differences of neighbouring float32 positions are exact,
so the GPU's error is the rounding of a few cross products and a
normalisation: 2e-5 is far above it while folds are absent.
"""
import numpy as np
import pytest

import cloth_scenes as cs
from helpers import make_scene
from test_gpu_parity import SCENES

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,steps", [("config1", 60), ("config3_small_wind", 40), ("ragged_45x19_floor", 30)])
def test_normals_match_oracle_on_simulated_states(cloth_lib, oracle_lib, name, steps):
    sc = SCENES[name]()
    with cloth_lib.Cloth(sc) as cl:
        cl.step(steps)
        n_gpu = cl.normals().cpu().numpy()
        pos, _ = cl.read()
    n_ref = oracle_lib.normals(pos, sc.nx, sc.ny)
    assert np.max(np.abs(n_gpu - n_ref)) <= 2e-5


def test_normals_of_the_initial_flat_cloth_and_minimal_grids(cloth_lib, oracle_lib):
    for nx, ny in ((1, 1), (1, 5), (2, 2), (61, 3)):
        sc = make_scene(nx, ny, du=(0.1, 0, 0), dv=(0, -0.1, 0), total_mass=0.1)
        with cloth_lib.Cloth(sc) as cl:
            n_gpu = cl.normals().cpu().numpy()
            pos, _ = cl.read()
        np.testing.assert_allclose(n_gpu, oracle_lib.normals(pos, nx, ny), atol=1e-6)


@pytest.mark.parametrize("nx,ny", [(30, 5), (31, 6), (60, 10), (91, 11), (2, 7), (7, 2)])
def test_normals_at_strip_boundaries(cloth_lib, oracle_lib, nx, ny):
    # The kernel walks strips of 30 output columns and 5 rows: sizes on and
    # one past those boundaries, on a bumped (non-flat) cloth.
    X0 = cs.flat_grid(nx, ny, (0.0, 0.0, 0.0), (0.05, 0.0, 0.0), (0.0, 0.05, 0.0))
    X0 = np.asarray(X0, np.float64).reshape(-1, 3)
    X0[:, 2] = 0.03 * np.sin(7.0 * X0[:, 0]) * np.cos(5.0 * X0[:, 1])
    sc = make_scene(nx, ny, du=(0.05, 0, 0), dv=(0, 0.05, 0), total_mass=0.1, pos=X0.astype(np.float32))
    with cloth_lib.Cloth(sc) as cl:
        n_gpu = cl.normals().cpu().numpy()
        pos, _ = cl.read()
    np.testing.assert_allclose(n_gpu, oracle_lib.normals(pos, nx, ny), atol=2e-5)
