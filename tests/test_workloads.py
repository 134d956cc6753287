"""The seeded synthetic inputs match the workload recipe they stand in for.

The configurations: 10x10x20 with 6 wells (seed 1), 48x48x96 with 24 (seed
2), 96x96x192 with 80 (seed 3), 64x64x128 with 40 (seed 5), all at h = 0.5
bohr; wells of depth U[1, 3] Ha and standard deviation 1 bohr on the wire
axis; Gaussian absorbers of height 0.5 Ha and standard deviation 2 bohr at the
two cell ends (Section 1).  The uneven batch: 64 wires, x and y axes in
16..48, z twice 16..48, 8-40 wells, 32-256 pairs in 2-8 windows, sub-seeds
4000 + s.
"""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("name,grid,wells,seed,n_r,p,n_E", [
    ("wire_10x10x20", (10, 10, 20), 6, 1, 48, 4, 32),
    ("wire_48x48x96", (48, 48, 96), 24, 2, 400, 8, 128),
    ("wire_96x96x192", (96, 96, 192), 80, 3, 2000, 32, 0),
    ("wire_64x64x128", (64, 64, 128), 40, 5, 1000, 16, 256),
])
def test_configuration_table(name, grid, wells, seed, n_r, p, n_E):
    c = W.CONFIGS[name]
    assert (c["nx"], c["ny"], c["nz"]) == grid and c["h"] == 0.5
    assert (c["n_wells"], c["seed"], c["n_r"], c["p"], c["n_E"]) == (wells, seed, n_r, p, n_E)


def test_wells_and_absorbers_of_a_small_wire():
    w = W.make_wire(8, 7, 20, 0.5, 5, 11)
    assert w.N == 8 * 7 * 20 and w.V.shape == (w.N,)
    assert np.all((w.d_wells >= 1.0) & (w.d_wells <= 3.0))
    assert np.all((w.z_wells >= 0.0) & (w.z_wells <= 19 * 0.5))
    # brute force at a few points: V(r) = -sum_w d_w exp(-|r - r_w|^2 / 2)
    x, y, z = W.coordinates(8, 7, 20, 0.5)
    for (i, j, k) in [(0, 0, 0), (3, 4, 7), (7, 6, 19), (4, 3, 10)]:
        r2 = x[i] ** 2 + y[j] ** 2 + (z[k] - w.z_wells) ** 2
        v = -np.sum(w.d_wells * np.exp(-r2 / 2.0))
        assert abs(w.V[(k * 7 + j) * 8 + i] - v) <= 1e-14
    # absorbers: 0.5 Ha on the end planes, 0.5 exp(-1/2) one standard deviation (4 planes) in
    gl = w.gamma_L.reshape(20, 7, 8)
    gr = w.gamma_R.reshape(20, 7, 8)
    assert np.allclose(gl[0], 0.5) and np.allclose(gr[19], 0.5)
    assert np.allclose(gl[4], 0.5 * np.exp(-0.5)) and np.allclose(gr[15], 0.5 * np.exp(-0.5))
    assert np.all(gl >= 0) and np.all(np.diff(gl[:, 0, 0]) < 0) and np.all(np.diff(gr[:, 0, 0]) > 0)


def test_wire_axis_is_the_grid_centre_line():
    x, y, z = W.coordinates(6, 5, 4, 0.5)
    assert np.allclose(x, -x[::-1]) and np.allclose(y, -y[::-1]) and z[0] == 0.0 and z[-1] == 1.5


def test_uneven_batch_recipe():
    specs = W.batch_systems(seed=4, count=64)
    assert len(specs) == 64
    for s, sp in enumerate(specs):
        assert 16 <= sp["nx"] <= 48 and 16 <= sp["ny"] <= 48
        assert sp["nz"] % 2 == 0 and 16 <= sp["nz"] // 2 <= 48
        assert 8 <= sp["n_wells"] <= 40 and 32 <= sp["n_r"] <= 256 and 2 <= sp["p"] <= 8
        assert sp["seed"] == 4000 + s
    # uneven: the grids differ
    assert len({(sp["nx"], sp["ny"], sp["nz"]) for sp in specs}) > 32
    # seeded: the same table twice
    assert W.batch_systems(seed=4, count=64) == specs
