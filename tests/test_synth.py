"""The seeded input recipes (no arithmetic of the method): the grid of Section 2.1, the
velocity fields and sources the workloads are built from, and their determinism."""
import numpy as np

import synth


def test_grid_is_the_interior_nodes():
    x, h = synth.grid(7)
    assert h == 1.0 / 8
    assert np.allclose(x, np.arange(1, 8) / 8.0)


def test_random_medium_recipe_of_the_bench_workload():
    # c = 1 + 0.2 g, g Gaussian-filtered (width 1/32) N(0, 1) noise of unit standard deviation
    w = synth.workload("n1023_random")
    c = w["c"]
    assert c.shape == (1023, 1023)
    assert abs(c.std() - 0.2) < 1e-12
    assert c.min() > 0.0
    g = (c - 1.0) / 0.2
    # smooth on the filter's scale (32 nodes): neighbouring nodes almost equal, nodes a
    # filter width apart much less correlated
    lag1 = np.corrcoef(g[:, :-1].ravel(), g[:, 1:].ravel())[0, 1]
    lag64 = np.corrcoef(g[:, :-64].ravel(), g[:, 64:].ravel())[0, 1]
    assert lag1 > 0.99 and lag64 < 0.5
    # seeded: the same field again, another seed a different one
    assert np.array_equal(c, synth.velocity_random(1023, 1 / 32, 1))
    assert not np.allclose(c, synth.velocity_random(1023, 1 / 32, 2))


def test_point_sources_of_the_bench_workload():
    # 64 discrete deltas (mass one: 1/h^2 at one node) at seeded positions inside the PML
    w = synth.workload("n1023_random")
    n, pml = w["n"], w["pml"]
    f = w["f"]
    _, h = synth.grid(n)
    eta = pml * h
    assert f.shape == (64, n, n)
    for s in range(64):
        nz = np.argwhere(f[s] != 0)
        assert len(nz) == 1
        j, i = nz[0]
        assert f[s, j, i] == 1.0 / (h * h)
        x1, x2 = (i + 1) * h, (j + 1) * h
        assert eta - h <= x1 <= 1 - eta + h and eta - h <= x2 <= 1 - eta + h
    assert np.array_equal(f, synth.workload("n1023_random")["f"])


def test_lens_and_gaussian_source():
    n = 511
    c = synth.velocity_lens(n)
    mid = n // 2                                   # node (256 h, 256 h) = (0.5, 0.5)
    assert abs(c[mid, mid] - 2.0 / 3.0) < 1e-12
    assert abs(c[0, 0] - 4.0 / 3.0) < 1e-6
    f = synth.source_gaussian(n)
    assert np.unravel_index(np.argmax(np.abs(f)), f.shape) == (mid, mid)
    assert abs(f[mid, mid] - 1.0) < 1e-12
