"""The seeded synthetic inputs: meshes are closed, outward wound and of the
stated sizes; the random stream is reproducible."""
import numpy as np
import pytest

from workloads import (WORKLOADS, PCG32, random_complex_vectors, icosphere, capped_cylinder,
                       cube, mesh_signed_volume, fibonacci_directions)


@pytest.mark.parametrize("make,ntri,vol", [
    (lambda: icosphere(2, 0.2), 320, 4 / 3 * np.pi * 0.2**3),
    (lambda: capped_cylinder(0.15, 3.0), 1200, np.pi * 0.15**2 * 3.0),
    (lambda: cube(0.3), 432, 0.027),
])
def test_meshes_closed_outward_and_sized(make, ntri, vol):
    v, t = make()
    assert t.shape == (ntri, 3)
    edges = {}
    for a, b, c in t:
        for x, y in ((a, b), (b, c), (c, a)):
            edges[(x, y)] = edges.get((x, y), 0) + 1
    assert all(n == 1 and edges.get((y, x)) == 1 for (x, y), n in edges.items())
    sv = mesh_signed_volume(v, t)
    assert 0.9 * vol < sv <= 1.0001 * vol


def test_pcg32_reference_stream_and_vectors():
    # first outputs of O'Neill's pcg32 demo: seed 42, stream 54
    g = PCG32(42, 54)
    assert [g.next_u32() for _ in range(6)] == [0xa15c02b7, 0x7b47f409, 0xba1d3330,
                                                  0x83d2f293, 0xbfa4784b, 0xcbed606e]
    a = random_complex_vectors(5, 2, 300)
    b = random_complex_vectors(5, 2, 300)
    assert np.array_equal(a, b) and a.shape == (2, 300)
    assert np.all(np.abs(a.real) <= 1) and np.all(np.abs(a.imag) <= 1)
    big = random_complex_vectors(5, 1, 100000)
    assert abs(big.real.mean()) < 0.01 and abs(big.imag.var() - 1 / 3) < 0.01


def test_workload_sizes():
    sizes = {"sphere_row_4": 1280, "sonic_crystal_3x20": 72000,
             "sphere_array_32x32": 327680, "cube_lattice_16x16x4": 442368,
             "barrier_cylinders_3x25x5": 126000, "sphere_array_5x10_fine": 256000}
    for name, N in sizes.items():
        w = WORKLOADS[name]
        v, t = w.mesh()
        assert len(t) * int(np.prod(w.counts)) == N
    # the barrier's open cylinder segments: normals radially outward, cells
    # stacked without gaps from the ground plane z = -0.2 upwards
    w = WORKLOADS["barrier_cylinders_3x25x5"]
    v, t = w.mesh()
    tri = v[t]
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    cen = tri.mean(axis=1)
    assert (np.einsum("ij,ij->i", nrm[:, :2], cen[:, :2]) > 0).all()
    assert v[:, 2].min() == w.plane[1] and v[:, 2].max() - v[:, 2].min() == w.lattice[2, 2]
    d = fibonacci_directions(64)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0) and abs(d.mean(0)).max() < 0.05
