"""The half-space host plan of the library (perpendicular lattice axis,
mirrored cells evaluated exactly, nearest far mirrored cell) against the
oracle, on the CPU: fmpb_halfspace_plan does no device work."""
import numpy as np
import pytest

from oracle import halfspace as hs
from workloads import WORKLOADS, icosphere

gb = pytest.importorskip("paper_2201_12050_gb300")

CASES = [
    ((3, 2, 1), np.diag([0.5, 0.5, 1.0]), (2, -0.3)),
    ((2, 1, 3), np.diag([0.5, 1.0, 0.55]), (2, -0.26)),
    ((3, 2, 1), np.diag([-0.5, 0.45, 1.0]), (0, 0.27)),
    ((3, 1, 4), np.diag([0.7, 1.0, 0.7]), (2, -0.45)),
]


@pytest.mark.parametrize("counts,lattice,plane", CASES)
def test_plan_matches_the_oracle(counts, lattice, plane):
    v, t = icosphere(1, 0.2)
    h, n_near, dmin = gb.halfspace_plan(v, t, counts, lattice, *plane)
    pl = hs.Plane(plane[0], plane[1], 1.0)
    assert h == hs.hankel_axis(lattice, counts, pl)
    near = hs.image_near_offsets(lattice, counts, pl)
    assert n_near == len(near)
    far = [np.linalg.norm(hs.image_shift(lattice, counts, pl, d)) for d in hs.image_offsets(counts) if d not in near]
    assert (not far and dmin == 1e300) or abs(dmin - min(far)) <= 1e-12 * min(far)


def test_barrier_workload_plan():
    w = WORKLOADS["barrier_cylinders_3x25x5"]
    v, t = w.mesh()
    h, n_near, dmin = gb.halfspace_plan(v, t, w.counts, w.lattice, w.plane[0], w.plane[1])
    assert h == 2 and n_near == 9 and abs(dmin - 0.8) < 1e-12


def test_plan_rejects_oblique_lattices_and_crossing_cells():
    v, t = icosphere(0, 0.2)
    with pytest.raises(gb.FmpbError):
        gb.halfspace_plan(v, t, (2, 2, 1), np.array([[0.5, 0, 0.1], [0, 0.5, 0], [0, 0, 1.0]]), 2, -0.3)
    with pytest.raises(gb.FmpbError):
        gb.halfspace_plan(v, t, (2, 1, 1), np.diag([0.5, 1.0, 1.0]), 2, 0.1)
    with pytest.raises(gb.FmpbError):
        gb.halfspace_plan(v, t, (1, 1, 3), np.diag([1.0, 1.0, -0.5]), 2, -0.3)
    with pytest.raises(gb.FmpbError):
        gb.halfspace_plan(v, t, (2, 1, 1), np.diag([0.5, 1.0, 1.0]), 3, -0.3)


@pytest.mark.parametrize("counts,lattice,plane", CASES[:2])
def test_plan_on_nine_node_elements(counts, lattice, plane):
    # the same plan from a quadrilateral cell, and the one-side check read from
    # its element centres and nodes: a plane through the spheres is refused
    from workloads import quad9_sphere
    nodes, el = quad9_sphere(2, 0.2)
    h, n_near, dmin = gb.halfspace_plan(nodes, el, counts, lattice, *plane)
    pl = hs.Plane(plane[0], plane[1], 1.0)
    assert h == hs.hankel_axis(lattice, counts, pl)
    assert n_near == len(hs.image_near_offsets(lattice, counts, pl))
    with pytest.raises(gb.FmpbError, match="EMESH"):
        gb.halfspace_plan(nodes, el, counts, lattice, plane[0], 0.05)
