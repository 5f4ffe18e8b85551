"""Pins against the counts the paper prints (tests/golden/paper_storage_counts.txt).

* The oracle's offset sets hold as many blocks as the storage formulas of
  Sec. 2.2 (PBEM), Sec. 2.3 (half space) and Sec. 3.2-3.3 (near field of the
  FMM form) state, for the paper's own grids.
* Brute force on a tiny grid: dense matrices assembled pair by pair have
  exactly that many distinct cell blocks.  In free space the blocks depend
  only on the cell offset (block Toeplitz, Sec. 2.2); with a mirror plane
  perpendicular to a lattice axis (the paper's symmetry plane, Sec. 2.3) the
  image part adds as many distinct blocks again (block Hankel along that
  axis).  A dropped offset or a wrong image shift changes the count.
* The sphere-array example of Sec. 4.1: 600 nine-node quadrilaterals per
  sphere, N_dof = 3000 M_y for M_x = 5.
"""
import os
import re

import numpy as np
import pytest

from oracle import bem, halfspace as hs
from workloads import WORKLOADS, icosphere, quad9_sphere

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_storage_counts.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, expr, _where = [s.strip() for s in line.split("|", 2)]
        out[name] = expr
    return out


def value(name, Mx=1, My=1):
    expr = _golden()[name]
    assert re.fullmatch(r"[0-9MxMy*()+\- ]+", expr), expr
    return eval(expr, {"__builtins__": {}}, {"Mx": Mx, "My": My})


def _distinct_blocks(A, n, tol=1e-10):
    """Number of distinct n x n cell blocks of A (equal within tol of the
    larger block's largest entry)."""
    reps = []
    nb = A.shape[0] // n
    for a in range(nb):
        for b in range(nb):
            blk = A[a * n:(a + 1) * n, b * n:(b + 1) * n]
            if not any(np.abs(blk - r).max() <= tol * max(np.abs(r).max(), np.abs(blk).max()) for r in reps):
                reps.append(blk)
    return len(reps)


# the paper's grids: the sphere array (M_x = 5, M_y = 5 ... 100) and the
# sonic crystal of the headline workload
GRIDS = [(5, 5), (5, 10), (5, 100), (3, 20), (2, 3)]


@pytest.mark.parametrize("Mx,My", GRIDS)
def test_offset_sets_hold_the_printed_number_of_blocks(Mx, My):
    counts = (Mx, My, 1)
    assert len(bem.all_offsets(counts)) == value("pbem_blocks", Mx, My)
    assert len(bem.all_offsets(counts)) + len(hs.image_offsets(counts)) == value("halfspace_blocks", Mx, My)
    near = bem.near_offsets(counts)
    assert len(near) == value("near_blocks")
    assert len({d[1] for d in near}) == value("near_rows")


def test_dense_free_space_matrix_has_the_printed_number_of_distinct_blocks():
    v, t = icosphere(0, 0.2)
    counts, L = (2, 3, 1), np.diag([0.5, 0.55, 1.0])
    A = bem.dense_matrix(v, t, L, counts, 3.5)
    assert _distinct_blocks(A, len(t)) == value("pbem_blocks", 2, 3)


def test_dense_half_space_matrix_stores_twice_the_blocks():
    # mirror plane y = -0.26 perpendicular to the second lattice axis (the
    # paper's xz symmetry plane): the image part is block Hankel along y
    v, t = icosphere(0, 0.2)
    counts, L = (2, 3, 1), np.diag([0.5, 0.55, 1.0])
    pl = hs.Plane(1, -0.26, 1.0)
    assert hs.hankel_axis(L, counts, pl) == 1
    k = 3.5
    A = bem.dense_matrix(v, t, L, counts, k)
    Ah = hs.dense_matrix_halfspace(v, t, L, counts, k, pl) - A
    n = len(t)
    assert _distinct_blocks(Ah, n) == value("pbem_blocks", 2, 3)
    assert _distinct_blocks(A, n) + _distinct_blocks(Ah, n) == value("halfspace_blocks", 2, 3)


def test_sphere_array_discretisation_matches_the_example():
    nodes, el = quad9_sphere(10, 0.1)
    assert len(el) == value("sphere_elements")
    for My in (5, 10, 100):
        assert 5 * My * len(el) == value("array_dofs", 5, My)
    w = WORKLOADS["sphere_array_5x5_q9"]
    assert w.counts[0] == 5 and int(np.prod(w.counts)) * len(el) == value("array_dofs", 5, w.counts[1])
    assert int(np.prod(w.counts)) * len(el) == value("array_5x5_dofs")
    # elements with an edge on the equator z = 0, from above: one ring around
    # the sphere (the cube-sphere's equator is a grid line for an even m)
    zmin = np.array([nodes[e, 2].min() for e in el])
    ring = np.sum(np.abs(zmin) < 1e-12)
    assert ring == value("sphere_circumference")
    assert np.allclose(np.linalg.norm(nodes, axis=1), 0.1)
