"""The FMPBEM2 host plan of the library (octree depth, interaction lists of
every near offset, exact entries kept, distinct M2L translations) against the
oracle's octree and lists, on the CPU: fmpb_near2_plan_counts does no device
work, so these run without a GPU."""
import numpy as np
import pytest

from oracle import bem, fmm2
from workloads import icosphere, cube

gb = pytest.importorskip("paper_2201_12050_gb300")


def _oracle_counts(v, t, counts, lattice, levels):
    cell = bem.CellMesh(v, t)
    tree = fmm2.Octree(cell, levels)
    L = np.asarray(lattice, dtype=float)
    n_m2l = n_p2p = 0
    translations = set()
    for d in bem.near_offsets(counts):
        m2l, p2p = fmm2.interaction_lists(tree, -np.asarray(d, dtype=float) @ L)
        n_m2l += len(m2l)
        for l, a, b in m2l:
            translations.add((l, a[0] - b[0], a[1] - b[1], a[2] - b[2], d))
        for a, b in p2p:
            n_p2p += len(tree.leaf_elements(a)) * len(tree.leaf_elements(b))
    return n_m2l, n_p2p, len(translations)


@pytest.mark.parametrize("mesh,counts,lattice,levels", [
    ("ico1", (4, 3, 1), np.diag([0.6, 0.6, 1.0]), 1),
    ("ico1", (4, 3, 1), np.diag([0.6, 0.6, 1.0]), 2),
    ("ico2", (3, 2, 1), np.diag([0.5, 0.55, 1.0]), 3),
    ("cube", (2, 2, 2), np.diag([0.5, 0.5, 0.5]), 2),
    ("ico2", (5, 1, 1), np.diag([0.45, 1.0, 1.0]), 0),
])
def test_plan_counts_match_the_oracle_lists(mesh, counts, lattice, levels):
    v, t = {"ico1": lambda: icosphere(1, 0.2), "ico2": lambda: icosphere(2, 0.2),
            "cube": lambda: cube(0.3, 4)}[mesh]()
    lv, n_m2l, n_p2p, n_k = gb.near2_plan_counts(v, t, counts, lattice, near_levels=levels)
    if levels == 0:
        # the shallowest depth with at most 32 elements per leaf on average
        assert lv >= 1
        cell = bem.CellMesh(v, t)
        assert len(t) / len(fmm2.Octree(cell, lv).boxes[lv]) <= 32.0
        if lv > 1:
            assert len(t) / len(fmm2.Octree(cell, lv - 1).boxes[lv - 1]) > 32.0
    else:
        assert lv == levels
    assert (n_m2l, n_p2p, n_k) == _oracle_counts(v, t, counts, lattice, lv)


def test_single_element_cell_is_one_box_per_level():
    v = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.0, 0.1, 0.0]])
    t = np.array([[0, 1, 2]], dtype=np.int32)
    lv, n_m2l, n_p2p, n_k = gb.near2_plan_counts(v, t, (3, 1, 1), np.diag([0.5, 1.0, 1.0]), near_levels=2)
    assert lv == 2 and (n_m2l, n_p2p, n_k) == _oracle_counts(v, t, (3, 1, 1), np.diag([0.5, 1.0, 1.0]), 2)


def test_plan_rejects_bad_arguments():
    v, t = icosphere(0, 0.2)
    with pytest.raises(gb.FmpbError):
        gb.near2_plan_counts(v, t, (2, 1, 1), np.diag([0.5, 1.0, 1.0]), near_levels=11)
    with pytest.raises(gb.FmpbError):
        gb.near2_plan_counts(v, t, (2, 1, 1), np.diag([0.5, 1.0, 1.0]), n_t_near=99)
    bad = np.array(t)
    bad[0, 0] = 1000
    with pytest.raises(gb.FmpbError):
        gb.near2_plan_counts(v, bad, (2, 1, 1), np.diag([0.5, 1.0, 1.0]))


@pytest.mark.parametrize("m,counts,lattice,levels", [
    (3, (4, 3, 1), np.diag([0.6, 0.6, 1.0]), 2),
    (3, (3, 2, 1), np.diag([0.5, 0.55, 1.0]), 3),
    (4, (2, 2, 2), np.diag([0.5, 0.5, 0.5]), 2),
])
def test_plan_on_nine_node_elements_matches_the_oracle_lists(m, counts, lattice, levels):
    # the octree of the element centres with box radii over all nine nodes
    from oracle import quad9
    from workloads import quad9_sphere
    nodes, el = quad9_sphere(m, 0.2)
    cell = quad9._Fmm2Cell(quad9.Q9Mesh(nodes, el))
    tree = fmm2.Octree(cell, levels)
    L = np.asarray(lattice, dtype=float)
    n_m2l = n_p2p = 0
    for d in bem.near_offsets(counts):
        m2l, p2p = fmm2.interaction_lists(tree, -np.asarray(d, dtype=float) @ L)
        n_m2l += len(m2l)
        n_p2p += sum(len(tree.leaf_elements(a)) * len(tree.leaf_elements(b)) for a, b in p2p)
    lv, got_m2l, got_p2p, _ = gb.near2_plan_counts(nodes, el, counts, lattice, near_levels=levels)
    assert (lv, got_m2l, got_p2p) == (levels, n_m2l, n_p2p)
