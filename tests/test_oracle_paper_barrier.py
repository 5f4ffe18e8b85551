"""Pins against the values the paper prints for its sound barrier study
(Sec. 4.2; tests/golden/paper_barrier_example.txt).

* The cylinder barrier workload has the printed grid, spacing, footprint,
  height and dof count, and its stand-in cell (flat triangles, constant
  pressure) has as many dofs as the paper's cell of 12 x 7 linear-pressure
  quadrilaterals.
* The first Bragg frequency n c / (2 d sin theta) of the printed spacing is the
  printed 428.75 Hz with the speed of sound of the inputs, and the workload
  solves at that frequency.
* The monopoles sit where the paper puts them, with its source strengths.
* The dof counts of the wall models fix the discontinuous quadratic pressure
  of the oracle's quadrilaterals at eight nodes per element (serendipity):
  4140 elements give the printed 33120 dofs, and 500 cells of two layers of
  four elements the printed 32000; linear pressure has four.
"""
import os

import numpy as np

from oracle.quad9_order import PressureBasis
from workloads import SPEED_OF_SOUND, WORKLOADS

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_barrier_example.txt")


def printed():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, val, _what = [s.strip() for s in line.split("|", 2)]
        vals = [float(x) for x in val.split(",")]
        out[name] = vals[0] if len(vals) == 1 else vals
    return out


def test_cylinder_barrier_workload_matches_the_printed_geometry():
    g = printed()
    w = WORKLOADS["barrier_cylinders_3x25x5"]
    assert list(w.counts) == g["cylinder_cells"]
    L = np.asarray(w.lattice)
    d = g["cylinder_spacing_m"]
    assert np.allclose(np.diag(L)[:2], d) and np.allclose(L - np.diag(np.diag(L)), 0.0)
    v, t = w.mesh()
    r = np.max(np.hypot(v[:, 0], v[:, 1]))
    assert np.isclose(r, g["cylinder_radius_m"])
    h_cell = np.ptp(v[:, 2])
    assert np.isclose(h_cell * w.counts[2], g["cylinder_height_m"]) and np.isclose(L[2, 2], h_cell)
    footprint = [(w.counts[1] - 1) * d + 2 * r, (w.counts[0] - 1) * d + 2 * r]
    assert np.allclose(footprint, g["cylinder_footprint_m"])
    cells = int(np.prod(w.counts))
    assert cells * len(t) == g["cylinder_dofs"]
    # the paper's cell: 12 linear-pressure elements around, 35 / M_z along the height
    per_cell_paper = (g["cylinder_elements_around"] * g["cylinder_elements_height"] / w.counts[2]
                      * PressureBasis(1).nb)
    assert len(t) == per_cell_paper


def test_first_bragg_frequency_is_the_printed_value_and_is_solved():
    g = printed()
    f = 1 * SPEED_OF_SOUND / (2 * g["cylinder_spacing_m"] * np.sin(np.pi / 2))
    assert np.isclose(f, g["bragg_hz"], rtol=0, atol=1e-9)
    w = WORKLOADS["barrier_cylinders_3x25x5"]
    assert np.isclose(np.asarray(w.wavenumbers), 2 * np.pi * g["bragg_hz"] / SPEED_OF_SOUND).any()


def test_monopoles_are_placed_as_printed():
    g = printed()
    w = WORKLOADS["barrier_cylinders_3x25x5"]
    axis, offset, Rp = w.plane
    assert axis == 2 and Rp == 1.0                      # sound-hard ground
    (x1, a1), (x2, a2) = w.monopoles
    assert [x1[1], x2[1]] == g["monopole_y_m"] and [a1, a2] == g["monopole_amplitude_pa"]
    assert np.isclose(x1[2] - offset, g["monopole_height_m"]) and np.isclose(x2[2] - offset, g["monopole_height_m"])


def test_wall_dof_counts_fix_quadratic_pressure_at_eight_nodes():
    g = printed()
    nb2 = PressureBasis(2).nb
    assert g["wall_elements"] * nb2 == g["wall_dofs"]
    assert g["wall_cells"] * g["wall_cell_elements"] * nb2 == g["wall_periodic_dofs"]
    # nine nodes (a Lagrange biquadratic) would not give the printed counts
    assert g["wall_elements"] * 9 != g["wall_dofs"]
    assert PressureBasis(1).nb == 4 and PressureBasis(0).nb == 1
