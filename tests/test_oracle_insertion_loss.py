"""Pins of the oracle's insertion loss (Eq. (insertionloss)):

* the printed formula on a hand-made example (|p_inc| summing to twice
  |p| gives 20 log10 2 dB);
* with no surface response (p = 0 on the boundary) the total field is the
  incident field and the insertion loss is 0 dB exactly;
* scaling every source amplitude by the same factor leaves it unchanged.
"""
import numpy as np

from oracle import bem, halfspace as hs
from workloads import icosphere


def test_formula_on_a_hand_made_example():
    p_inc = np.array([1.0, -1.0j, 0.6 + 0.8j])
    p_tot = np.array([0.5, 0.5j, -0.3 - 0.4j])
    assert abs(hs.insertion_loss_from_fields(p_inc, p_tot) - 20 * np.log10(2.0)) < 1e-14


def test_zero_surface_pressure_gives_zero_loss_and_scaling_invariance():
    v, t = icosphere(0, 0.2)
    counts, L = (2, 1, 2), np.diag([0.5, 1.0, 0.55])
    pl = hs.Plane(2, -0.26, 1.0)
    k = 2.0
    pts = np.array([[1.5, 0.2, 0.3], [2.0, -0.4, 0.6], [2.5, 0.1, 0.1]])
    inc = [("monopole", [-2.0, 0.5, 0.4], 2.0), ("monopole", [-2.0, -0.5, 0.4], 1.0)]
    N = len(t) * 4
    P0 = np.zeros((2, N), dtype=complex)
    assert abs(hs.insertion_loss(v, t, L, counts, k, P0, pts, inc, pl)) < 1e-14
    rng = np.random.default_rng(6)
    P = rng.normal(size=(2, N)) + 1j * rng.normal(size=(2, N))
    il = hs.insertion_loss(v, t, L, counts, k, P, pts, inc, pl)
    inc3 = [(kd, vec, 3.0 * a) for kd, vec, a in inc]
    assert abs(hs.insertion_loss(v, t, L, counts, k, 3.0 * P, pts, inc3, pl) - il) < 1e-12
