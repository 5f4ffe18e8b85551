"""The truncation rule of the library (n_t = 0: the smallest n_t >= 4 whose
U_0 K(d) V_0 reproduces the exact block of the nearest far cell on four
probe vectors to 1e-6; Sec. 3.1's "sufficiently large" n_t, grown with
frequency as in the accuracy study of Sec. 4) against the oracle's
computation of the same criterion, through the C ABI.  Both sides build
their blocks and tables in FP64 and agree on them to about 1e-12; the
chosen n_t's probe errors in these cases lie 20 % or more below the 1e-6
threshold and the previous n_t's well above it."""
import numpy as np
import pytest
import torch

from oracle import bem, fmm
from workloads import cube, icosphere, random_complex_vectors

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")


@pytest.mark.parametrize("mesh,counts,L,k,beta", [
    ("sphere1", (4, 4, 1), np.diag([0.6, 0.6, 1.0]), 4.0, 0.0),
    ("sphere1", (4, 3, 1), np.diag([0.6, 0.6, 1.0]), 12.0, 0.3 + 0.2j),
    ("sphere2", (5, 1, 1), np.diag([0.5, 1.0, 1.0]), 2.0, 0.0),
    ("cube", (3, 3, 3), np.diag([0.5, 0.5, 0.5]), 2 * np.pi * 800 / 343.0, 0.0),   # 108 triangles
])
def test_truncation_rule_matches_oracle(mesh, counts, L, k, beta):
    if mesh == "cube":
        v, t = cube(0.3, 3)
    else:
        v, t = icosphere(1 if mesh == "sphere1" else 2, 0.2)
    cell = bem.CellMesh(v, t)
    d, errs = fmm.truncation_errors(cell, L, counts, k, beta, nt_max=14)
    ref = next(n for n in range(4, 15) if errs[n] <= 1e-6)
    op = gb.Operator(v, t, counts, L, k, form=gb.FORM_FMM, beta=beta)
    assert op.info["n_t"] == ref, (op.info["n_t"], ref, errs)
    # the probe error is a difference of O(1) products near 1e-6: the two
    # sides' 1e-12 agreement of blocks and tables leaves about 1e-6 of it
    assert abs(op.info["n_t_rule_err"] - errs[ref]) <= 1e-3 * errs[ref]
    # the operator at that n_t is the oracle's explicit FMPBEM product
    x = random_complex_vectors(81, 1, op.N)
    y = op.matvec(torch.as_tensor(x, device="cuda")).cpu().numpy()
    y_ref = fmm.fmm_matvec_explicit(cell, L, counts, k, ref, x, beta=beta)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-12


def test_truncation_rule_without_far_cells_and_when_it_cannot_be_met():
    v, t = icosphere(1, 0.2)
    op = gb.Operator(v, t, (2, 2, 1), np.diag([0.6, 0.6, 1.0]), 4.0, form=gb.FORM_FMM)
    assert op.info["n_t"] == 4 and op.info["n_t_rule_err"] == 0.0
    # a given n_t is kept, and reports no rule error
    op = gb.Operator(v, t, (4, 4, 1), np.diag([0.6, 0.6, 1.0]), 4.0, form=gb.FORM_FMM, n_t=7)
    assert op.info["n_t"] == 7 and op.info["n_t_rule_err"] == -1.0
    # far above the cell's resolution no n_t up to 20 reaches 1e-6: AUTO
    # falls back to the exact PBEM form, a forced FMM form keeps n_t = 20
    auto = gb.Operator(v, t, (4, 1, 1), np.diag([0.6, 1.0, 1.0]), 90.0)
    assert auto.info["form_name"] == "pbem"
    forced = gb.Operator(v, t, (4, 1, 1), np.diag([0.6, 1.0, 1.0]), 90.0, form=gb.FORM_FMM)
    assert forced.info["n_t"] == 20 and forced.info["n_t_rule_err"] > 1e-6
