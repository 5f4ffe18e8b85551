"""fmpb_solve_batch: the systems of several operators (one lattice at several
frequencies) in one GMRES, through the C ABI.  Each system keeps its own
Krylov basis and convergence test, and the batched products of operators of
one shape are the same arithmetic as their single products (tensor-core
columns and DFT lines are independent), so each result must equal its own
fmpb_solve up to the rounding of the Gram-Schmidt reductions, whose
partitioning depends on the number of systems: within 1e-6 relative here
(BF16 solves to 1e-5; FP64 and MIXED to 1e-10, within 1e-8)."""
import numpy as np
import pytest
import torch

from workloads import fibonacci_directions, icosphere

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")

COUNTS, LATTICE = (4, 3, 1), np.diag([0.6, 0.6, 1.0])


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _batch_vs_solo(ops, dirs, tol, restart=30):
    bs = torch.stack([op.rhs_plane_wave(dirs) for op in ops])
    p, info = gb.solve_batch(ops, bs, tol=tol, restart=restart)
    for o, op in enumerate(ops):
        ps, infos = op.solve(bs[o].clone(), tol=tol, restart=restart)
        for r in range(len(dirs)):
            assert info[o][r]["converged"] and infos[r]["converged"]
            assert abs(info[o][r]["iters"] - infos[r]["iters"]) <= 1, (o, r, info[o][r], infos[r])
        yield o, _rel(p[o], ps)


@pytest.mark.parametrize("precision,tol,bound", [("BF16", 1e-5, 1e-6), ("MIXED", 1e-10, 1e-8)])
def test_batched_tensor_core_solves_equal_single_solves(precision, tol, bound):
    v, t = icosphere(1, 0.2)
    ops = [gb.Operator(v, t, COUNTS, LATTICE, k, form=gb.FORM_FMM, n_t=6, precision=getattr(gb, precision))
           for k in (2.0, 3.5, 5.0)]
    dirs = fibonacci_directions(4)
    for o, err in _batch_vs_solo(ops, dirs, tol):
        assert err < bound, (o, err)


def test_batched_pbem_solves_equal_single_solves():
    # operators without a fused product: each applies its own within the
    # shared iteration (float-float products of the PBEM form)
    v, t = icosphere(1, 0.2)
    ops = [gb.Operator(v, t, (3, 2, 1), np.diag([0.5, 0.5, 1.0]), k, form=gb.FORM_PBEM) for k in (2.0, 4.0)]
    for o, err in _batch_vs_solo(ops, [[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]], 1e-10):
        assert err < 1e-8, (o, err)


def test_batch_argument_errors():
    v, t = icosphere(1, 0.2)
    a = gb.Operator(v, t, COUNTS, LATTICE, 2.0, form=gb.FORM_FMM, n_t=6, precision=gb.BF16)
    b = gb.Operator(v, t, (3, 3, 1), LATTICE, 2.0, form=gb.FORM_FMM, n_t=6, precision=gb.BF16)
    m = gb.Operator(v, t, COUNTS, LATTICE, 2.0, form=gb.FORM_FMM, n_t=6, precision=gb.MIXED)
    rhs = torch.zeros((2, 1, a.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(gb.FmpbError):
        gb.solve_batch([a, m], rhs)                      # MIXED beside BF16
    with pytest.raises(ValueError):
        gb.solve_batch([a, b], rhs)                      # another size
