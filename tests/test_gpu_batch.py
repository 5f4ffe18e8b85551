"""fmpb_solve_batch: the systems of several operators (one lattice at several
frequencies) in one GMRES, through the C ABI.  Each system keeps its own
Krylov basis and convergence test, and the batched products of operators of
one shape are their single products (tensor-core columns and DFT lines are
independent), up to the plan the DFT-pass autotuner picks for the batch's
longer lines (FP32 passes: another split rounds differently, about 1e-7,
and the BF16 rounding of the next product's input turns that into about
1e-5).  So a few iterations of the batched solve equal those of single
solves to 1e-4.  Converged solves agree to the tolerance's reach: BF16 operators
round every product's input vector to BF16, which makes the product
slightly nonlinear and lets iterates that differ in the last bits drift
apart at that rounding level, so their solves (to 1e-3) are only checked
for convergence and residual; MIXED (outer residuals in float-float) and
FP64 solves to 1e-10 agree within 1e-7 and 1e-8."""
import numpy as np
import pytest
import torch

from workloads import fibonacci_directions, icosphere

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")

COUNTS, LATTICE = (4, 3, 1), np.diag([0.6, 0.6, 1.0])


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _batch_vs_solo(ops, dirs, tol, restart=30, maxit=1000, exact_iters=True):
    bs = torch.stack([op.rhs_plane_wave(dirs) for op in ops])
    p, info = gb.solve_batch(ops, bs, tol=tol, restart=restart, maxit=maxit, raise_on_noconv=False)
    for o, op in enumerate(ops):
        ps, infos = op.solve(bs[o].clone(), tol=tol, restart=restart, maxit=maxit, raise_on_noconv=False)
        for r in range(len(dirs)):
            assert info[o][r]["converged"] == infos[r]["converged"]
            if exact_iters:
                assert abs(info[o][r]["iters"] - infos[r]["iters"]) <= 1, (o, r, info[o][r], infos[r])
        yield o, _rel(p[o], ps), info[o]


def test_batched_tensor_core_products_equal_single_products():
    # three Arnoldi steps: the iterates depend on the products, which must be
    # the single products' (a product with another operator's tables would
    # differ at order one)
    v, t = icosphere(1, 0.2)
    ops = [gb.Operator(v, t, COUNTS, LATTICE, k, form=gb.FORM_FMM, n_t=6, precision=gb.BF16) for k in (2.0, 3.5, 5.0)]
    for o, err, _ in _batch_vs_solo(ops, fibonacci_directions(4), 1e-12, restart=3, maxit=3):
        assert err < 1e-4, (o, err)


def test_batched_bf16_solves_converge():
    v, t = icosphere(1, 0.2)
    ops = [gb.Operator(v, t, COUNTS, LATTICE, k, form=gb.FORM_FMM, n_t=6, precision=gb.BF16) for k in (2.0, 3.5, 5.0)]
    bs = torch.stack([op.rhs_plane_wave(fibonacci_directions(4)) for op in ops])
    p, info = gb.solve_batch(ops, bs, tol=1e-3)
    y64 = [gb.Operator(v, t, COUNTS, LATTICE, k, form=gb.FORM_FMM, n_t=6) for k in (2.0, 3.5, 5.0)]
    for o in range(3):
        # converged on the GMRES estimate; the recomputed residual of a BF16
        # operator sits at its input-rounding level (a few 1e-3)
        assert all(i["converged"] and i["relres_true"] < 2e-2 for i in info[o])
        # against the FP64 operator the BF16 solution leaves a residual at the BF16 rounding level
        assert _rel(y64[o].matvec(p[o]), bs[o]) < 2e-2


def test_batched_mixed_solves_equal_single_solves():
    v, t = icosphere(1, 0.2)
    ops = [gb.Operator(v, t, COUNTS, LATTICE, k, form=gb.FORM_FMM, n_t=6, precision=gb.MIXED) for k in (2.0, 3.5, 5.0)]
    for o, err, info in _batch_vs_solo(ops, fibonacci_directions(4), 1e-10, exact_iters=False):
        assert all(i["converged"] for i in info)
        assert err < 1e-7, (o, err)


def test_batched_pbem_solves_equal_single_solves():
    # operators without a fused product: each applies its own within the
    # shared iteration (float-float products of the PBEM form)
    v, t = icosphere(1, 0.2)
    ops = [gb.Operator(v, t, (3, 2, 1), np.diag([0.5, 0.5, 1.0]), k, form=gb.FORM_PBEM) for k in (2.0, 4.0)]
    for o, err, info in _batch_vs_solo(ops, [[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]], 1e-10):
        assert all(i["converged"] for i in info)
        assert err < 1e-8, (o, err)


def test_batch_argument_errors():
    v, t = icosphere(1, 0.2)
    a = gb.Operator(v, t, COUNTS, LATTICE, 2.0, form=gb.FORM_FMM, n_t=6, precision=gb.BF16)
    b = gb.Operator(v, t, (3, 3, 1), LATTICE, 2.0, form=gb.FORM_FMM, n_t=6, precision=gb.BF16)
    m = gb.Operator(v, t, COUNTS, LATTICE, 2.0, form=gb.FORM_FMM, n_t=6, precision=gb.MIXED)
    rhs = torch.zeros((2, 1, a.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(gb.FmpbError):
        gb.solve_batch([a, m], rhs)                      # MIXED beside BF16
    with pytest.raises(gb.FmpbError):
        gb.solve_batch([a, b], rhs)                      # another size (refused by the library)
    with pytest.raises(ValueError):
        gb.solve_batch([a, a], rhs[:, :, :-1].contiguous())   # right-hand sides of the wrong length
