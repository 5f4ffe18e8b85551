"""Linear solves for the oracle (Sec. 4: GMRES with a relative tolerance).
Oracle code: test infrastructure only.

Dense systems use LAPACK through numpy (a library primitive); matrix-free
systems use scipy's GMRES (restart 30, x0 = 0, no preconditioner, relative
residual tolerance), the reading taken for the solver settings the paper
leaves open.
"""
import numpy as np
from scipy.sparse.linalg import LinearOperator, gmres


def dense_solve(A, b):
    return np.linalg.solve(A, b)


def gmres_solve(matvec, b, tol=1e-8, restart=30, maxiter=2000):
    n = b.shape[0]
    op = LinearOperator((n, n), matvec=matvec, dtype=complex)
    its = [0]

    def cb(_):
        its[0] += 1

    x, info = gmres(op, b, rtol=tol, atol=0.0, restart=restart, maxiter=maxiter,
                    callback=cb, callback_type="pr_norm")
    return x, info, its[0]
