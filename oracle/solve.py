"""Linear solves for the oracle (Sec. 4 solves the systems of Eqs.
(toeplitzBEM) and (FMPBEMsystem); the oracle's reference solutions are the
exact ones of the dense systems).
Oracle code: test infrastructure only.

Dense systems use LAPACK through numpy (a library primitive).
"""
import numpy as np


def dense_solve(A, b):
    return np.linalg.solve(A, b)
