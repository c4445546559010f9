"""Oracle: exact solution of A u = f by block forward substitution (time stepping).

A is block lower triangular (eq. amatdef), so u^n = A_(0)^{-1} (f^n - sum_{k=1}^{n} A_(k) u^{n-k}),
n = 0..N-1, with A_(0) = a_0 I + b_0 L factorised once by a sparse LU.  This is the textbook
special case the iterative solution must reproduce (to within tol times a conditioning factor).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import splu

from .operators import laplacian


def timestep_solve(prob, f: np.ndarray) -> np.ndarray:
    N, M = prob.N, prob.M
    if prob.meta.get("blocks") is not None:
        # general blocks given as matrices: a dense LU of A_(0), the block sum as written
        from scipy.linalg import lu_factor, lu_solve
        B = np.asarray(prob.meta["blocks"], dtype=np.float64)
        lu0 = lu_factor(B[0])
        F = np.asarray(f, dtype=np.float64).reshape(N, M)
        U = np.zeros((N, M))
        for n in range(N):
            rhs = F[n] - sum((B[k] @ U[n - k] for k in range(1, n + 1)), np.zeros(M))
            U[n] = lu_solve(lu0, rhs)
        return U.reshape(-1)
    L = laplacian(prob)
    I = sp.identity(M, format="csc")
    A0 = (prob.a[0] * I + prob.b[0] * L).tocsc()
    lu = splu(A0)
    F = np.asarray(f, dtype=np.float64).reshape(N, M)
    U = np.zeros((N, M))
    for n in range(N):
        rhs = F[n].copy()
        acc_a = np.zeros(M)
        acc_b = np.zeros(M)
        for k in range(1, n + 1):
            if prob.a[k] != 0.0:
                acc_a += prob.a[k] * U[n - k]
            if prob.b[k] != 0.0:
                acc_b += prob.b[k] * U[n - k]
        rhs -= acc_a + L @ acc_b
        U[n] = lu.solve(rhs)
    return U.reshape(-1)
