"""Plain definitions of the solution of eq. (sylv), for small inputs.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A X + X B = -f g^* is the linear system (I_m kron A + B^T kron I_n) vec(X)
= -vec(f g^*) (column-major vec), uniquely solvable when Lambda(A) and
Lambda(-B) are disjoint (Sec. 2).  Bartels-Stewart (scipy.linalg
.solve_sylvester, a library routine) solves the same equation through Schur
forms.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _dense(M):
    return M.toarray() if hasattr(M, "toarray") else np.asarray(M)


def kron_solve(A, B, f, g) -> np.ndarray:
    """X from the n*m x n*m Kronecker system (use for n*m <= a few thousand)."""
    A, B = _dense(A), _dense(B)
    n, m = A.shape[0], B.shape[0]
    K = np.kron(np.eye(m), A) + np.kron(B.T, np.eye(n))
    rhs = -(f @ g.conj().T).reshape(-1, order="F")
    return np.linalg.solve(K, rhs).reshape((n, m), order="F")


def bartels_stewart(A, B, f, g) -> np.ndarray:
    """X from scipy.linalg.solve_sylvester(A, B, -f g^*)."""
    return sla.solve_sylvester(_dense(A), _dense(B), -(f @ g.conj().T))


def dense_residual(A, B, f, g, X) -> np.ndarray:
    A, B = _dense(A), _dense(B)
    return A @ X + X @ B + f @ g.conj().T
