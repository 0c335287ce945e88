"""Plain definitions of the solution of eq. (sylv), for small inputs.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A X + X B = -f g^* is the linear system (I_m kron A + B^T kron I_n) vec(X)
= -vec(f g^*) (column-major vec), uniquely solvable when Lambda(A) and
Lambda(-B) are disjoint (Sec. 2).  Bartels-Stewart (scipy.linalg
.solve_sylvester, a library routine) solves the same equation through Schur
forms.  The generalized equation A X C + M X B = -f g^* (eq. (gsylv)) is
(C^T kron A + B^T kron M) vec(X) = -vec(f g^*); multiplied by M^{-1} from the
left and C^{-1} from the right it is the standard equation
M^{-1} A X + X B C^{-1} = -M^{-1} f g^* C^{-1}, which Bartels-Stewart solves.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _dense(M):
    return M.toarray() if hasattr(M, "toarray") else np.asarray(M)


def kron_solve(A, B, f, g, M=None, C=None) -> np.ndarray:
    """X from the n*m x n*m Kronecker system (use for n*m <= a few thousand)."""
    A, B = _dense(A), _dense(B)
    n, m = A.shape[0], B.shape[0]
    Md = np.eye(n) if M is None else _dense(M)
    Cd = np.eye(m) if C is None else _dense(C)
    K = np.kron(Cd.T, A) + np.kron(B.T, Md)
    rhs = -(f @ g.conj().T).reshape(-1, order="F")
    return np.linalg.solve(K, rhs).reshape((n, m), order="F")


def bartels_stewart(A, B, f, g, M=None, C=None) -> np.ndarray:
    """X from scipy.linalg.solve_sylvester(A, B, -f g^*), for the generalized
    equation after multiplying by M^{-1} and C^{-1}."""
    A, B = _dense(A), _dense(B)
    rhs = -(f @ g.conj().T)
    if M is not None:
        Md = _dense(M)
        A, rhs = np.linalg.solve(Md, A), np.linalg.solve(Md, rhs)
    if C is not None:
        Ci = np.linalg.inv(_dense(C))
        B, rhs = B @ Ci, rhs @ Ci
    return sla.solve_sylvester(A, B, rhs)


def dense_residual(A, B, f, g, X, M=None, C=None) -> np.ndarray:
    A, B = _dense(A), _dense(B)
    AX = A @ X if C is None else A @ X @ _dense(C)
    XB = X @ B if M is None else _dense(M) @ X @ B
    return AX + XB + f @ g.conj().T
