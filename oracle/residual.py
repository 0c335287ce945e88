"""Norms through low-rank factors.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ||w t^*||_2, the computed residual norm of eq. (adi_resexact), via thin QR
  of both factors (||Q_w R_w R_t^* Q_t^*|| = ||R_w R_t^*||).
* The true Sylvester residual of eq. (adi_res_inexact),
  R = A Z Gamma Y^* C + M Z Gamma Y^* B + f g^*  (M = C = I unless given),
  factored as U W^* with U = [A Z, M Z, f], W = [C^* Y Gamma^*, B^* Y Gamma^*, g];
  its exact 2-norm replaces the paper's a-posteriori eigs estimate (Sec. 4).
* Frobenius norm of the difference of two factored solutions.
"""
from __future__ import annotations

import numpy as np


def block_norm2(M: np.ndarray) -> float:
    """Spectral norm of a tall n x r block (largest singular value)."""
    if M.size == 0:
        return 0.0
    M = M.reshape(M.shape[0], -1)
    return float(np.linalg.norm(M, 2))


def lowrank_norm2(U: np.ndarray, W: np.ndarray) -> float:
    """||U W^*||_2 for tall U (n x p), W (m x p)."""
    _, Ru = np.linalg.qr(U)
    _, Rw = np.linalg.qr(W)
    return float(np.linalg.norm(Ru @ Rw.conj().T, 2))


def lowrank_fro(U: np.ndarray, W: np.ndarray) -> float:
    """||U W^*||_F for tall U, W."""
    _, Ru = np.linalg.qr(U)
    _, Rw = np.linalg.qr(W)
    return float(np.linalg.norm(Ru @ Rw.conj().T, "fro"))


def true_residual_norm2(A, B, f, g, Z, gamma, Y, M=None, C=None) -> float:
    """||A X C + M X B + f g^*||_2 for X = Z diag(gamma) Y^* (eq. adi_res_inexact;
    M = C = I when not given)."""
    Yg = Y * np.conj(gamma)[None, :]
    U = np.hstack([A @ Z, Z if M is None else M @ Z, f])
    W = np.hstack([Yg if C is None else C.conj().T @ Yg, B.conj().T @ Yg, g])
    return lowrank_norm2(U, W)


def sampled_residual(A, B, f, g, Z, gamma, Y, rows, cols) -> np.ndarray:
    """Entries R[rows][:, cols] of R = A X + X B + f g^* for X = Z diag(gamma) Y^*,
    evaluated exactly from the sparsity of A and B (for factors too large to
    form R): (A X)_ij uses X at the nonzero columns of row i of A, (X B)_ij
    uses X at the nonzero rows of column j of B."""
    A = A.tocsr()
    Bc = B.tocsc()
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    nr = np.unique(np.concatenate([A.indices[A.indptr[i]:A.indptr[i + 1]] for i in rows] + [rows]))
    nc = np.unique(np.concatenate([Bc.indices[Bc.indptr[j]:Bc.indptr[j + 1]] for j in cols] + [cols]))
    G = gamma[:, None] * Y[cols].conj().T            # kr x |cols|
    XA = Z[nr] @ G                                    # X[nr, cols]
    XB = Z[rows] @ (gamma[:, None] * Y[nc].conj().T)  # X[rows, nc]
    Ar = A[rows][:, nr]
    Bs = Bc[nc][:, cols]
    return Ar @ XA + XB @ Bs + f[rows] @ g[cols].conj().T


def factored_diff_fro(Z1, g1, Y1, Z2, g2, Y2) -> float:
    """||Z1 diag(g1) Y1^* - Z2 diag(g2) Y2^*||_F."""
    U = np.hstack([Z1 * g1[None, :], -Z2 * g2[None, :]])
    W = np.hstack([Y1, Y2])
    return lowrank_fro(U, W)


def factored_fro(Z, g, Y) -> float:
    return lowrank_fro(Z * g[None, :], Y)
