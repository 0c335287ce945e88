"""Restarted GMRES(m) with right Jacobi preconditioning for shifted systems.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Solves (Op + sigma I) x = b for one column b, the inner systems of
Algorithm 1: (A + beta_k I) z = w_{k-1}(:, l) and (B^T + conj(alpha_k) I)
y = t_{k-1}(:, l); with a mass matrix, (Op + sigma Mass) x = b, the systems
(A + beta_k M) z = w_{k-1}(:, l) and (B + alpha_k C)^* y = t_{k-1}(:, l) of
the generalized equation (eq. (lradi_g), Algorithm 1).  The paper's guidance for the inner solver (Sec. 3.3,
"Further implementation aspects"):

* each of the r columns is solved separately, to ||r(:,l)|| <= delta_k / r;
* right preconditioning, so the Krylov residual estimate is the residual of
  the original system; the true residual is recomputed after termination and
  a new cycle starts if it is not yet below the tolerance.

The paper uses BiCGstab/MINRES in its experiments; restarted GMRES is the
textbook method of Saad and Schultz (1986) with Givens rotations for the
Hessenberg least-squares problem.  Orthogonalisation is modified
Gram-Schmidt, classical Gram-Schmidt applied twice (CGS2), or CGS2 with the
second pass delayed by one step (DCGS2, Swirydowicz, Langou, Ananthan, Yang
and Thomas, Numer. Linear Algebra Appl. 28 (2021); Bielich et al., Parallel
Comput. 112 (2022)); all are written out plainly below.  Initial guess
x0 = 0 (the paper is silent).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class GmresResult:
    x: np.ndarray           # approximate solution
    resnorm: float          # ||b - (Op + sigma I) x||_2, recomputed explicitly
    iters: int              # Arnoldi steps (operator applications inside cycles)
    cycles: int             # restart cycles run
    converged: bool
    history: list           # Givens residual estimates, one per Arnoldi step


def givens(a, b):
    """Rotation [[c, s], [-conj(s), c]] (c real) mapping (a, b) to (rho, 0)."""
    aa, ab = abs(a), abs(b)
    if ab == 0.0:
        return 1.0, 0.0 * a
    if aa == 0.0:
        return 0.0, np.conj(b) / ab
    rho = np.hypot(aa, ab)
    c = aa / rho
    s = (a / aa) * np.conj(b) / rho
    return c, s


def mgs_step(V, w):
    """Modified Gram-Schmidt of w against the rows of V: (h, w - V^T h)."""
    h = np.zeros(V.shape[0], dtype=np.result_type(V.dtype, w.dtype))
    for i in range(V.shape[0]):
        h[i] = np.vdot(V[i], w)
        w = w - h[i] * V[i]
    return h, w


def cgs2_step(V, w):
    """Classical Gram-Schmidt applied twice: h1 = V^* w, w1 = w - V h1,
    h2 = V^* w1, w2 = w1 - V h2; returns (h1 + h2, w2).  V holds the
    orthonormal vectors as rows."""
    h1 = V.conj() @ w
    w = w - V.T @ h1
    h2 = V.conj() @ w
    w = w - V.T @ h2
    return h1 + h2, w


def arnoldi_dcgs2(apply, v0, k):
    """k Arnoldi steps with delayed reorthogonalisation, starting from the
    unit vector v0; returns (V, H) with V (k+1) x n orthonormal rows and H
    the (k+1) x k Hessenberg matrix of apply(V[:k].T) = V.T @ H, plus the
    number of operator applications.

    Step j works on u_j, the once-orthogonalised candidate for v_j (u_0 = v0):
      y = apply(u_j)                         (the product of step j)
      s = V_<j^* u_j,  alpha = u_j^* u_j      (the delayed second pass)
      z = V_<j^* y,    gamma = u_j^* y        (first pass of the next column)
      beta = sqrt(alpha - |s|^2)              (norm of u_j - V_<j s)
      column j-1 of H = (first-pass coefficients) + s, H[j, j-1] = beta
      v_j = (u_j - V_<j s) / beta
      u_{j+1} = (y - V_<j z - v_j (v_j^* y)) / beta,  v_j^* y = (gamma - s^* z) / beta
    and the first-pass coefficients of column j are V_<=j^* A v_j, which
    follow from z, gamma, s and the columns of H so far because
    A V_<j = V_<=j H (no further product):
      h1 = ([z; v_j^* y] - H[:j+1, :j] s) / beta.
    A product is skipped at the last step (its result is never used)."""
    n = v0.shape[0]
    dtype = v0.dtype
    V = np.zeros((k + 1, n), dtype)
    H = np.zeros((k + 1, k), dtype)
    u = v0.copy()
    h1 = None
    napply = 0
    for j in range(k + 1):
        y = apply(u) if j < k else None
        napply += y is not None
        s = V[:j].conj() @ u
        alpha = np.vdot(u, u).real
        beta = np.sqrt(max(alpha - np.vdot(s, s).real, 0.0))
        if j >= 1:
            H[:j, j - 1] = h1 + s
            H[j, j - 1] = beta
        if beta == 0.0:
            return V[:j], H[:j, :max(j - 1, 0)], napply
        V[j] = (u - V[:j].T @ s) / beta
        if j == k:
            break
        z = V[:j].conj() @ y
        gamma = np.vdot(u, y)
        vy = (gamma - np.vdot(s, z)) / beta
        h1 = (np.concatenate([z, [vy]]) - H[:j + 1, :j] @ s) / beta
        u = (y - V[:j].T @ z - V[j] * vy) / beta
    return V, H, napply


def shifted_apply(S, sigma, x, mass=None):
    """(Op + sigma I) x, or (Op + sigma Mass) x with a mass matrix."""
    return S @ x + sigma * (x if mass is None else mass @ x)


def gmres(S, sigma, b, tol: float, restart: int = 30, max_iters: int = 20000,
          jacobi: bool = False, ortho: str = "cgs2", mass=None, x0=None) -> GmresResult:
    """GMRES(restart) for (S + sigma I) x = b, stop when ||b - (S+sigma I)x|| <= tol.

    S is a scipy sparse matrix, sigma a real or complex scalar; with a
    (sparse) mass matrix the system is (S + sigma Mass) x = b.  With
    jacobi=True the method runs on (S + sigma I) P^{-1} u = b with
    P = diag(S) + sigma I (diag(S) + sigma diag(Mass)) and returns x = P^{-1} u.
    x0: initial guess (zero when None); the cycles then solve for the
    correction from the residual b - (S + sigma I) x0.
    """
    dtype = np.result_type(S.dtype, np.asarray(sigma).dtype, b.dtype)
    n = b.shape[0]
    b = b.astype(dtype)
    dmass = 1.0 if mass is None else mass.diagonal().astype(dtype)
    pinv = 1.0 / (S.diagonal().astype(dtype) + sigma * dmass) if jacobi else np.ones(n, dtype)
    x = np.zeros(n, dtype) if x0 is None else np.asarray(x0, dtype).copy()
    r = b.copy() if x0 is None else b - shifted_apply(S, sigma, x, mass)
    beta = np.linalg.norm(r)
    hist = []
    iters = cycles = 0
    if beta <= tol:
        return GmresResult(x, beta, 0, 0, True, hist)
    m = restart
    if ortho == "dcgs2":
        return _gmres_dcgs2(S, sigma, b, tol, m, max_iters, pinv, dtype, mass, x)
    while True:
        cycles += 1
        V = np.zeros((m + 1, n), dtype)
        R = np.zeros((m + 1, m), dtype)     # Hessenberg columns, rotated in place
        cs = np.zeros(m)
        sn = np.zeros(m, dtype)
        g = np.zeros(m + 1, dtype)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = shifted_apply(S, sigma, pinv * V[j], mass)
            iters += 1
            h = np.zeros(j + 2, dtype)
            if ortho == "mgs":
                h[: j + 1], w = mgs_step(V[: j + 1], w)
            elif ortho == "cgs2":
                h[: j + 1], w = cgs2_step(V[: j + 1], w)
            else:
                raise ValueError(ortho)
            hn = np.linalg.norm(w)
            h[j + 1] = hn
            if hn > 0.0:
                V[j + 1] = w / hn
            # apply the previous rotations to the new column
            for i in range(j):
                t0 = cs[i] * h[i] + sn[i] * h[i + 1]
                t1 = -np.conj(sn[i]) * h[i] + cs[i] * h[i + 1]
                h[i], h[i + 1] = t0, t1
            c, s = givens(h[j], h[j + 1])
            cs[j], sn[j] = c, s
            h[j] = c * h[j] + s * h[j + 1]
            h[j + 1] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            R[: j + 2, j] = h
            est = abs(g[j + 1])
            hist.append(est)
            j_done = j + 1
            if est <= tol or iters >= max_iters:
                break
        # least-squares solution: back substitution with the rotated R
        k = j_done
        y = np.zeros(k, dtype)
        for i in range(k - 1, -1, -1):
            acc = g[i] - R[i, i + 1: k] @ y[i + 1: k]
            y[i] = acc / R[i, i] if R[i, i] != 0 else 0.0
        x = x + pinv * (V[:k].T @ y)
        r = b - shifted_apply(S, sigma, x, mass)
        beta = np.linalg.norm(r)
        if beta <= tol:
            return GmresResult(x, beta, iters, cycles, True, hist)
        if iters >= max_iters:
            return GmresResult(x, beta, iters, cycles, False, hist)


def _gmres_dcgs2(S, sigma, b, tol, m, max_iters, pinv, dtype, mass=None, x0=None) -> GmresResult:
    """The restarted GMRES above with the Arnoldi steps of arnoldi_dcgs2.

    Column j-1 of the Hessenberg matrix is complete once step j has the
    delayed second-pass coefficients of u_j; its Givens update and the stop
    test follow, so a cycle that stops there has already formed the product
    of step j (unused).  Arnoldi steps are counted as completed columns."""
    n = b.shape[0]
    x = np.zeros(n, dtype) if x0 is None else x0.copy()
    r = b - shifted_apply(S, sigma, x, mass)
    beta0 = np.linalg.norm(r)
    hist = []
    iters = cycles = 0
    if beta0 <= tol:
        return GmresResult(x, beta0, 0, 0, True, hist)
    while True:
        cycles += 1
        V = np.zeros((m + 1, n), dtype)
        H = np.zeros((m + 1, m), dtype)     # Hessenberg columns as formed
        R = np.zeros((m + 1, m), dtype)     # the same columns, rotated
        cs = np.zeros(m)
        sn = np.zeros(m, dtype)
        g = np.zeros(m + 1, dtype)
        g[0] = beta0
        u = r / beta0
        h1 = None
        k = 0
        for j in range(m + 1):
            y = shifted_apply(S, sigma, pinv * u, mass) if j < m else None
            s = V[:j].conj() @ u
            alpha = np.vdot(u, u).real
            beta = np.sqrt(max(alpha - np.vdot(s, s).real, 0.0))
            if j >= 1:
                c_ = j - 1
                H[:j, c_] = h1 + s
                H[j, c_] = beta
                h = H[: j + 1, c_].copy()
                for i in range(c_):
                    t0 = cs[i] * h[i] + sn[i] * h[i + 1]
                    t1 = -np.conj(sn[i]) * h[i] + cs[i] * h[i + 1]
                    h[i], h[i + 1] = t0, t1
                c, sg = givens(h[c_], h[c_ + 1])
                cs[c_], sn[c_] = c, sg
                h[c_] = c * h[c_] + sg * h[c_ + 1]
                h[c_ + 1] = 0.0
                g[c_ + 1] = -np.conj(sg) * g[c_]
                g[c_] = c * g[c_]
                R[: j + 1, c_] = h
                iters += 1
                est = abs(g[c_ + 1])
                hist.append(est)
                k = j
                if est <= tol or j == m or iters >= max_iters or beta == 0.0:
                    break
            V[j] = (u - V[:j].T @ s) / beta
            z = V[:j].conj() @ y
            gamma = np.vdot(u, y)
            vy = (gamma - np.vdot(s, z)) / beta
            h1 = (np.concatenate([z, [vy]]) - H[: j + 1, :j] @ s) / beta
            u = (y - V[:j].T @ z - V[j] * vy) / beta
        y_ = np.zeros(k, dtype)
        for i in range(k - 1, -1, -1):
            acc = g[i] - R[i, i + 1: k] @ y_[i + 1: k]
            y_[i] = acc / R[i, i] if R[i, i] != 0 else 0.0
        x = x + pinv * (V[:k].T @ y_)
        r = b - shifted_apply(S, sigma, x, mass)
        beta0 = np.linalg.norm(r)
        if beta0 <= tol:
            return GmresResult(x, beta0, iters, cycles, True, hist)
        if iters >= max_iters:
            return GmresResult(x, beta0, iters, cycles, False, hist)


def bicgstab(S, sigma, b, tol: float, max_iters: int = 20000, jacobi: bool = False,
             mass=None, x0=None, trace=None) -> GmresResult:
    """BiCGstab (van der Vorst, SIAM J. Sci. Stat. Comput. 13 (1992)) for
    (S + sigma I) x = b, or (S + sigma Mass) x = b, with right Jacobi
    preconditioning: the short-recurrence inner solver the paper uses for
    its unsymmetric systems (Sec. 3.3 "Further implementation aspects",
    Sec. 4).  Right preconditioning keeps the recurrence residual that of the
    original system; after termination the true residual is recomputed and,
    if it is not below tol, the method starts again from the current iterate
    (fresh shadow vector).  iters counts BiCGstab steps (two operator
    applications each); history holds the recurrence residual norms.  A
    breakdown (rho or the step denominator zero) restarts the same way.
    trace (tests only): called after every full step with the step's vectors
    rhat, v, s, t and the new residual r."""
    dtype = np.result_type(S.dtype, np.asarray(sigma).dtype, b.dtype)
    n = b.shape[0]
    b = b.astype(dtype)
    dmass = 1.0 if mass is None else mass.diagonal().astype(dtype)
    pinv = 1.0 / (S.diagonal().astype(dtype) + sigma * dmass) if jacobi else np.ones(n, dtype)
    x = np.zeros(n, dtype) if x0 is None else np.asarray(x0, dtype).copy()
    r = b.copy() if x0 is None else b - shifted_apply(S, sigma, x, mass)
    rn = np.linalg.norm(r)
    hist = []
    iters = cycles = 0
    while rn > tol and iters < max_iters:
        cycles += 1
        rhat = r.copy()
        rho = alpha = omega = 1.0
        v = np.zeros(n, dtype)
        p = np.zeros(n, dtype)
        while iters < max_iters:
            rho_new = np.vdot(rhat, r)
            if rho_new == 0.0 or omega == 0.0:
                break
            beta = (rho_new / rho) * (alpha / omega)
            p = r + beta * (p - omega * v)
            ph = pinv * p
            v = shifted_apply(S, sigma, ph, mass)
            den = np.vdot(rhat, v)
            iters += 1
            if den == 0.0:
                break
            alpha = rho_new / den
            s = r - alpha * v
            if np.linalg.norm(s) <= tol:
                x = x + alpha * ph
                hist.append(np.linalg.norm(s))
                break
            sh = pinv * s
            t = shifted_apply(S, sigma, sh, mass)
            tt = np.vdot(t, t).real
            omega = np.vdot(t, s) / tt if tt > 0.0 else 0.0
            x = x + alpha * ph + omega * sh
            r = s - omega * t
            if trace is not None:
                trace(dict(rhat=rhat, v=v, s=s, t=t, r=r))
            rho = rho_new
            hist.append(np.linalg.norm(r))
            if hist[-1] <= tol:
                break
        r = b - shifted_apply(S, sigma, x, mass)
        rn = np.linalg.norm(r)
    return GmresResult(x, rn, iters, cycles, rn <= tol, hist)
