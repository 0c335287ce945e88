"""Algorithm 1 (inexact LR-ADI for Sylvester equations).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Solves A X + X B = -f g^* (eq. (sylv)), or with nonsingular M, C the
generalized equation A X C + M X B = -f g^* (eq. (gsylv)), for
X ~ Z Gamma Y^*, following the steps of Algorithm 1 in the paper's order
(M = I, C = I when they are not given):

  w_0 = f, t_0 = g, Z = Y = Gamma = [], k = 1
  while ||w_{k-1} t_{k-1}^*|| >= tau ||f g^*||:
      (delta^A_k, delta^B_k) from the controller (Sec. 3.3)
      solve (A + beta_k M) z_k = w_{k-1}      to ||r^A_k|| <= delta^A_k
      solve (B + alpha_k C)^* y_k = t_{k-1}   to ||r^B_k|| <= delta^B_k
      gamma_k = -(beta_k + alpha_k)
      w_k = w_{k-1} + gamma_k M z_k,  t_k = t_{k-1} + conj(gamma_k) C^* y_k
      Z = [Z, z_k], Y = [Y, y_k], Gamma = diag(Gamma, gamma_k I_r)
      u_k, v_k by eq. (upd_resgap) (with ||M z_k||, ||C^T y_k||)
      k = k + 1

Readings where the paper is silent or inconsistent:
* The inner systems use (A + beta_k I) and (B + alpha_k I)^* as in
  Algorithm 1 and eq. (lradi_basic) (eq. (linres) swaps the shifts).
* Gamma's diagonal is gamma_k = -(beta_k + alpha_k) (Algorithm 1), not the
  fADI entry beta_k - alpha_k.
* eps = tau ||f g^*||_2: the absolute residual-gap target; delta_min,
  delta_max and the fixed tolerance are absolute numbers.
* Each of the r columns is solved separately to delta_k / r; ||r^A_k|| etc.
  are spectral norms of the n x r blocks.
* u, v use the achieved inner residual norms.
* Shifts are reused cyclically when k exceeds their number.
* With complex shifts, conjugate pairs (alpha_{k+1}, beta_{k+1}) =
  (conj alpha_k, conj beta_k) are consecutive and the outer stop test is
  skipped after the first member of a pair.
* An inner solve that reaches its iteration cap keeps its best iterate and
  its achieved residual feeds u, v.
* recycle="prev": each iterative inner solve starts from the multiple of
  the previous step's solution (same side and column) with the smallest
  residual (recycled_guess), a reading of the paper's outlook (Sec. 5).
* Inner solvers: "direct" (sparse LU), "gmres" (restarted GMRES, right
  Jacobi) or "bicgstab" (the paper's short-recurrence choice, right Jacobi),
  for both sides (inner) or per side (inner_A, inner_B).  When exactly one
  side is direct, its tolerance is 0 and the other side's follows the
  simplified rule of Sec. 3.3 ("Combination of direct and iterative linear
  solves"): ||r|| <= hat-eps_k / ||w_{k-1}|| (or / ||t_{k-1}||).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import controller as ctl
from .gmres import bicgstab, gmres
from .residual import block_norm2, lowrank_norm2

DEFAULTS = dict(strategy="bl_mid", inner="gmres", inner_A=None, inner_B=None, restart=30, max_inner=20000,
                jacobi=False, xi=1.0, dmin_A=None, dmin_B=None, dmax_A=0.1,
                dmax_B=0.1, kmax=50, fixed_tol=None, ortho="cgs2",
                keep_inner_residuals=False, recycle=None)


@dataclass
class LradiResult:
    Z: np.ndarray
    Y: np.ndarray
    gamma: np.ndarray           # diagonal of Gamma (length k*r)
    steps: int                  # outer steps taken
    converged: bool
    res_comp: float             # ||w t^*|| / ||f g^*|| at exit
    inner_its_A: int
    inner_its_B: int
    history: list = field(default_factory=list)
    S_A: np.ndarray | None = None
    S_B: np.ndarray | None = None
    w: np.ndarray | None = None
    t: np.ndarray | None = None


def _as_scipy(M):
    if hasattr(M, "to_scipy"):
        return M.to_scipy()
    return sp.csr_matrix(M)


def _is_pair_start(alpha, beta, idx):
    """True when shift idx opens a conjugate pair completed by idx+1."""
    L = len(alpha)
    a, b = alpha[idx], beta[idx]
    if np.imag(a) == 0 and np.imag(b) == 0:
        return False
    if idx + 1 >= L:
        return False
    return np.conj(a) == alpha[idx + 1] and np.conj(b) == beta[idx + 1]


def recycled_guess(S, sigma, b, u, mass=None):
    """The multiple c u of the previous step's solution u with the smallest
    residual ||b - c (S + sigma Mass) u||: c = (v^* b) / (v^* v), v the
    shifted operator applied to u.  A reading of the paper's outlook (Sec. 5:
    reuse what earlier shifted solves computed for the later ones); the
    paper defines no such method.  Zero when u is zero."""
    v = S @ u + sigma * (u if mass is None else mass @ u)
    vv = np.vdot(v, v).real
    return (np.vdot(v, b) / vv) * u if vv > 0.0 else np.zeros_like(u)


def _iterative(solver, S, sigma, b, tol, o, mass, x0=None):
    if solver == "gmres":
        return gmres(S, sigma, b, tol, o["restart"], o["max_inner"], o["jacobi"], o["ortho"], mass=mass, x0=x0)
    return bicgstab(S, sigma, b, tol, o["max_inner"], o["jacobi"], mass=mass, x0=x0)


def lradi(A, B, f, g, alpha, beta, tau: float = 1e-8, M=None, C=None, **opts) -> LradiResult:
    o = dict(DEFAULTS)
    unknown = set(opts) - set(o)
    if unknown:
        raise TypeError(f"unknown options {sorted(unknown)}")
    o.update(opts)
    if o["dmin_A"] is None:
        o["dmin_A"] = tau / 20
    if o["dmin_B"] is None:
        o["dmin_B"] = tau / 20
    if o["fixed_tol"] is None:
        o["fixed_tol"] = tau / 20
    solver_A = o["inner_A"] or o["inner"]
    solver_B = o["inner_B"] or o["inner"]
    for sv in (solver_A, solver_B):
        if sv not in ("direct", "gmres", "bicgstab"):
            raise ValueError(f"unknown inner solver {sv!r}")
    direct_side = None
    if solver_A == "direct" and solver_B != "direct":
        direct_side = "A"
    elif solver_B == "direct" and solver_A != "direct":
        direct_side = "B"
    SA = _as_scipy(A)
    SBt = _as_scipy(B).T.tocsr()            # (B + alpha C)^* = B^T + conj(alpha) C^T for real B, C
    SM = None if M is None else _as_scipy(M)
    SCt = None if C is None else _as_scipy(C).conj().T.tocsr()
    alpha = np.asarray(alpha)
    beta = np.asarray(beta)
    cplx = np.iscomplexobj(alpha) or np.iscomplexobj(beta) or np.iscomplexobj(f)
    dt = np.complex128 if cplx else np.float64
    n, r = f.shape
    m = g.shape[0]
    w = f.astype(dt).copy()
    t = g.astype(dt).copy()
    nfg = lowrank_norm2(f, g)
    if nfg == 0.0:
        # f g^* = 0: X = 0 solves eq. (sylv) exactly, no step is taken
        return LradiResult(np.zeros((n, 0), dt), np.zeros((m, 0), dt), np.zeros(0, dt), 0, True,
                           0.0, 0, 0, [], None, None, w, t)
    eps = tau * nfg
    Zs, Ys, gammas, hist = [], [], [], []
    SAs, SBs = [], []
    u = v = 0.0
    itsA_tot = itsB_tot = 0
    lu_cache = {}
    k = 1
    converged = False
    pair_open = False
    res = lowrank_norm2(w, t)
    while True:
        if not pair_open and res < tau * nfg:
            converged = True
            break
        if k > o["kmax"]:
            break
        idx = (k - 1) % len(alpha)
        a_k, b_k = alpha[idx], beta[idx]
        N_w, N_t = block_norm2(w), block_norm2(t)
        dA, dB, eh = ctl.inner_tolerances(
            o["strategy"], k=k, kmax=o["kmax"], eps=eps, xi=o["xi"], u_prev=u, v_prev=v,
            N_w=N_w, N_t=N_t, dmin_A=o["dmin_A"], dmax_A=o["dmax_A"],
            dmin_B=o["dmin_B"], dmax_B=o["dmax_B"], fixed_tol=o["fixed_tol"], direct=direct_side)
        z = np.zeros((n, r), dt)
        y = np.zeros((m, r), dt)
        itsA = itsB = 0
        okA = okB = True
        for l in range(r):
            if solver_A == "direct":
                key = ("A", complex(b_k))
                if key not in lu_cache:
                    mA = sp.eye(n) if SM is None else SM
                    lu_cache[key] = spla.splu((SA + b_k * mA).astype(dt).tocsc())
                z[:, l] = lu_cache[key].solve(w[:, l])
            else:
                x0 = None
                if o["recycle"] == "prev" and Zs:
                    x0 = recycled_guess(SA, b_k, w[:, l].astype(dt), Zs[-1][:, l].astype(dt), SM)
                ra = _iterative(solver_A, SA, b_k, w[:, l], dA / r, o, SM, x0)
                z[:, l] = ra.x
                itsA += ra.iters
                okA &= ra.converged
            if solver_B == "direct":
                key = ("B", complex(a_k))
                if key not in lu_cache:
                    mB = sp.eye(m) if SCt is None else SCt
                    lu_cache[key] = spla.splu((SBt + np.conj(a_k) * mB).astype(dt).tocsc())
                y[:, l] = lu_cache[key].solve(t[:, l])
            else:
                x0 = None
                if o["recycle"] == "prev" and Ys:
                    x0 = recycled_guess(SBt, np.conj(a_k), t[:, l].astype(dt), Ys[-1][:, l].astype(dt), SCt)
                rb = _iterative(solver_B, SBt, np.conj(a_k), t[:, l], dB / r, o, SCt, x0)
                y[:, l] = rb.x
                itsB += rb.iters
                okB &= rb.converged
        Mz = z if SM is None else SM @ z
        Cy = y if SCt is None else SCt @ y          # C^* y
        rA = w - (SA @ z + b_k * Mz)
        rB = t - (SBt @ y + np.conj(a_k) * Cy)
        gam = -(b_k + a_k)
        w = w + gam * Mz
        t = t + np.conj(gam) * Cy
        Zs.append(z); Ys.append(y); gammas.extend([gam] * r)
        if o["keep_inner_residuals"]:
            SAs.append(rA); SBs.append(rB)
        nrA, nrB = block_norm2(rA), block_norm2(rB)
        u = u + abs(gam) * block_norm2(Mz) * nrB
        v = v + abs(gam) * block_norm2(Cy) * nrA
        itsA_tot += itsA; itsB_tot += itsB
        res = lowrank_norm2(w, t)
        hist.append(dict(k=k, alpha=a_k, beta=b_k, dA=dA, dB=dB, eps_hat=eh, nrA=nrA, nrB=nrB,
                         itsA=itsA, itsB=itsB, okA=okA, okB=okB, u=u, v=v,
                         res_comp=res / nfg, N_w=N_w, N_t=N_t))
        pair_open = _is_pair_start(alpha, beta, idx) and not pair_open
        k += 1
    Z = np.hstack(Zs) if Zs else np.zeros((n, 0), dt)
    Y = np.hstack(Ys) if Ys else np.zeros((m, 0), dt)
    return LradiResult(Z, Y, np.array(gammas, dtype=dt), k - 1, converged, res / nfg,
                       itsA_tot, itsB_tot, hist,
                       np.hstack(SAs) if SAs else None, np.hstack(SBs) if SBs else None,
                       w, t)
