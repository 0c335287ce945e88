"""Algorithm 1 with real arithmetic for complex conjugate shift pairs.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For real A, B, M, C, f, g the paper keeps the complex formulation and notes
(Sec. 3.3, "Complex shift parameters") that a double step per conjugate pair
needs only one complex solve and gives real factors.  This module writes that
double step out.  Steps k and k+1 use the shift pairs (alpha, beta) and
(conj alpha, conj beta), gamma = -(alpha + beta):

  z1 = (A + beta M)^{-1} w,        z2 = (A + conj(beta) M)^{-1} (w + gamma M z1)
  y1 = (B + alpha C)^{-*} t,       y2 = (B + conj(alpha) C)^{-*} (t + conj(gamma) C^* y1)

From (A + conj(b) M)^{-1} M (A + b M)^{-1} = [(A + conj(b) M)^{-1} - (A + b M)^{-1}] / (b - conj(b)) and
(A + conj(b) M)^{-1} w = conj(z1) for real w:

  Im(beta) != 0:  z2 = conj(z1) - gamma Im(z1) / Im(beta)        (one complex solve)
  Im(beta) == 0:  z1 real,  z2 = z1 + gamma q,  (A + beta M) q = M z1   (two real solves)

and on the B side, with B^T + conj(alpha) C^T for y1:

  Im(alpha) != 0: y2 = conj(y1) + conj(gamma) Im(y1) / Im(alpha)
  Im(alpha) == 0: y1 real,  y2 = y1 + conj(gamma) q,  (B^T + alpha C^T) q = C^T y1.

So [z1, z2] = [a1, a2] P and [y1, y2] = [b1, b2] Q with real n x r blocks
a1, a2 (Re z1, Im z1, or z1, q) and b1, b2, and 2 x 2 complex P, Q; the two
steps add [a1, a2] (G kron I_r) [b1, b2]^T to X with the real core
G = P diag(gamma, conj gamma) Q^*, and w, t stay real.

Readings (the paper gives no formulas):
* Inner residuals of the derived second solution: with r1 = w - (A + beta M) z1,
  r2 = (w + gamma M z1) - (A + conj(beta) M) z2 = conj(r1) - gamma Im(r1) / Im(beta),
  so ||r2|| <= ||r1|| (1 + |gamma| / |Im beta|); the one complex solve runs to
  delta / (1 + |gamma| / |Im beta|) so that both steps meet delta.  With a
  real shift r2 = r1 + gamma r_q; the two real solves run to delta / 2 and
  delta / (2 |gamma|).  (delta per column: delta / r, as in oracle.lradi.)
* One controller evaluation per pair (at its first step) gives delta for
  both steps; u, v of eq. (upd_resgap) add both steps with their actual
  residuals, as in the complex formulation.
* Pairs must be complete (the second member present); real shift pairs take
  the plain real step of Algorithm 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import controller as ctl
from .gmres import bicgstab, gmres
from .lradi import DEFAULTS, _as_scipy, _is_pair_start
from .residual import block_norm2, lowrank_norm2


@dataclass
class LradiRealResult:
    Z: np.ndarray               # real n x kr
    Y: np.ndarray               # real m x kr
    Gamma: np.ndarray           # real kr x kr, block diagonal (1 x 1 or 2 x 2 blocks, kron I_r)
    steps: int                  # outer steps taken (a pair counts two)
    converged: bool
    res_comp: float
    inner_its_A: int
    inner_its_B: int
    complex_solves: int         # columns solved in complex arithmetic
    history: list = field(default_factory=list)
    w: np.ndarray | None = None
    t: np.ndarray | None = None
    # per step of the equivalent complex formulation (keep_inner_residuals=True):
    # z_k, y_k, gamma_k and the inner residuals r^A_k, r^B_k
    steps_complex: list | None = None


def _coeffs_complex(c, im_shift):
    """P with [x1, x2] = [Re x1, Im x1] P when the pair's shift on this side
    is complex: x2 = conj(x1) - c Im(x1) / Im(shift), c = gamma on the A side
    (shift beta) and -conj(gamma) on the B side (shift alpha)."""
    return np.array([[1.0, 1.0], [1j, -1j - c / im_shift]])


def _coeffs_real(c):
    """P with [x1, x2] = [x1, q] P when the shift on this side is real:
    x2 = x1 + c q, c = gamma (A side) or conj(gamma) (B side)."""
    return np.array([[1.0, 1.0], [0.0, c]])


def _solve(kind, S, sigma, rhs, tol, o, mass, lu_cache, key):
    """One column: sparse LU ("direct") or the iterative oracle solvers."""
    if kind == "direct":
        if key not in lu_cache:
            n = S.shape[0]
            mm = sp.identity(n) if mass is None else mass
            dt = np.result_type(S.dtype, np.asarray(sigma).dtype, np.float64)
            lu_cache[key] = spla.splu((S + sigma * mm).astype(dt).tocsc())
        return lu_cache[key].solve(rhs.astype(lu_cache[key].U.dtype)), 0
    if kind == "gmres":
        r = gmres(S, sigma, rhs, tol, o["restart"], o["max_inner"], o["jacobi"], o["ortho"], mass=mass)
    else:
        r = bicgstab(S, sigma, rhs, tol, o["max_inner"], o["jacobi"], mass=mass)
    return r.x, r.iters


def lradi_real(A, B, f, g, alpha, beta, tau: float = 1e-8, M=None, C=None, **opts) -> LradiRealResult:
    o = dict(DEFAULTS)
    unknown = set(opts) - set(o)
    if unknown:
        raise TypeError(f"unknown options {sorted(unknown)}")
    o.update(opts)
    for key in ("dmin_A", "dmin_B", "fixed_tol"):
        if o[key] is None:
            o[key] = tau / 20
    kind = o["inner"]
    if o["inner_A"] or o["inner_B"]:
        raise ValueError("lradi_real uses one inner solver for both sides")
    SA = _as_scipy(A)
    SBt = _as_scipy(B).T.tocsr()
    SM = None if M is None else _as_scipy(M)
    SCt = None if C is None else _as_scipy(C).T.tocsr()
    alpha = np.asarray(alpha)
    beta = np.asarray(beta)
    n, r = f.shape
    m = g.shape[0]
    w = np.asarray(f, dtype=np.float64).copy()
    t = np.asarray(g, dtype=np.float64).copy()
    nfg = lowrank_norm2(f, g)
    empty = LradiRealResult(np.zeros((n, 0)), np.zeros((m, 0)), np.zeros((0, 0)), 0, True, 0.0, 0, 0, 0,
                            [], w, t, [] if o["keep_inner_residuals"] else None)
    if nfg == 0.0:
        return empty
    eps = tau * nfg
    mulM = (lambda x: x) if SM is None else (lambda x: SM @ x)
    mulC = (lambda x: x) if SCt is None else (lambda x: SCt @ x)
    opA = lambda sig, x: SA @ x + sig * mulM(x)
    opB = lambda sig, x: SBt @ x + sig * mulC(x)
    Zs, Ys, blocks, hist = [], [], [], []
    cplx_steps = [] if o["keep_inner_residuals"] else None
    u = v = 0.0
    itsA_tot = itsB_tot = n_cplx = 0
    lu_cache = {}
    k = 1
    converged = False
    res = lowrank_norm2(w, t)
    L = len(alpha)
    while True:
        if res < tau * nfg:
            converged = True
            break
        if k > o["kmax"]:
            break
        idx = (k - 1) % L
        a_k, b_k = alpha[idx], beta[idx]
        pair = _is_pair_start(alpha, beta, idx)
        if not pair and (np.imag(a_k) != 0 or np.imag(b_k) != 0):
            raise ValueError(f"shift {idx} is complex but its conjugate does not follow it")
        N_w, N_t = block_norm2(w), block_norm2(t)
        dA, dB, eh = ctl.inner_tolerances(
            o["strategy"], k=k, kmax=o["kmax"], eps=eps, xi=o["xi"], u_prev=u, v_prev=v,
            N_w=N_w, N_t=N_t, dmin_A=o["dmin_A"], dmax_A=o["dmax_A"],
            dmin_B=o["dmin_B"], dmax_B=o["dmax_B"], fixed_tol=o["fixed_tol"])
        gam = -(b_k + a_k)
        if not pair:
            # the real step of Algorithm 1
            a_k, b_k, gam = float(np.real(a_k)), float(np.real(b_k)), float(np.real(gam))
            z = np.zeros((n, r)); y = np.zeros((m, r))
            for l in range(r):
                z[:, l], ia = _solve(kind, SA, b_k, w[:, l], dA / r, o, SM, lu_cache, ("A", b_k))
                y[:, l], ib = _solve(kind, SBt, a_k, t[:, l], dB / r, o, SCt, lu_cache, ("B", a_k))
                itsA_tot += ia; itsB_tot += ib
            Mz, Cy = mulM(z), mulC(y)
            rA = w - opA(b_k, z)
            rB = t - opB(a_k, y)
            nrA, nrB = block_norm2(rA), block_norm2(rB)
            w = w + gam * Mz
            t = t + gam * Cy
            u += abs(gam) * block_norm2(Mz) * nrB
            v += abs(gam) * block_norm2(Cy) * nrA
            Zs.append(z); Ys.append(y); blocks.append(np.array([[gam]]))
            if cplx_steps is not None:
                cplx_steps.append(dict(z=z, y=y, gamma=gam, rA=rA, rB=rB))
            res = lowrank_norm2(w, t)
            hist.append(dict(k=k, pair=False, dA=dA, dB=dB, eps_hat=eh, nrA=[nrA], nrB=[nrB], u=u, v=v,
                             res_comp=res / nfg))
            k += 1
            continue
        # ---- double step for the pair (a_k, b_k), (conj a_k, conj b_k) ----
        a1 = np.zeros((n, r)); a2 = np.zeros((n, r))
        b1 = np.zeros((m, r)); b2 = np.zeros((m, r))
        if np.imag(b_k) != 0:
            fac = 1.0 + abs(gam) / abs(np.imag(b_k))
            for l in range(r):
                zc, ia = _solve(kind, SA, b_k, w[:, l].astype(complex), dA / r / fac, o, SM, lu_cache, ("A", complex(b_k)))
                a1[:, l], a2[:, l] = zc.real, zc.imag
                itsA_tot += ia; n_cplx += 1
            P = _coeffs_complex(gam, np.imag(b_k))
        else:
            br = float(np.real(b_k))
            for l in range(r):
                a1[:, l], ia = _solve(kind, SA, br, w[:, l], dA / r / 2, o, SM, lu_cache, ("A", br))
                itsA_tot += ia
            Ma1 = mulM(a1)
            for l in range(r):
                a2[:, l], ia = _solve(kind, SA, br, Ma1[:, l], dA / r / (2 * abs(gam)), o, SM, lu_cache, ("A", br))
                itsA_tot += ia
            P = _coeffs_real(gam)
        if np.imag(a_k) != 0:
            fac = 1.0 + abs(gam) / abs(np.imag(a_k))
            for l in range(r):
                yc, ib = _solve(kind, SBt, np.conj(a_k), t[:, l].astype(complex), dB / r / fac, o, SCt, lu_cache,
                                ("B", complex(np.conj(a_k))))
                b1[:, l], b2[:, l] = yc.real, yc.imag
                itsB_tot += ib; n_cplx += 1
            Q = _coeffs_complex(-np.conj(gam), np.imag(a_k))
        else:
            ar = float(np.real(a_k))
            for l in range(r):
                b1[:, l], ib = _solve(kind, SBt, ar, t[:, l], dB / r / 2, o, SCt, lu_cache, ("B", ar))
                itsB_tot += ib
            Cb1 = mulC(b1)
            for l in range(r):
                b2[:, l], ib = _solve(kind, SBt, ar, Cb1[:, l], dB / r / (2 * abs(gam)), o, SCt, lu_cache, ("B", ar))
                itsB_tot += ib
            Q = _coeffs_real(np.conj(gam))
        # the two steps of the complex formulation, for residuals and u, v
        z1 = a1 * P[0, 0] + a2 * P[1, 0]
        z2 = a1 * P[0, 1] + a2 * P[1, 1]
        y1 = b1 * Q[0, 0] + b2 * Q[1, 0]
        y2 = b1 * Q[0, 1] + b2 * Q[1, 1]
        g1, g2 = gam, np.conj(gam)
        rA1 = w - opA(b_k, z1)
        rB1 = t - opB(np.conj(a_k), y1)
        w1 = w + g1 * mulM(z1)
        t1 = t + np.conj(g1) * mulC(y1)
        rA2 = w1 - opA(np.conj(b_k), z2)
        rB2 = t1 - opB(a_k, y2)
        w2 = w1 + g2 * mulM(z2)
        t2 = t1 + np.conj(g2) * mulC(y2)
        nrA = [block_norm2(rA1), block_norm2(rA2)]
        nrB = [block_norm2(rB1), block_norm2(rB2)]
        u += abs(g1) * block_norm2(mulM(z1)) * nrB[0] + abs(g2) * block_norm2(mulM(z2)) * nrB[1]
        v += abs(g1) * block_norm2(mulC(y1)) * nrA[0] + abs(g2) * block_norm2(mulC(y2)) * nrA[1]
        G = P @ np.diag([g1, g2]) @ Q.conj().T
        if abs(G.imag).max() > 1e-10 * abs(G).max() or abs(w2.imag).max() > 1e-8 * (abs(w2).max() + 1e-300) \
                or abs(t2.imag).max() > 1e-8 * (abs(t2).max() + 1e-300):
            raise FloatingPointError("double step did not stay real")
        w, t = w2.real.copy(), t2.real.copy()
        Zs.append(np.hstack([a1, a2])); Ys.append(np.hstack([b1, b2])); blocks.append(G.real)
        if cplx_steps is not None:
            cplx_steps.append(dict(z=z1, y=y1, gamma=g1, rA=rA1, rB=rB1))
            cplx_steps.append(dict(z=z2, y=y2, gamma=g2, rA=rA2, rB=rB2))
        res = lowrank_norm2(w, t)
        hist.append(dict(k=k, pair=True, dA=dA, dB=dB, eps_hat=eh, nrA=nrA, nrB=nrB, u=u, v=v,
                         res_comp=res / nfg))
        k += 2
    Z = np.hstack(Zs) if Zs else np.zeros((n, 0))
    Y = np.hstack(Ys) if Ys else np.zeros((m, 0))
    kr = Z.shape[1]
    Gam = np.zeros((kr, kr))
    pos = 0
    for Gb in blocks:
        s = Gb.shape[0] * r
        Gam[pos:pos + s, pos:pos + s] = np.kron(Gb, np.eye(r))
        pos += s
    return LradiRealResult(Z, Y, Gam, k - 1, converged, res / nfg, itsA_tot, itsB_tot, n_cplx, hist,
                           w, t, cplx_steps)
