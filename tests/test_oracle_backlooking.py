"""Why the literal back-looking rule (eq. (ADI_relax2_prak)) fails on the
convection-diffusion workloads: measured on a reduced member of the 2D
benchmark family (A: N = 48, omega = 50 (x, y); B: N = 40, omega = 20 (y, -x);
r = 2, seed 1, 12 real shift pairs, right-Jacobi GMRES(30)) with the oracle.

* The delta_min clamp of eq. (bound_tols) (tau / 20, Sec. 4) lets the inner
  residuals of step 1 overrun the budget k xi eps / (2 c kmax) of
  eq. (ADI_relax2_theo): u_1 + v_1 > budget_1.
* The literal |.| then turns the overrun into the target:
  hat-eps_k = (u + v - budget) / c grows with u + v, the tolerances grow with
  it, and the true residual gap ||Delta R_k|| (Definition resgapADI, through
  Theorem 2: Delta R = -(S^A Gamma Y^* + Z Gamma (S^B)^*)) ends far above eps,
  although the computed residual meets tau.  Without back-looking
  (eq. (ADI_relax1_prak)) the gap stays below eps.
* The constants check-c_k = max(||C_k(A)||, ||C_k(B)||) + 1 of Theorem 3 are
  far above c = 2 + sqrt(2) for several of these real shift pairs (the
  assumptions behind c, Sec. 3.3.1, do not hold), so c is no bound here.

Running this file as a script prints the per-step table.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2312_02891_gb300 import workloads as W
from oracle import controller as ctl
from oracle.lradi import lradi
from oracle.residual import lowrank_norm2

KMAX = 50


def _problem():
    return W.make_problem("red2d", 48, 2, "xy", 50.0, 40, 2, "rot2", 20.0, 2, 1, 12, restart=30, jacobi=True)


def cayley_norm(S, a, b):
    """||(S - a I)(S + b I)^{-1}||_2 (the operator C_k of eq. (fadi_error))."""
    n = S.shape[0]
    lu = spla.splu((S + b * sp.identity(n)).tocsc())
    Sm = (S - a * sp.identity(n)).tocsr()
    op = spla.LinearOperator((n, n), matvec=lambda x: Sm @ lu.solve(x),
                             rmatvec=lambda y: lu.solve(Sm.T @ y, trans="T"), dtype=float)
    return float(spla.svds(op, k=1, return_singular_vectors=False, tol=1e-6)[0])


def per_step(p, strategy, with_c=False):
    r = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy=strategy, jacobi=True,
              keep_inner_residuals=True, kmax=KMAX)
    nfg = lowrank_norm2(p.f, p.g)
    eps = p.tau * nfg
    A, B = p.A.to_scipy().tocsc(), p.B.to_scipy().tocsc()
    L, rk = len(p.alpha), p.r
    cache, rows = {}, []
    for h in r.history:
        k = h["k"]
        kk = k * rk
        G = r.gamma[:kk]
        gap = lowrank_norm2(np.hstack([r.S_A[:, :kk] * G[None, :], r.Z[:, :kk] * G[None, :]]),
                            np.hstack([r.Y[:, :kk], r.S_B[:, :kk]]))
        row = dict(k=k, uv=h["u"] + h["v"], gap=gap, budget=k * eps / (2 * ctl.C_BOUND * KMAX),
                   eps_hat=h["eps_hat"], dA=h["dA"], dB=h["dB"], res=h["res_comp"])
        if with_c:
            idx = (k - 1) % L
            if idx not in cache:
                a, b = float(np.real(p.alpha[idx])), float(np.real(p.beta[idx]))
                cache[idx] = (cayley_norm(A, a, b), cayley_norm(B, b, a))
            row["cA"], row["cB"] = cache[idx]
            row["cchk"] = max(cache[idx]) + 1
        rows.append(row)
    return r, eps, rows


@pytest.fixture(scope="module")
def red2d():
    return _problem()


def test_literal_back_looking_relaxes_past_the_gap_target(red2d):
    r, eps, rows = per_step(red2d, "bl_mid")
    assert r.converged and r.res_comp < red2d.tau          # the computed residual meets tau ...
    assert rows[0]["uv"] > rows[0]["budget"]              # ... the delta_min clamp overruns step 1's budget
    over = [x for x in rows if x["uv"] > x["budget"]]
    assert len(over) == len(rows)
    # from step 2 on, hat-eps_k follows the overrun of the previous steps:
    # |budget_k - u_{k-1} - v_{k-1}| / c = (u_{k-1} + v_{k-1} - budget_k) / c
    for prev, x in zip(rows, rows[1:]):
        assert prev["uv"] > x["budget"]
        assert x["eps_hat"] == pytest.approx((prev["uv"] - x["budget"]) / ctl.C_BOUND, rel=1e-9)
    assert rows[-1]["eps_hat"] > 1e4 * rows[0]["eps_hat"]
    # ... and the true residual gap ends far above eps (the paper's Theorem 3 target)
    assert rows[-1]["gap"] > 10 * eps
    assert all(x["gap"] <= x["uv"] * (1 + 1e-9) for x in rows)        # u + v bounds the gap


def test_without_back_looking_the_gap_stays_below_eps(red2d):
    r, eps, rows = per_step(red2d, "nobl_mid")
    assert r.converged
    assert rows[-1]["gap"] < eps
    assert all(x["gap"] <= x["uv"] * (1 + 1e-9) for x in rows)


@pytest.mark.slow
def test_cayley_constants_exceed_c(red2d):
    p = red2d
    A, B = p.A.to_scipy().tocsc(), p.B.to_scipy().tocsc()
    chk = [max(cayley_norm(A, float(np.real(a)), float(np.real(b))),
               cayley_norm(B, float(np.real(b)), float(np.real(a)))) + 1
           for a, b in zip(p.alpha[:4], p.beta[:4])]
    assert max(chk) > 10 * ctl.C_BOUND


if __name__ == "__main__":
    p = _problem()
    for strategy in ("bl_mid", "nobl_mid"):
        r, eps, rows = per_step(p, strategy, with_c=True)
        print(f"\n{strategy}: steps {r.steps}, computed residual {r.res_comp:.2e}, eps {eps:.2e}\n")
        print("| k | c^A_k | c^B_k | check-c_k | u_k + v_k | true gap | budget | hat-eps_k | delta^A_k | delta^B_k |")
        print("|---|---|---|---|---|---|---|---|---|---|")
        for x in rows:
            print(f"| {x['k']} | {x['cA']:.2f} | {x['cB']:.2f} | {x['cchk']:.2f} | {x['uv']:.2e} | {x['gap']:.2e} | "
                  f"{x['budget']:.2e} | {x['eps_hat']:.2e} | {x['dA']:.2e} | {x['dB']:.2e} |")
