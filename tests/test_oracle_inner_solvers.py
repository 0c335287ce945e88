"""Pins of the oracle's other inner solvers: BiCGstab (the short-recurrence
method the paper uses for its unsymmetric systems, Sec. 4) and the
combination of direct and iterative solves (Sec. 3.3, "Combination of direct
and iterative linear solves"), where the criteria reduce to
||r^B_k|| <= hat-eps_k / ||w_{k-1}|| when the A-side systems are solved
directly.  Checked against sparse LU, a one-step closed form, the dense
solution of eq. (sylv), Theorem 2 (eq. (adi_res_inexact)) with the inner
residuals these solvers leave, and Table 2's qualitative results.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2312_02891_gb300 import workloads as W
from oracle import controller as ctl
from oracle.dense import dense_residual, kron_solve
from oracle.gmres import bicgstab, gmres, shifted_apply
from oracle.lradi import lradi
from oracle.residual import true_residual_norm2


@pytest.fixture(scope="module")
def tiny():
    return W.problem_config("tiny2d")


@pytest.fixture(scope="module")
def micro():
    return W.make_problem("micro", 8, 2, "xy", 10.0, 7, 2, "rot2", 5.0, 2, 3, 8)


@pytest.fixture(scope="module")
def small():
    return W.problem_config("small2d")


def X_of(res):
    return (res.Z * res.gamma[None, :]) @ res.Y.conj().T


@pytest.mark.parametrize("jacobi", [False, True])
@pytest.mark.parametrize("sigma", [-151.5, -300.0 + 200.0j])
@pytest.mark.parametrize("with_mass", [False, True])
def test_bicgstab_matches_sparse_solve(tiny, jacobi, sigma, with_mass):
    S = tiny.A.to_scipy()
    n = S.shape[0]
    Mm = W.mass_matrix(12, 2).to_scipy() * (13.0 ** 2) if with_mass else None
    Op = S + sigma * (Mm if with_mass else sp.identity(n))
    b = tiny.f[:, 0].astype(np.result_type(sigma, np.float64))
    x_ref = spla.spsolve(Op.tocsc(), b)
    res = bicgstab(S, sigma, b, 1e-12 * np.linalg.norm(b), 5000, jacobi, mass=Mm)
    assert res.converged
    assert np.linalg.norm(res.x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    # the reported residual is the recomputed true residual
    assert res.resnorm == pytest.approx(np.linalg.norm(b - Op @ res.x), rel=1e-10, abs=1e-15)
    assert res.resnorm <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("sigma", [-151.5, -300.0 + 200.0j])
def test_bicgstab_step_conditions(tiny, sigma):
    """The two conditions that define a BiCGstab step (van der Vorst 1992):
    alpha makes the intermediate residual s = r - alpha v orthogonal to the
    shadow vector (rhat^* s = 0, the BiCG condition), and omega minimises
    ||s - omega t||, so the new residual is orthogonal to t (t^* r = 0).  A
    conjugation slip in either coefficient breaks one of them for a complex
    shift, although the iteration may still converge."""
    S = tiny.A.to_scipy()
    b = W.normal(11, 0, 0, tiny.A.n).astype(complex)
    steps = []
    res = bicgstab(S, sigma, b, 1e-12, jacobi=True, trace=steps.append)
    assert res.converged and len(steps) >= 5
    for st in steps:
        rh, s, t, r = st["rhat"], st["s"], st["t"], st["r"]
        assert abs(np.vdot(rh, s)) <= 1e-10 * np.linalg.norm(rh) * np.linalg.norm(s)
        assert abs(np.vdot(t, r)) <= 1e-10 * np.linalg.norm(t) * np.linalg.norm(r)


@pytest.mark.parametrize("n", [5, 6, 8])
@pytest.mark.parametrize("sigma", [0.5, 1.0 + 0.7j])
def test_bicgstab_terminates_in_n_steps(n, sigma):
    """In exact arithmetic BiCGstab's residual is the BiCG residual times a
    product of first-degree factors, and BiCG terminates after at most n
    steps, so on a small nonsymmetric system (distinct eigenvalues, no
    breakdown) the recurrence residual drops to rounding level exactly at step
    n.  A wrong search direction (beta or the q = p - omega v correction)
    loses this."""
    M = np.diag(2.0 * np.arange(1, n + 1)) + 0.3 * W.normal(21, 1, 0, n * n).reshape(n, n)
    b = W.normal(21, 2, 0, n).astype(complex)
    nb = np.linalg.norm(b)
    res = bicgstab(sp.csr_matrix(M), sigma, b, 1e-12 * nb, max_iters=3 * n)
    assert res.converged and res.iters == n and res.cycles == 1
    assert res.history[n - 2] > 1e-8 * nb and res.history[n - 1] <= 1e-13 * nb


@pytest.mark.parametrize("solver", ["gmres", "bicgstab"])
def test_jacobi_of_the_shifted_pencil(solver):
    """Right Jacobi for (Op + sigma Mass) x = b divides by the diagonal of the
    pencil, diag(Op) + sigma diag(Mass): when Op and Mass are diagonal the
    preconditioned operator is the identity and one step solves the system
    exactly (a preconditioner built from diag(Op) + sigma alone would not)."""
    n = 40
    d1 = 1.0 + np.arange(n, dtype=float)
    d2 = 0.5 + 0.25 * np.arange(n, dtype=float)
    S, Mass = sp.diags(d1).tocsr(), sp.diags(d2).tocsr()
    b = W.normal(17, 0, 0, n)
    sigma = 3.0
    f = gmres if solver == "gmres" else bicgstab
    res = f(S, sigma, b, 1e-12 * np.linalg.norm(b), jacobi=True, mass=Mass)
    assert res.converged and res.iters == 1
    assert np.allclose(res.x, b / (d1 + sigma * d2), rtol=1e-13)


def test_bicgstab_multiple_of_identity_takes_one_step():
    """Op = c I: p = r, v = (c + sigma) r, alpha = 1 / (c + sigma), s = 0:
    one step gives x = b / (c + sigma) (up to rounding)."""
    n, c, sigma = 50, -4.0, -1.5
    b = np.linspace(1.0, 2.0, n)
    res = bicgstab(sp.identity(n, format="csr") * c, sigma, b, 1e-12)
    assert res.converged and res.iters == 1
    assert np.allclose(res.x, b / (c + sigma), rtol=1e-15, atol=0)


def test_lradi_with_bicgstab_solves_the_dense_equation_and_theorem2(micro):
    p = micro
    A, B = p.A.to_scipy(), p.B.to_scipy()
    Xd = kron_solve(A, B, p.f, p.g)
    res = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner="bicgstab", strategy="bl_mid",
                keep_inner_residuals=True)
    assert res.converged
    X = X_of(res)
    assert np.linalg.norm(X - Xd) <= 1e-5 * np.linalg.norm(Xd)
    nfg = np.linalg.norm(p.f @ p.g.T, 2)
    assert true_residual_norm2(A, B, p.f, p.g, res.Z, res.gamma, res.Y) <= 3 * p.tau * nfg
    # eq. (adi_res_inexact) with the BiCGstab residuals
    G = np.diag(res.gamma)
    R = dense_residual(A, B, p.f, p.g, X)
    rhs = res.w @ res.t.conj().T - res.S_A @ G @ res.Y.conj().T - res.Z @ G @ res.S_B.conj().T
    assert np.linalg.norm(R - rhs) <= 1e-10 * np.linalg.norm(R) + 1e-14
    # every inner solve met its per-column target delta / r (the achieved
    # block norms are at most the requested block tolerances)
    for h in res.history:
        assert h["okA"] and h["okB"]
        assert h["nrA"] <= h["dA"] * (1 + 1e-12) and h["nrB"] <= h["dB"] * (1 + 1e-12)


def test_bicgstab_dynamic_tolerances_keep_exact_outer_count_and_save_inner_steps(small):
    """Table 2 with the paper's inner solver: the dynamic rule takes the
    outer steps of exact solves and fewer BiCGstab steps than fixed
    tolerances."""
    p = small
    ex = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner="direct")
    fx = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner="bicgstab", strategy="fixed")
    dy = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner="bicgstab", strategy="nobl_mid")
    assert ex.converged and fx.converged and dy.converged
    assert abs(dy.steps - ex.steps) <= 1 and abs(fx.steps - ex.steps) <= 1
    assert dy.inner_its_A + dy.inner_its_B < fx.inner_its_A + fx.inner_its_B
    # relaxation: the requested tolerances grow over the run (Fig. 3)
    assert dy.history[-1]["dA"] > 100 * dy.history[0]["dA"]


def test_select_direct_lies_on_the_admissible_curve():
    """With delta = 0 on the direct side the selected tolerance is the point
    of eq. (tolBfromtolA) on the curve: delta^B N_w = hat-eps (A direct),
    delta^A N_t = hat-eps (B direct), unless clamped by eq. (bound_tols)."""
    eh, Nw, Nt = 3e-12, 0.7, 0.2
    dA, dB = ctl.select_direct("A", eh, Nw, Nt, 1e-15, 1.0, 1e-15, 1.0)
    assert dA == 0.0 and dB == pytest.approx(eh / Nw, rel=1e-15)
    assert 0.0 * Nt + dB * Nw + 2 * 0.0 * dB == pytest.approx(eh, rel=1e-15)
    dA, dB = ctl.select_direct("B", eh, Nw, Nt, 1e-15, 1.0, 1e-15, 1.0)
    assert dB == 0.0 and dA == pytest.approx(eh / Nt, rel=1e-15)
    # clamped to delta_min
    _, dB = ctl.select_direct("A", eh, Nw, Nt, 1e-15, 1.0, 1e-9, 1.0)
    assert dB == 1e-9
    with pytest.raises(ValueError):
        ctl.select_direct("C", eh, Nw, Nt, 0, 1, 0, 1)


@pytest.mark.parametrize("iterative", ["gmres", "bicgstab"])
def test_one_side_direct(small, iterative):
    """Sec. 3.3 and the paper's Ex. 3: A-side systems solved directly, the
    B side iteratively with ||r^B_k|| <= hat-eps_k / ||w_{k-1}||.  The run
    converges with the outer steps of exact solves, the A-side residuals are
    at rounding level, the B-side tolerance follows the simplified rule at
    every step, and the B side needs fewer inner steps than with the fixed
    tolerance."""
    p = small
    ex = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner="direct")
    dy = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner_A="direct", inner_B=iterative,
               strategy="bl_mid", jacobi=True)
    fx = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner_A="direct", inner_B=iterative,
               strategy="fixed", jacobi=True)
    assert dy.converged and fx.converged
    assert abs(dy.steps - ex.steps) <= 1
    assert dy.inner_its_A == 0 and dy.inner_its_B < fx.inner_its_B
    eps = p.tau * np.linalg.norm(p.f @ p.g.T, 2)
    kmax = 50
    u = v = 0.0
    for h in dy.history:
        assert h["dA"] == 0.0
        assert h["nrA"] <= 1e-10 * h["N_w"]
        eh = ctl.eps_hat_bl(eps, int(h["k"]), kmax, u, v, 1.0)
        want = max(min(eh / h["N_w"], 0.1), p.tau / 20)
        assert h["dB"] == pytest.approx(want, rel=1e-12)
        assert h["nrB"] <= h["dB"] * (1 + 1e-12)
        u, v = h["u"], h["v"]
    A, B = p.A.to_scipy(), p.B.to_scipy()
    assert true_residual_norm2(A, B, p.f, p.g, dy.Z, dy.gamma, dy.Y) <= 3 * eps


# ---------------------------------------------------------------- initial guesses

def test_initial_guess_is_used_by_both_solvers():
    """x0 = the exact solution: no step is taken and x0 is returned; a
    nonzero x0 elsewhere still reaches the tolerance (the cycles solve for the
    correction from b - (S + sigma I) x0)."""
    p = W.problem_config("tiny2d")
    S = p.A.to_scipy()
    n = S.shape[0]
    sigma = -40.0
    b = np.random.default_rng(2).standard_normal(n)
    xs = spla.spsolve((S + sigma * sp.identity(n)).tocsc(), b)
    for solve in (lambda x0: gmres(S, sigma, b, 1e-10, 30, 500, True, "cgs2", x0=x0),
                  lambda x0: gmres(S, sigma, b, 1e-10, 30, 500, True, "dcgs2", x0=x0),
                  lambda x0: bicgstab(S, sigma, b, 1e-10, 500, True, x0=x0)):
        r = solve(xs)
        assert r.iters == 0 and np.array_equal(r.x, xs)
        r = solve(0.5 * xs)
        assert r.converged and np.linalg.norm(b - shifted_apply(S, sigma, r.x)) <= 1e-10


def test_recycled_guess_minimises_the_residual_over_the_previous_solution():
    """recycled_guess(c u): the residual b - c v (v = (S + sigma I) u) is
    orthogonal to v, and no other multiple of u has a smaller residual."""
    from oracle.lradi import recycled_guess
    p = W.problem_config("tiny2d")
    S = p.A.to_scipy()
    n = S.shape[0]
    rng = np.random.default_rng(5)
    b, u = rng.standard_normal(n), rng.standard_normal(n)
    sigma = -30.0 + 7.0j
    x0 = recycled_guess(S, sigma, b.astype(complex), u.astype(complex))
    v = shifted_apply(S, sigma, u.astype(complex))
    res = b - shifted_apply(S, sigma, x0)
    assert abs(np.vdot(v, res)) <= 1e-12 * np.linalg.norm(v) * np.linalg.norm(b)
    c = np.vdot(v, b) / np.vdot(v, v)
    for d in (1e-3, -1e-3, 1e-3j):
        assert np.linalg.norm(b - (c + d) * v) > np.linalg.norm(res)
    assert not recycled_guess(S, sigma, b, np.zeros(n)).any()


@pytest.mark.parametrize("inner", ["gmres", "bicgstab"])
def test_recycled_initial_guesses_keep_the_solution(inner):
    """With recycle="prev" the inner solves start from the recycled guess; the
    outer steps and the solution are those of x0 = 0 (within the inexactness),
    and with direct solves the option changes nothing."""
    p = W.problem_config("small2d")
    a = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy="nobl_mid", jacobi=True, inner=inner)
    b = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy="nobl_mid", jacobi=True, inner=inner,
              recycle="prev")
    assert a.converged and b.converged and a.steps == b.steps
    Xa = (a.Z * a.gamma[None, :]) @ a.Y.conj().T
    Xb = (b.Z * b.gamma[None, :]) @ b.Y.conj().T
    assert np.linalg.norm(Xa - Xb) <= 1e-6 * np.linalg.norm(Xa)
    d1 = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner="direct", kmax=6)
    d2 = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner="direct", kmax=6, recycle="prev")
    assert np.array_equal(d1.Z, d2.Z) and np.array_equal(d1.Y, d2.Y)
