"""Pins of the CPU oracle against what the paper and the mathematics fix.

Closed forms (diagonal A, B; one exact ADI step), two independent dense
solutions of eq. (sylv), the residual factorisation of eq. (adi_resexact),
the identities of Theorem 1 (eq. (adi_AZ_BTY)) and Theorem 2
(eq. (adi_res_inexact)), the Sylvester equation solved by Gamma (proof of
Theorem 2), the residual-gap bound behind eq. (upd_resgap), the geometry of
the admissible tolerances (eq. (relax_AB), (tolBfromtolA), Fig. 1), GMRES
facts, and the qualitative results of Table 2.  Mutated inputs (transposed
operand, sign error) must fail the same checks.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2312_02891_gb300 import workloads as W
from oracle import controller as ctl
from oracle.dense import bartels_stewart, dense_residual, kron_solve
from oracle.gmres import arnoldi_dcgs2, cgs2_step, gmres, mgs_step
from oracle.lradi import lradi
from oracle.residual import (block_norm2, factored_diff_fro, factored_fro, lowrank_fro,
                             lowrank_norm2, true_residual_norm2)


@pytest.fixture(scope="module")
def tiny():
    return W.problem_config("tiny2d")


@pytest.fixture(scope="module")
def micro():
    """n = 64, m = 49, r = 2: small enough for the n*m Kronecker system."""
    return W.make_problem("micro", 8, 2, "xy", 10.0, 7, 2, "rot2", 5.0, 2, 3, 8)


@pytest.fixture(scope="module")
def small():
    return W.problem_config("small2d")


def X_of(res):
    return (res.Z * res.gamma[None, :]) @ res.Y.conj().T


# ---------------------------------------------------------------- closed forms

def test_diagonal_closed_form():
    """A = diag(a), B = diag(b): X_ij = -f_i g_j / (a_i + b_j) (eq. (sylv))."""
    rng = np.random.default_rng(0)
    n, m = 30, 20
    a = -rng.uniform(1, 50, n)
    b = -rng.uniform(1, 50, m)
    f = rng.standard_normal((n, 1))
    g = rng.standard_normal((m, 1))
    X = -(f @ g.T) / (a[:, None] + b[None, :])
    A, B = sp.diags(a).tocsr(), sp.diags(b).tocsr()
    assert np.allclose(kron_solve(A, B, f, g), X, rtol=1e-12, atol=0)
    assert np.allclose(bartels_stewart(A, B, f, g), X, rtol=1e-10, atol=0)
    # LR-ADI with exact solves and the eigenvalues as shifts is exact after
    # min(n, m) steps on the shared spectrum; here use 12 greedy shifts
    alpha, beta = W.select_shift_pairs(a, b, 12)
    res = lradi(A, B, f, g, alpha, beta, 1e-10, inner="direct", kmax=200)
    assert res.converged
    assert np.linalg.norm(X_of(res) - X) <= 1e-8 * np.linalg.norm(X)


def test_one_exact_step_scalar():
    """n = m = 1, alpha = a, beta = b: one step gives X = -fg/(a+b) exactly,
    which fixes gamma_k = -(beta_k + alpha_k) and the shift placement
    (A + beta I), (B + alpha I)^* of Algorithm 1."""
    a, b, fv, gv = -3.0, -7.0, 2.0, 0.5
    A, B = sp.csr_matrix([[a]]), sp.csr_matrix([[b]])
    f, g = np.array([[fv]]), np.array([[gv]])
    res = lradi(A, B, f, g, [a], [b], 1e-12, inner="direct")
    assert res.steps == 1 and res.converged
    assert X_of(res)[0, 0] == pytest.approx(-fv * gv / (a + b), rel=1e-15)
    assert res.gamma[0] == pytest.approx(-(a + b))
    assert abs(res.w[0, 0]) < 1e-15 and abs(res.t[0, 0]) < 1e-15
    # shifts in swapped roles (linres as printed) would not be exact in one step
    bad = lradi(A, B, f, g, [b], [a], 1e-12, inner="direct", kmax=1)
    assert abs(X_of(bad)[0, 0] - (-fv * gv / (a + b))) > 1e-3


# --------------------------------------------------------- dense definitions

def test_kron_and_bartels_stewart_agree(micro):
    A, B = micro.A.to_scipy(), micro.B.to_scipy()
    X1 = kron_solve(A, B, micro.f, micro.g)
    X2 = bartels_stewart(A, B, micro.f, micro.g)
    assert np.linalg.norm(X1 - X2) <= 1e-10 * np.linalg.norm(X1)
    R = dense_residual(A, B, micro.f, micro.g, X1)
    assert np.linalg.norm(R) <= 1e-11 * np.linalg.norm(micro.f @ micro.g.T) * 1e3


@pytest.mark.parametrize("strategy", ["direct", "bl_mid", "nobl_mid", "fixed"])
def test_lradi_converges_to_dense_solution(tiny, micro, strategy):
    A, B = micro.A.to_scipy(), micro.B.to_scipy()
    Xk = kron_solve(A, B, micro.f, micro.g)
    kw = dict(inner="direct") if strategy == "direct" else dict(strategy=strategy)
    res = lradi(micro.A, micro.B, micro.f, micro.g, micro.alpha, micro.beta, micro.tau, **kw)
    assert res.converged
    assert np.linalg.norm(X_of(res) - Xk) <= 1e-5 * np.linalg.norm(Xk)
    A, B = tiny.A.to_scipy(), tiny.B.to_scipy()
    X = bartels_stewart(A, B, tiny.f, tiny.g)
    kw = dict(inner="direct") if strategy == "direct" else dict(strategy=strategy)
    res = lradi(tiny.A, tiny.B, tiny.f, tiny.g, tiny.alpha, tiny.beta, tiny.tau, **kw)
    assert res.converged and res.res_comp < tiny.tau
    nfg = lowrank_norm2(tiny.f, tiny.g)
    tr = np.linalg.norm(dense_residual(A, B, tiny.f, tiny.g, X_of(res)), 2) / nfg
    assert tr < 2e-8
    assert np.linalg.norm(X_of(res) - X) <= 1e-5 * np.linalg.norm(X)


def test_small2d_matches_bartels_stewart(small):
    X = bartels_stewart(small.A.to_scipy(), small.B.to_scipy(), small.f, small.g)
    for kw in (dict(inner="direct"), dict(strategy="nobl_mid")):
        res = lradi(small.A, small.B, small.f, small.g, small.alpha, small.beta, small.tau, **kw)
        assert np.linalg.norm(X_of(res) - X) <= 1e-6 * np.linalg.norm(X)


@pytest.mark.parametrize("mutation", ["transpose_B", "negate_g"])
def test_mutated_inputs_fail_the_dense_check(micro, mutation):
    """The checks above are sensitive: a transposed operand or a sign error in
    the right-hand side moves X far from the dense solution of the original
    equation."""
    tiny = micro
    A, B = tiny.A.to_scipy(), tiny.B.to_scipy()
    X = kron_solve(A, B, tiny.f, tiny.g)
    args = dict(A=tiny.A, B=tiny.B, f=tiny.f, g=tiny.g, alpha=tiny.alpha, beta=tiny.beta)
    if mutation == "transpose_B":
        args["B"] = B.T.tocsr()
    else:
        args["g"] = -tiny.g
    res = lradi(tau=tiny.tau, inner="direct", kmax=60, **args)
    assert np.linalg.norm(X_of(res) - X) > 1e-3 * np.linalg.norm(X)


# ----------------------------------------------------------- exact identities

def test_residual_factorisation_exact_solves(small):
    """eq. (adi_resexact): with exact solves R_k = w_k t_k^*."""
    A, B = small.A.to_scipy(), small.B.to_scipy()
    res = lradi(small.A, small.B, small.f, small.g, small.alpha, small.beta, small.tau,
                inner="direct", kmax=6)
    R = dense_residual(A, B, small.f, small.g, X_of(res))
    assert np.linalg.norm(R - res.w @ res.t.conj().T, 2) <= 1e-11 * np.linalg.norm(R, 2)


def _sigma(vals, gam, r):
    k = len(vals)
    S = np.zeros((k, k), dtype=np.result_type(vals, gam))
    for i in range(k):
        S[i, i] = vals[i]
        S[i, :i] = -gam[i]
    return np.kron(S, np.eye(r))


def test_theorem1_and_2_inexact(tiny):
    """eq. (adi_AZ_BTY) and eq. (adi_res_inexact) with the inner residuals
    S^A, S^B of GMRES solves stopped at the dynamic tolerances."""
    res = lradi(tiny.A, tiny.B, tiny.f, tiny.g, tiny.alpha, tiny.beta, tiny.tau,
                strategy="bl_mid", keep_inner_residuals=True)
    A, B = tiny.A.to_scipy().toarray(), tiny.B.to_scipy().toarray()
    r, k = tiny.r, res.steps
    L = len(tiny.alpha)
    al = np.array([tiny.alpha[i % L] for i in range(k)])
    be = np.array([tiny.beta[i % L] for i in range(k)])
    gam = -(al + be)
    E = np.kron(np.ones((k, 1)), np.eye(r))
    lhs = A @ res.Z
    rhs = res.Z @ _sigma(al, gam, r) + res.w @ E.T - res.S_A
    assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(lhs)
    lhsB = B.T @ res.Y
    rhsB = res.Y @ _sigma(np.conj(be), np.conj(gam), r) + res.t @ E.T - res.S_B
    assert np.linalg.norm(lhsB - rhsB) <= 1e-10 * np.linalg.norm(lhsB)
    # Theorem 2: R_true = w t^* - S^A Gamma Y^* - Z Gamma (S^B)^*
    G = np.diag(res.gamma)
    R = dense_residual(A, B, tiny.f, tiny.g, X_of(res))
    rhs2 = res.w @ res.t.conj().T - res.S_A @ G @ res.Y.conj().T - res.Z @ G @ res.S_B.conj().T
    assert np.linalg.norm(R - rhs2) <= 1e-10 * np.linalg.norm(R) + 1e-14
    # Gamma solves sigma^alpha Gamma + Gamma (sigma^beta)^* + gamma gamma^T = 0
    gv = np.kron(gam[:, None], np.eye(r))
    M = _sigma(al, gam, r) @ G + G @ _sigma(np.conj(be), np.conj(gam), r).conj().T + gv @ gv.T
    assert np.linalg.norm(M) <= 1e-12 * np.linalg.norm(gv @ gv.T)
    # residual gap bounded by the back-looking estimates (eq. (ADIresgapbound1), (upd_resgap))
    gap = np.linalg.norm(res.S_A @ G @ res.Y.conj().T + res.Z @ G @ res.S_B.conj().T, 2)
    assert gap <= res.history[-1]["u"] + res.history[-1]["v"] + 1e-20


def test_lowrank_norms_match_dense_complex():
    """The factored norms with complex factors and a complex core (conjugate
    transposes, not transposes): ||U W^*||_2 and the residual of
    X = Z diag(gamma) Y^* against the dense matrices."""
    rng = np.random.default_rng(9)
    U = rng.standard_normal((30, 3)) + 1j * rng.standard_normal((30, 3))
    V = rng.standard_normal((20, 3)) + 1j * rng.standard_normal((20, 3))
    assert lowrank_norm2(U, V) == pytest.approx(np.linalg.norm(U @ V.conj().T, 2), rel=1e-12)
    assert lowrank_fro(U, V) == pytest.approx(np.linalg.norm(U @ V.conj().T), rel=1e-12)
    n, m, k, r = 12, 9, 4, 2
    A = sp.csr_matrix(rng.standard_normal((n, n)))
    B = sp.csr_matrix(rng.standard_normal((m, m)))
    f, g = rng.standard_normal((n, r)), rng.standard_normal((m, r))
    Z = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    Y = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    gam = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    X = (Z * gam[None, :]) @ Y.conj().T
    R = A @ X + X @ B + f @ g.conj().T
    assert true_residual_norm2(A, B, f, g, Z, gam, Y) == pytest.approx(np.linalg.norm(R, 2), rel=1e-10)


def test_inner_solves_meet_the_per_column_target(tiny):
    """Sec. 3.3: each of the r column systems of a step is solved to
    delta_k / r (so that the n x r block residual meets delta_k); the stored
    inner residuals of every converged solve satisfy it column by column."""
    r = tiny.r
    res = lradi(tiny.A, tiny.B, tiny.f, tiny.g, tiny.alpha, tiny.beta, tiny.tau, strategy="nobl_mid",
                keep_inner_residuals=True)
    for k, h in enumerate(res.history):
        for S, d, ok in ((res.S_A, h["dA"], h["okA"]), (res.S_B, h["dB"], h["okB"])):
            assert ok
            cols = np.linalg.norm(S[:, k * r:(k + 1) * r], axis=0)
            assert np.all(cols <= d / r * (1 + 1e-10)), (k, cols, d / r)


def test_sampled_residual_matches_dense(tiny):
    from oracle.residual import sampled_residual
    res = lradi(tiny.A, tiny.B, tiny.f, tiny.g, tiny.alpha, tiny.beta, tiny.tau, strategy="bl_mid", kmax=4)
    A, B = tiny.A.to_scipy(), tiny.B.to_scipy()
    R = dense_residual(A, B, tiny.f, tiny.g, X_of(res))
    rows, cols = np.array([0, 5, 17, 143]), np.array([0, 3, 50, 99])
    S = sampled_residual(A, B, tiny.f, tiny.g, res.Z, res.gamma, res.Y, rows, cols)
    assert np.allclose(S, R[np.ix_(rows, cols)], rtol=1e-12, atol=1e-14 * np.abs(R).max())


def test_lowrank_norms_match_dense(tiny):
    rng = np.random.default_rng(4)
    U, V = rng.standard_normal((50, 3)), rng.standard_normal((40, 3))
    assert lowrank_norm2(U, V) == pytest.approx(np.linalg.norm(U @ V.T, 2), rel=1e-12)
    assert lowrank_fro(U, V) == pytest.approx(np.linalg.norm(U @ V.T), rel=1e-12)
    assert block_norm2(U) == pytest.approx(np.linalg.svd(U, compute_uv=False)[0], rel=1e-14)
    res = lradi(tiny.A, tiny.B, tiny.f, tiny.g, tiny.alpha, tiny.beta, tiny.tau, strategy="bl_mid")
    A, B = tiny.A.to_scipy(), tiny.B.to_scipy()
    R = dense_residual(A, B, tiny.f, tiny.g, X_of(res))
    assert true_residual_norm2(A, B, tiny.f, tiny.g, res.Z, res.gamma, res.Y) == pytest.approx(
        np.linalg.norm(R, 2), rel=1e-8)
    res2 = lradi(tiny.A, tiny.B, tiny.f, tiny.g, tiny.alpha, tiny.beta, tiny.tau, inner="direct")
    d = factored_diff_fro(res.Z, res.gamma, res.Y, res2.Z, res2.gamma, res2.Y)
    assert d == pytest.approx(np.linalg.norm(X_of(res) - X_of(res2)), rel=1e-6)
    assert factored_fro(res.Z, res.gamma, res.Y) == pytest.approx(np.linalg.norm(X_of(res)), rel=1e-12)


# ------------------------------------------------------------------ controller

def test_controller_constants():
    # c = 2 + sqrt(2), c^2 = 6 + 4 sqrt(2) = 11.656854...
    assert ctl.C_BOUND ** 2 == pytest.approx(11.65685424949238, rel=1e-15)
    # eps = 1e-8, kmax = 50, xi = 1: 1e-8 / (2 * 11.65685... * 50) = 8.5786437627e-12
    assert ctl.eps_hat_nobl(1e-8, 50) == pytest.approx(8.578643762690485e-12, rel=1e-14)
    # back-looking with u = v = 0 at k = 1 coincides with the plain rule
    assert ctl.eps_hat_bl(1e-8, 1, 50, 0.0, 0.0) == pytest.approx(ctl.eps_hat_nobl(1e-8, 50), rel=1e-15)
    # literal |.|: a budget exceeded by u + v gives back a positive value
    assert ctl.eps_hat_bl(1e-8, 1, 50, 1e-9, 0.0) > 0


def test_back_looking_target_beyond_the_first_step():
    """eq. (ADI_relax2_prak) at k > 1 with u, v > 0, under and over budget.

    c = 2 + sqrt(2) = 3.414213562373095, so 2 c kmax = 341.4213562373095 for
    kmax = 50 and 136.5685424949238 for kmax = 20; the budget is
    xi k eps / (2 c kmax) and hat-eps = |budget - u - v| / c."""
    # k = 10, eps = 1e-8, xi = 1, u = 1e-11, v = 2e-11 (under budget):
    # budget = 1e-7 / 341.4213562373095 = 2.9289321881345246e-10,
    # budget - u - v = 2.6289321881345246e-10, / c = 7.699964106250138e-11
    assert ctl.eps_hat_bl(1e-8, 10, 50, 1e-11, 2e-11) == pytest.approx(7.699964106250138e-11, rel=1e-13)
    # k = 2, u = 5e-11, v = 3e-11 (over budget): budget = 2e-8 / 341.42... =
    # 5.85786437626905e-11, budget - u - v = -2.14213562373095e-11; the
    # literal |.| gives 2.14213562373095e-11 / c = 6.2741699796952045e-12
    assert ctl.eps_hat_bl(1e-8, 2, 50, 5e-11, 3e-11) == pytest.approx(6.2741699796952045e-12, rel=1e-12)
    # xi = 0.5, k = 4, kmax = 20, eps = 2e-9, u = 1e-12, v = 0:
    # budget = 0.5 * 4 * 2e-9 / 136.5685424949238 = 2.928932188134525e-11,
    # minus 1e-12 = 2.828932188134525e-11, / c = 8.285750543877043e-12
    assert ctl.eps_hat_bl(2e-9, 4, 20, 1e-12, 0.0, xi=0.5) == pytest.approx(8.285750543877043e-12, rel=1e-13)
    # the same through the controller entry point, which feeds eq. (simple_tols)
    _, _, eh = ctl.inner_tolerances("bl_mid", k=10, kmax=50, eps=1e-8, xi=1.0, u_prev=1e-11, v_prev=2e-11,
                                    N_w=1.0, N_t=1.0, dmin_A=1e-12, dmax_A=0.1, dmin_B=1e-12, dmax_B=0.1,
                                    fixed_tol=5e-10)
    assert eh == pytest.approx(7.699964106250138e-11, rel=1e-13)


def test_pair_detection():
    """A conjugate pair is a shift (alpha, beta), not both real, followed by
    (conj alpha, conj beta): both members must be conjugate, and the last
    shift of the list opens no pair."""
    from oracle.lradi import _is_pair_start
    a = np.array([-1 + 2j, -1 - 2j, -3.0, -3.0])
    assert _is_pair_start(a, np.array([-2 + 1j, -2 - 1j, -4.0, -4.0]), 0)
    assert _is_pair_start(a, np.array([-2.0, -2.0, -4.0, -4.0]), 0)       # real beta, complex alpha
    assert not _is_pair_start(a, np.array([-2 + 1j, -2 + 1j, -4.0, -4.0]), 0)
    assert not _is_pair_start(a, np.array([-2.0, -5.0, -4.0, -4.0]), 0)
    assert not _is_pair_start(a, np.array([-2.0, -2.0, -4.0, -4.0]), 2)   # both real
    assert not _is_pair_start(np.array([-1.0, -1 + 2j]), np.array([-2.0, -2 + 1j]), 1)


def test_selection_rules_hand_values():
    """eq. (simple_tols), eq. (one_side) and its mirror, and the fixed rule
    with a directly solved side, on numbers worked by hand (hat-eps = 1e-6,
    ||w|| = 2, ||t|| = 4, delta_max = 0.1)."""
    e, Nw, Nt = 1e-6, 2.0, 4.0
    # mid, delta_min = 5e-8 on both sides: delta^A = (min(0.1, 1e-6 / 4) - 5e-8) / 2
    # = (2.5e-7 - 5e-8) / 2 = 1e-7 (the literal midpoint: minus delta_min);
    # delta^B on the curve: (1e-6 - 1e-7 * 4) / (2 * 1e-7 + 2) = 6e-7 / 2.0000002
    # = 2.99999970000003e-7
    dA, dB = ctl.select_mid(e, Nw, Nt, 5e-8, 0.1, 5e-8, 0.1)
    assert dA == pytest.approx(1e-7, rel=1e-14)
    assert dB == pytest.approx(2.9999997000000295e-07, rel=1e-13)
    # B preferred, delta^A_min = 3e-7, delta^B_min = 1e-9: delta^B = 1e-9; delta^A on
    # the curve (1e-6 - 1e-9 * 2) / (2e-9 + 4) = 2.49499999875e-7, below
    # delta^A_min, so the clamp of eq. (bound_tols) on the A side gives 3e-7
    dA, dB = ctl.select_prefer_B(e, Nw, Nt, 3e-7, 0.1, 1e-9, 0.1)
    assert dB == 1e-9 and dA == pytest.approx(3e-7, rel=1e-15)
    dA, dB = ctl.select_prefer_B(e, Nw, Nt, 1e-9, 0.1, 1e-9, 0.1)
    assert dA == pytest.approx(2.4949999987525e-07, rel=1e-13)
    # fixed tolerances with one side solved directly: that side's tolerance is 0
    kw = dict(k=3, kmax=50, eps=1e-8, xi=1.0, u_prev=0.0, v_prev=0.0, N_w=Nw, N_t=Nt, dmin_A=1e-9,
              dmax_A=0.1, dmin_B=1e-9, dmax_B=0.1, fixed_tol=5e-10)
    assert ctl.inner_tolerances("fixed", direct="A", **kw)[:2] == (0.0, 5e-10)
    assert ctl.inner_tolerances("fixed", direct="B", **kw)[:2] == (5e-10, 0.0)
    assert ctl.inner_tolerances("fixed", **kw)[:2] == (5e-10, 5e-10)


def test_fig1_axis_values():
    """Fig. 1 (c = 3, eps = 1e-8, ||t|| = 1e-5, ||w|| = 2e-3): the curve
    Psi = 0 meets the axes at eps/(c ||w||) and eps/(c ||t||)."""
    c, e, Nt, Nw = 3.0, 1e-8, 1e-5, 2e-3
    assert ctl.tol_B_from_A(e / c, 0.0, Nw, Nt) == pytest.approx(1.6666666666666667e-06, rel=1e-14)
    assert ctl.tol_B_from_A(e / c, 3.3333333333333335e-04, Nw, Nt) == pytest.approx(0.0, abs=1e-20)
    assert ctl.tol_A_from_B(e / c, 0.0, Nw, Nt) == pytest.approx(3.3333333333333335e-04, rel=1e-14)


def test_mid_selection_lies_on_the_admissible_curve():
    """Unclamped, (delta^A, delta^B) satisfies eq. (ADI_relax1_prak) with
    equality: dA ||t|| + dB ||w|| + 2 dA dB = hat-eps (eq. (relax_AB))."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        eh = 10 ** rng.uniform(-12, -8)
        Nw, Nt = 10 ** rng.uniform(-4, 0, 2)
        dA, dB = ctl.select_mid(eh, Nw, Nt, 1e-30, 1.0, 1e-30, 1.0)
        assert dA == pytest.approx(0.5 * (eh / Nt - 1e-30))
        assert dA * Nt + dB * Nw + 2 * dA * dB == pytest.approx(eh, rel=1e-12)
        a1, b1 = ctl.select_prefer_A(eh, Nw, Nt, 1e-14, 1.0, 1e-30, 1.0)
        assert a1 == 1e-14 and a1 * Nt + b1 * Nw + 2 * a1 * b1 == pytest.approx(eh, rel=1e-12)
        a2, b2 = ctl.select_prefer_B(eh, Nw, Nt, 1e-30, 1.0, 1e-14, 1.0)
        assert b2 == 1e-14 and a2 * Nt + b2 * Nw + 2 * a2 * b2 == pytest.approx(eh, rel=1e-12)
    # clamps of eq. (bound_tols)
    dA, dB = ctl.select_mid(1e-30, 1.0, 1.0, 1e-10, 0.1, 2e-10, 0.1)
    assert dA == 1e-10 and dB == 2e-10
    dA, dB = ctl.select_mid(10.0, 1e-6, 1e-6, 1e-10, 0.1, 2e-10, 0.05)
    assert dA == pytest.approx(0.5 * (0.1 - 1e-10)) and dB == 0.05


def test_theorem3_bound_on_a_run(tiny):
    """With tolerances obeying eq. (ADI_relax1_theo) for c = check-c_k computed
    exactly, the residual gap after kmax steps is at most eps (Theorem 3)."""
    A, B = tiny.A.to_scipy().toarray(), tiny.B.to_scipy().toarray()
    n, m, r = A.shape[0], B.shape[0], tiny.r
    L = len(tiny.alpha)
    kmax = 8
    eps = 1e-9
    f, g = tiny.f, tiny.g
    w, t = f.copy(), g.copy()
    Z, Y, gl, SA, SB = [], [], [], [], []
    for k in range(kmax):
        a, b = tiny.alpha[k % L], tiny.beta[k % L]
        CA = (A - a * np.eye(n)) @ np.linalg.inv(A + b * np.eye(n))
        CB = (B - b * np.eye(m)) @ np.linalg.inv(B + a * np.eye(m))
        cc = max(np.linalg.norm(CA, 2), np.linalg.norm(CB, 2)) + 1
        Nw, Nt = block_norm2(w), block_norm2(t)
        dA, dB = ctl.select_mid(eps / kmax / cc, Nw, Nt, 1e-300, 1.0, 1e-300, 1.0)
        z = np.zeros((n, r)); y = np.zeros((m, r))
        for l in range(r):
            z[:, l] = gmres(sp.csr_matrix(A), b, w[:, l], dA / r, 30, 5000).x
            y[:, l] = gmres(sp.csr_matrix(B.T), a, t[:, l], dB / r, 30, 5000).x
        rA = w - (A + b * np.eye(n)) @ z
        rB = t - (B.T + a * np.eye(m)) @ y
        assert cc * (block_norm2(rA) * Nt + block_norm2(rB) * Nw + 2 * block_norm2(rA) * block_norm2(rB)) <= eps / kmax * (1 + 1e-9)
        gm = -(a + b)
        w, t = w + gm * z, t + gm * y
        Z.append(z); Y.append(y); gl += [gm] * r; SA.append(rA); SB.append(rB)
    G = np.diag(gl)
    gap = np.hstack(SA) @ G @ np.hstack(Y).T + np.hstack(Z) @ G @ np.hstack(SB).T
    assert np.linalg.norm(gap, 2) <= eps


# ----------------------------------------------------------------------- GMRES

def test_gmres_exact_krylov_dimension():
    """SPD tridiagonal, restart >= n: GMRES terminates in at most n steps."""
    n = 20
    T = sp.diags([-np.ones(n - 1), 2.5 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    b = np.random.default_rng(2).standard_normal(n)
    res = gmres(T, 0.0, b, 1e-12, restart=30, max_iters=100)
    assert res.converged and res.iters <= n and res.cycles == 1
    assert np.allclose(res.x, spla.spsolve(T.tocsc(), b), rtol=1e-9)


@pytest.mark.parametrize("jacobi", [False, True])
@pytest.mark.parametrize("sigma", [-40.0, -40.0 + 25.0j])
def test_gmres_matches_sparse_solve(tiny, jacobi, sigma):
    S = tiny.A.to_scipy()
    n = S.shape[0]
    b = np.random.default_rng(3).standard_normal(n)
    res = gmres(S, sigma, b, 1e-10, restart=10, max_iters=5000, jacobi=jacobi)
    xs = spla.spsolve((S + sigma * sp.eye(n)).tocsc(), b.astype(np.result_type(sigma, b)))
    assert res.converged
    assert np.linalg.norm(b - (S @ res.x + sigma * res.x)) <= 1e-10
    assert np.linalg.norm(res.x - xs) <= 1e-7 * np.linalg.norm(xs)
    # residual estimates never increase within a cycle
    h = np.array(res.history[:10])
    assert np.all(np.diff(h) <= 1e-12 * h[0])
    res2 = gmres(S, sigma, b, 1e-10, restart=10, max_iters=5000, jacobi=jacobi, ortho="mgs")
    assert abs(res2.iters - res.iters) <= 1


def test_cgs2_and_mgs_orthogonalise():
    rng = np.random.default_rng(9)
    V, _ = np.linalg.qr(rng.standard_normal((200, 12)))
    w = rng.standard_normal(200)
    for step in (cgs2_step, mgs_step):
        h, w2 = step(V.T.copy(), w.copy())
        assert np.allclose(h, V.T @ w, atol=1e-13)
        assert np.linalg.norm(V.T @ w2) <= 1e-13 * np.linalg.norm(w)
        assert np.allclose(V @ h + w2, w, atol=1e-13)


# --------------------------------------------------- qualitative (Table 2)

def test_dynamic_tolerances_keep_exact_outer_count_and_save_inner_steps(small):
    direct = lradi(small.A, small.B, small.f, small.g, small.alpha, small.beta, small.tau, inner="direct")
    fixed = lradi(small.A, small.B, small.f, small.g, small.alpha, small.beta, small.tau, strategy="fixed")
    for s in ("bl_mid", "nobl_mid"):
        dyn = lradi(small.A, small.B, small.f, small.g, small.alpha, small.beta, small.tau, strategy=s)
        assert dyn.steps == direct.steps == fixed.steps
        assert dyn.inner_its_A + dyn.inner_its_B < fixed.inner_its_A + fixed.inner_its_B
        assert dyn.Z.shape[1] == dyn.steps * small.r      # dim = it_out * r (Table 2)
    # relaxation: the requested tolerances grow over the run (Fig. 3)
    dyn = lradi(small.A, small.B, small.f, small.g, small.alpha, small.beta, small.tau, strategy="nobl_mid")
    dA = [h["dA"] for h in dyn.history]
    assert dA[-1] > 100 * dA[0]


def test_zero_rhs_gives_zero_solution():
    p = W.problem_config("tiny2d")
    res = lradi(p.A, p.B, np.zeros_like(p.f), p.g, p.alpha, p.beta, p.tau)
    assert res.steps == 0 and res.Z.shape[1] == 0


def test_conjugate_pairs_give_real_solution():
    """Complex shift pairs used together with their conjugates give a real X
    after each pair (the complex formulation of Sec. 3.3)."""
    p = W.make_problem("cplx", 10, 2, "rot2", 60.0, 9, 2, "rot2", 40.0, 1, 5, 6, real_shifts=False)
    assert np.any(np.imag(p.alpha) != 0) or np.any(np.imag(p.beta) != 0)
    res = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner="direct")
    X = X_of(res)
    assert res.converged
    assert np.linalg.norm(X.imag) <= 1e-10 * np.linalg.norm(X.real)
    Xd = kron_solve(p.A.to_scipy(), p.B.to_scipy(), p.f, p.g)
    assert np.linalg.norm(X.real - Xd) <= 1e-6 * np.linalg.norm(Xd)


# ------------------------------------------------------------------- inputs

def test_generator_is_deterministic_and_normalised():
    f1, g1 = W.rhs_factors(100, 80, 2, 5)
    f2, g2 = W.rhs_factors(100, 80, 2, 5)
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    assert np.linalg.norm(f1, 2) == pytest.approx(1.0) and np.linalg.norm(g1, 2) == pytest.approx(1.0)
    z = W.normal(1, 1, 0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_convdiff_operator_structure():
    N = 6
    A = W.convdiff(N, 2, "xy", 0.0).to_scipy().toarray()
    h = 1.0 / (N + 1)
    # pure diffusion: A = -(1/h^2) (T kron I + I kron T), T = tridiag(-1, 2, -1)
    T = np.diag(2 * np.ones(N)) - np.diag(np.ones(N - 1), 1) - np.diag(np.ones(N - 1), -1)
    L = (np.kron(np.eye(N), T) + np.kron(T, np.eye(N))) / h ** 2
    assert np.allclose(A, -L)
    ev = np.linalg.eigvalsh(A)
    lam_min = 2 * (2 - 2 * math.cos(math.pi * h)) / h ** 2
    assert ev.max() == pytest.approx(-lam_min, rel=1e-12)
    # convection: skew part of the centred difference, stable spectrum
    C = W.convdiff(8, 3, "zxy", 30.0).to_scipy().toarray()
    assert np.all(np.linalg.eigvals(C).real < 0)
    assert W.convdiff(8, 3, "zxy", 30.0).nnz == 7 * 512 - 6 * 64


# ------------------------------------------------------ delayed CGS2 (DCGS2)

@pytest.mark.parametrize("sigma", [0.0, -3.0 + 7.0j])
def test_dcgs2_arnoldi_relation_and_orthonormality(sigma):
    """The delayed second pass and the recovered first-pass coefficients give
    an Arnoldi decomposition: Op V_k = V_{k+1} H_k with V orthonormal, to
    rounding, on a nonsymmetric operator (real and complex shift)."""
    A = W.convdiff(9, 2, "rot2", 40.0).to_scipy()
    op = lambda x: A @ x + sigma * x
    v0 = W.normal(3, 2, 0, A.shape[0]).astype(np.complex128 if sigma != 0 else np.float64)
    v0 = v0 / np.linalg.norm(v0)
    k = 30
    V, H, napply = arnoldi_dcgs2(op, v0, k)
    assert V.shape[0] == k + 1 and H.shape == (k + 1, k) and napply == k
    nA = spla.norm(A) + abs(sigma)
    AV = np.stack([op(V[i]) for i in range(k)])
    assert np.abs(AV.T - V.T @ H).max() <= 1e-12 * nA
    assert np.abs(V.conj() @ V.T - np.eye(k + 1)).max() <= 1e-12
    assert np.all(np.abs(np.tril(H, -2)) == 0)        # Hessenberg
    assert np.all(H[np.arange(1, k + 1), np.arange(k)].real > 0)


@pytest.mark.parametrize("cplx", [False, True])
def test_dcgs2_gmres_matches_cgs2_gmres(small, cplx):
    """Same Krylov spaces in exact arithmetic: the delayed variant takes the
    same number of steps and returns the same solution as CGS2 (small2d
    A-side system, with and without Jacobi, real and complex shift), and both
    match the sparse LU solution (a conjugation slip in either Givens update
    breaks the complex case)."""
    S = small.A.to_scipy()
    sig = small.beta[0] + (0.3j * abs(small.beta[0]) if cplx else 0.0)
    rhs = small.f[:, 0].astype(complex) if cplx else small.f[:, 0]
    x_lu = spla.spsolve((S + sig * sp.identity(S.shape[0])).tocsc(), rhs)
    for jac in (False, True):
        a = gmres(S, sig, rhs, 1e-10, 30, 3000, jac, "cgs2")
        b = gmres(S, sig, rhs, 1e-10, 30, 3000, jac, "dcgs2")
        assert a.converged and b.converged and a.iters == b.iters and a.cycles == b.cycles
        assert np.linalg.norm(a.x - b.x) <= 1e-12 * np.linalg.norm(a.x)
        assert np.allclose(a.history, b.history, rtol=1e-6)
        assert np.linalg.norm(a.x - x_lu) <= 1e-6 * np.linalg.norm(x_lu)
        # the Givens estimates are the true residual norms of the GMRES
        # iterates (right preconditioning): the last one below the tolerance
        assert a.history[-1] <= 1e-10 and b.history[-1] <= 1e-10


def test_dcgs2_gmres_diagonal_operator_exact_steps():
    """GMRES on a diagonal operator with d distinct entries converges in d
    steps (minimal polynomial), also with the delayed orthogonalisation."""
    d = np.repeat([-1.0, -2.0, -5.0, -9.0], 25)
    S = sp.diags(d).tocsr()
    b = W.normal(4, 1, 0, d.size)
    res = gmres(S, 0.0, b, 1e-10 * np.linalg.norm(b), 30, 100, False, "dcgs2")
    assert res.converged and res.iters == 4 and res.cycles == 1
    assert np.allclose(res.x, b / d)
