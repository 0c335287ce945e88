"""Pins of the oracle's generalized path, A X C + M X B = -f g^* (eq. (gsylv)).

Algorithm 1 with the inner systems (A + beta_k M) z = w_{k-1},
(B + alpha_k C)^* y = t_{k-1} and the updates w_k = w_{k-1} + gamma_k M z_k,
t_k = t_{k-1} + conj(gamma_k) C^* y_k (eq. (lradi_g)), checked against: the
Kronecker form of eq. (gsylv) and Bartels-Stewart on the equivalent standard
equation (a library routine); a one-step closed form for n = m = 1; the
residual factorisation of eq. (adi_resexact); the identities of Theorem 1
(eq. (adi_AZ_BTY)) and Theorem 2 (eq. (adi_res_inexact)) with M and C; the
residual-gap estimate of eq. (upd_resgap) with ||M z||, ||C^T y||.  The
standard path (M = C = I) must be reproduced exactly.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2312_02891_gb300 import workloads as W
from oracle.dense import bartels_stewart, dense_residual, kron_solve
from oracle.gmres import gmres
from oracle.lradi import lradi
from oracle.lradi_real import lradi_real
from oracle.residual import block_norm2, true_residual_norm2


@pytest.fixture(scope="module")
def micro_g():
    """n = 64, m = 49, r = 2: small enough for the n*m Kronecker system."""
    return W.make_problem_g("micro_g", 8, 2, "xy", 10.0, 7, 2, "rot2", 5.0, 2, 3, 8)


@pytest.fixture(scope="module")
def tiny_g():
    return W.problem_config("tiny2d_g")


def X_of(res):
    return (res.Z * res.gamma[None, :]) @ res.Y.conj().T


def mats(p):
    return p.A.to_scipy(), p.B.to_scipy(), p.M.to_scipy(), p.C.to_scipy()


def test_mass_matrix_structure():
    """Q1 consistent mass: symmetric positive definite, 9 nonzeros in an
    interior row, interior row sums h^2 (the integral of a hat function),
    eigenvalues in (h^2/9, h^2] (1D: (h/6) tridiag(1,4,1) has eigenvalues
    (h/6)(4 + 2 cos(k pi/(N+1))))."""
    N = 9
    h = 1.0 / (N + 1)
    M = W.mass_matrix(N, 2).to_scipy().toarray()
    assert np.array_equal(M, M.T)
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > h * h / 9 and ev.max() <= h * h * (1 + 1e-12)
    i = 4 * N + 4                      # node (4, 4): no boundary neighbour
    assert np.count_nonzero(M[i]) == 9
    assert M[i].sum() == pytest.approx(h * h, rel=1e-14)
    lam1 = (h / 6) * (4 + 2 * np.cos(np.arange(1, N + 1) * np.pi / (N + 1)))
    assert np.allclose(np.sort(ev), np.sort(np.outer(lam1, lam1).ravel()), rtol=1e-12)


def test_generalized_dense_solutions_agree(micro_g):
    """The Kronecker form of eq. (gsylv) and Bartels-Stewart on
    M^{-1} A X + X B C^{-1} = -M^{-1} f g^* C^{-1} give the same X, which
    solves eq. (gsylv)."""
    A, B, M, C = mats(micro_g)
    X1 = kron_solve(A, B, micro_g.f, micro_g.g, M, C)
    X2 = bartels_stewart(A, B, micro_g.f, micro_g.g, M, C)
    assert np.linalg.norm(X1 - X2) <= 1e-10 * np.linalg.norm(X1)
    R = dense_residual(A, B, micro_g.f, micro_g.g, X1, M, C)
    assert np.linalg.norm(R) <= 1e-10 * np.linalg.norm(micro_g.f @ micro_g.g.T)
    # M, C swapped (a transposed role) is a different equation
    Xs = kron_solve(A, B, micro_g.f, micro_g.g, None, None)
    assert np.linalg.norm(Xs - X1) > 1e-2 * np.linalg.norm(X1)


def test_one_exact_step_generalized_scalar():
    """n = m = 1: a x c + mu x b = -f g.  With alpha = a/mu and beta = b/c
    (the eigenvalues of the pencils (a, mu), (b, c)) one step gives
    X = -f g / (a c + mu b), w_1 = t_1 = 0: this fixes the shift placement
    (A + beta M), (B + alpha C)^*, gamma = -(alpha + beta) and the updates
    with M z and C^* y of eq. (lradi_g)."""
    a, b, mu, c, fv, gv = -3.0, -7.0, 0.5, 2.0, 2.0, 0.5
    A, B = sp.csr_matrix([[a]]), sp.csr_matrix([[b]])
    M, C = sp.csr_matrix([[mu]]), sp.csr_matrix([[c]])
    f, g = np.array([[fv]]), np.array([[gv]])
    res = lradi(A, B, f, g, [a / mu], [b / c], 1e-12, M=M, C=C, inner="direct")
    assert res.steps == 1 and res.converged
    assert X_of(res)[0, 0] == pytest.approx(-fv * gv / (a * c + mu * b), rel=1e-14)
    assert res.gamma[0] == pytest.approx(-(a / mu + b / c))
    assert abs(res.w[0, 0]) <= 1e-15 * abs(fv) and abs(res.t[0, 0]) <= 1e-15 * abs(gv)


def test_identity_mass_reproduces_the_standard_path(micro_g):
    """M = I, C = I given explicitly: the same run as without them."""
    p = micro_g
    I_n, I_m = sp.identity(p.A.n, format="csr"), sp.identity(p.B.n, format="csr")
    for inner in ("direct", "gmres"):
        r0 = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner=inner, kmax=6)
        r1 = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, M=I_n, C=I_m, inner=inner, kmax=6)
        assert r0.steps == r1.steps
        assert np.allclose(r0.Z, r1.Z, rtol=1e-13, atol=0) and np.allclose(r0.Y, r1.Y, rtol=1e-13, atol=0)


@pytest.mark.parametrize("inner,strategy", [("direct", "fixed"), ("gmres", "bl_mid"), ("gmres", "nobl_mid")])
def test_generalized_lradi_converges_to_dense_solution(micro_g, inner, strategy):
    p = micro_g
    A, B, M, C = mats(p)
    Xd = kron_solve(A, B, p.f, p.g, M, C)
    res = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, M=p.M, C=p.C, inner=inner,
                strategy=strategy, kmax=60)
    assert res.converged and res.res_comp < p.tau
    X = X_of(res)
    assert np.linalg.norm(X.imag if np.iscomplexobj(X) else 0) <= 1e-12 * np.linalg.norm(X)
    # the true residual of eq. (gsylv) is small (Cor. 1: within eps of the exact one)
    nfg = np.linalg.norm(p.f @ p.g.T, 2)
    Rn = true_residual_norm2(A, B, p.f, p.g, res.Z, res.gamma, res.Y, M, C)
    assert Rn <= 3 * p.tau * nfg
    assert np.linalg.norm(X - Xd) <= 1e-5 * np.linalg.norm(Xd)
    # the run on the standard equation (M, C dropped) solves a different equation
    if inner == "direct":
        r0 = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner=inner, kmax=60)
        assert np.linalg.norm(X_of(r0) - Xd) > 1e-2 * np.linalg.norm(Xd)


@pytest.mark.parametrize("real_pairs,inner", [(False, "direct"), (False, "gmres"), (False, "bicgstab"),
                                               (True, "direct")])
def test_generalized_nonsymmetric_mass_matrices(micro_g, real_pairs, inner):
    """eq. (gsylv) with nonsymmetric M and C (the Q1 mass matrices plus a
    strictly lower part), so that every transpose and conjugate transpose of
    C and M in Algorithm 1 and in the inner solvers matters (the B-side
    systems use (B + alpha C)^*): the factored X matches the Kronecker
    solution."""
    pr = micro_g
    A, B, M, C = mats(pr)
    M2 = (M + 0.3 * sp.tril(M, -1)).tocsr()
    C2 = (C + 0.3 * sp.tril(C, -1)).tocsr()
    Xd = kron_solve(A, B, pr.f, pr.g, M2, C2)
    if real_pairs:
        res = lradi_real(pr.A, pr.B, pr.f, pr.g, pr.alpha, pr.beta, pr.tau, M=M2, C=C2, inner="direct",
                         strategy="fixed", kmax=60)
        X = res.Z @ res.Gamma @ res.Y.T
    else:
        res = lradi(pr.A, pr.B, pr.f, pr.g, pr.alpha, pr.beta, pr.tau, M=M2, C=C2, inner=inner,
                    strategy="fixed", kmax=60, jacobi=True)
        X = X_of(res)
    assert res.converged
    assert np.linalg.norm(X - Xd) <= (1e-6 if inner == "direct" else 1e-5) * np.linalg.norm(Xd)
    R = dense_residual(A, B, pr.f, pr.g, X, M2, C2)
    assert np.linalg.norm(R, 2) <= 3 * pr.tau * np.linalg.norm(pr.f @ pr.g.T, 2)


def test_generalized_residual_factorisation_exact_solves(tiny_g):
    """eq. (adi_resexact) for eq. (gsylv): with exact solves R_k = w_k t_k^*."""
    p = tiny_g
    A, B, M, C = mats(p)
    res = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, M=p.M, C=p.C, inner="direct", kmax=5)
    R = dense_residual(A, B, p.f, p.g, X_of(res), M, C)
    assert np.linalg.norm(R - res.w @ res.t.conj().T, 2) <= 1e-11 * np.linalg.norm(R, 2)
    # the factored norm agrees with the dense one
    Rn = true_residual_norm2(A, B, p.f, p.g, res.Z, res.gamma, res.Y, M, C)
    assert Rn == pytest.approx(np.linalg.norm(R, 2), rel=1e-9)


def _sigma(vals, gam, r):
    k = len(vals)
    S = np.zeros((k, k), dtype=np.result_type(vals, gam))
    for i in range(k):
        S[i, i] = vals[i]
        S[i, :i] = -gam[i]
    return np.kron(S, np.eye(r))


def test_generalized_theorem1_and_2_inexact(tiny_g):
    """eq. (adi_AZ_BTY): A Z = M Z sigma^alpha + w E^T - S^A,
    B^T Y = C^T Y sigma^beta + t E^T - S^B, and eq. (adi_res_inexact):
    R_true = w t^* - S^A Gamma Y^* C - M Z Gamma (S^B)^*, with the inner
    residuals of GMRES solves stopped at the dynamic tolerances; the residual
    gap is bounded by u_k + v_k of eq. (upd_resgap)."""
    p = tiny_g
    res = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, M=p.M, C=p.C, strategy="bl_mid",
                keep_inner_residuals=True)
    A, B, M, C = (x.toarray() for x in mats(p))
    r, k = p.r, res.steps
    L = len(p.alpha)
    al = np.array([p.alpha[i % L] for i in range(k)])
    be = np.array([p.beta[i % L] for i in range(k)])
    gam = -(al + be)
    E = np.kron(np.ones((k, 1)), np.eye(r))
    lhs = A @ res.Z
    rhs = M @ res.Z @ _sigma(al, gam, r) + res.w @ E.T - res.S_A
    assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(lhs)
    lhsB = B.T @ res.Y
    rhsB = C.T @ res.Y @ _sigma(np.conj(be), np.conj(gam), r) + res.t @ E.T - res.S_B
    assert np.linalg.norm(lhsB - rhsB) <= 1e-10 * np.linalg.norm(lhsB)
    G = np.diag(res.gamma)
    R = dense_residual(A, B, p.f, p.g, X_of(res), M, C)
    gapA = res.S_A @ G @ res.Y.conj().T @ C
    gapB = M @ res.Z @ G @ res.S_B.conj().T
    assert np.linalg.norm(R - (res.w @ res.t.conj().T - gapA - gapB)) <= 1e-10 * np.linalg.norm(R) + 1e-14
    assert np.linalg.norm(gapA + gapB, 2) <= res.history[-1]["u"] + res.history[-1]["v"] + 1e-20
    # the estimate uses ||M z|| and ||C^T y||: with ||z||, ||y|| instead it is
    # a different (here much larger) number, since ||M|| ~ h^2
    u_plain = sum(abs(gam[i]) * block_norm2(res.Z[:, i * r:(i + 1) * r]) * block_norm2(res.S_B[:, i * r:(i + 1) * r])
                  for i in range(k))
    assert u_plain > 10 * res.history[-1]["u"]


def test_gmres_with_mass_matrix_matches_sparse_solve(tiny_g):
    """(A + sigma M) x = b by GMRES (plain and right Jacobi with
    diag(A) + sigma diag(M), CGS2 and DCGS2) against a sparse LU solve."""
    import scipy.sparse.linalg as spla
    A, _, M, _ = mats(tiny_g)
    sigma = tiny_g.beta[0]
    b = tiny_g.f[:, 0]
    x_ref = spla.spsolve((A + sigma * M).tocsc(), b)
    for jac in (False, True):
        for ortho in ("cgs2", "dcgs2"):
            res = gmres(A, sigma, b, 1e-12 * np.linalg.norm(b), 30, 5000, jac, ortho, mass=M)
            assert res.converged
            assert np.linalg.norm(res.x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
            assert np.linalg.norm(b - (A @ res.x + sigma * (M @ res.x))) == pytest.approx(res.resnorm, rel=1e-6, abs=1e-15)


def test_generalized_dynamic_tolerances_keep_the_exact_outer_count(tiny_g):
    """Table 2's qualitative result on the generalized workload: the dynamic
    rule takes the outer steps of exact solves and fewer inner steps than
    fixed tolerances."""
    p = tiny_g
    ex = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, M=p.M, C=p.C, inner="direct")
    fx = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, M=p.M, C=p.C, strategy="fixed")
    dy = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, M=p.M, C=p.C, strategy="nobl_mid")
    assert ex.converged and fx.converged and dy.converged
    assert abs(dy.steps - ex.steps) <= 1 and abs(fx.steps - ex.steps) <= 1
    assert dy.inner_its_A + dy.inner_its_B < fx.inner_its_A + fx.inner_its_B
