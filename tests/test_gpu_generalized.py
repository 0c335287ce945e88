"""The generalized equation A X C + M X B = -f g^* (eq. (gsylv); Algorithm 1
with the mass matrices, eq. (lradi_g)) on the GPU against the oracle's
generalized path: the shifted operators (A + sigma M) P^{-1} element by
element (stencil storage of the 2D Q1 mass matrices, CSR for the 27-point
3D ones), the inner solves with mass matrices, and whole solves (outer steps,
factored X, the true residual of eq. (gsylv))."""
import numpy as np
import pytest

import paper_2312_02891_gb300 as P
from paper_2312_02891_gb300 import workloads as W
from oracle.gmres import bicgstab as obicg, gmres as ogmres, shifted_apply
from oracle.lradi import lradi
from oracle.residual import factored_diff_fro, factored_fro, lowrank_norm2, true_residual_norm2

pytestmark = pytest.mark.gpu


def _colmajor(torch, M):
    return torch.from_numpy(np.asfortranarray(M).T.copy()).cuda()


def _pair(dim, N):
    if dim == 2:
        A = W.convdiff(N, 2, "xy", 10.0)
    else:
        A = W.convdiff(N, 3, "zxy", 20.0)
    h = (1.0 / (N + 1)) ** dim
    Ah = A.to_scipy() * h
    return Ah.tocsr(), W.mass_matrix(N, dim).to_scipy().tocsr()


@pytest.mark.parametrize("dim,N", [(2, 17), (3, 7)])
@pytest.mark.parametrize("transpose", [0, 1])
@pytest.mark.parametrize("jacobi", [0, 1])
@pytest.mark.parametrize("cplx", [0, 1])
def test_shifted_operator_with_mass_matches_oracle(torch_cuda, dim, N, transpose, jacobi, cplx):
    torch = torch_cuda
    S, M = _pair(dim, N)
    op = P.sylv_op_create(S, transpose=bool(transpose), mass=M)
    St = S.T.tocsr() if transpose else S
    Mt = M.T.tocsr() if transpose else M
    n = S.shape[0]
    rng = np.random.default_rng(3)
    X = rng.standard_normal((n, 2))
    sigma = -0.37
    if cplx:
        X = X + 1j * rng.standard_normal((n, 2))
        sigma = -0.37 + 0.11j
    try:
        is_st, ndiag, nn = P.sylv_op_format(op)
        assert is_st == (1 if dim == 2 else 0) and nn == n
        dX = _colmajor(torch, X)
        dY = torch.zeros_like(dX)
        P.sylv_op_apply(op, sigma, jacobi, cplx, dX, dY, 2)
        torch.cuda.synchronize()
        Y = dY.cpu().numpy().T
    finally:
        P.sylv_op_destroy(op)
    pinv = 1.0 / (St.diagonal() + sigma * Mt.diagonal()) if jacobi else np.ones(n)
    ref = np.stack([shifted_apply(St, sigma, pinv * X[:, c], Mt) for c in range(2)], axis=1)
    scale = (abs(St) + abs(sigma) * abs(Mt)) @ np.abs(pinv[:, None] * X)
    assert np.all(np.abs(Y - ref) <= 1e-13 * scale + 1e-300)


@pytest.mark.parametrize("solver", ["gmres", "bicgstab"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_inner_solves_with_mass_match_oracle(torch_cuda, solver, precision):
    torch = torch_cuda
    S, M = _pair(2, 20)
    n = S.shape[0]
    sigma = -0.8
    rng = np.random.default_rng(4)
    Bm = rng.standard_normal((n, 2)) * 1e-3
    tol = 1e-10 * np.linalg.norm(Bm[:, 0])
    op = P.sylv_op_create(S, mass=M)
    try:
        dB = _colmajor(torch, Bm)
        dX = torch.zeros_like(dB)
        if solver == "gmres":
            rc, iters, res, _ = P.sylv_gmres(op, sigma, 1, 0, dB, dX, 2, tol, 30, 4000, precision=precision)
        else:
            rc, iters, res, _ = P.sylv_bicgstab(op, sigma, 1, 0, dB, dX, 2, tol, 4000, precision=precision)
        X = dX.cpu().numpy().T
    finally:
        P.sylv_op_destroy(op)
    assert rc == 0, P.sylv_last_error()
    for c in range(2):
        rr = np.linalg.norm(Bm[:, c] - shifted_apply(S, sigma, X[:, c], M))
        assert rr <= tol * (1 + 1e-6)
        if solver == "gmres":
            ref = ogmres(S, sigma, Bm[:, c], tol, 30, 4000, True, "cgs2", mass=M)
        else:
            ref = obicg(S, sigma, Bm[:, c], tol, 4000, True, mass=M)
        if precision == "fp64":
            assert abs(int(iters[c]) - ref.iters) <= 2, (iters[c], ref.iters)
        ev = np.linalg.norm(X[:, c] - ref.x) / np.linalg.norm(ref.x)
        assert ev <= 1e-4, ev


@pytest.mark.parametrize("name,strategy,inner,precision", [
    ("tiny2d_g", "nobl_mid", "gmres", "fp64"),
    ("small2d_g", "bl_mid", "gmres", "fp64"),
    ("small2d_g", "nobl_mid", "gmres", "fp64"),
    ("small2d_g", "nobl_mid", "bicgstab", "fp32"),
    ("small2d_g", "fixed", "gmres", "fp32"),
])
def test_generalized_lradi_matches_oracle(name, strategy, inner, precision):
    p = W.problem_config(name)
    jac = bool(p.opts.get("jacobi", False))
    with P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, M=p.M, Cm=p.C, strategy=strategy,
                        jacobi=int(jac), inner=inner, precision=precision) as s:
        st = s.solve()
        info = s.info()
        hist = s.history()
        Z, Y, gam = s.factors()
    assert st == 0, P.sylv_last_error()
    ref = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, M=p.M, C=p.C, strategy=strategy, jacobi=jac,
                inner=inner)
    assert ref.converged
    assert abs(info["steps"] - ref.steps) <= 1, (info["steps"], ref.steps)
    assert info["rel_res_comp"] < p.tau
    A, B, Mm, Cm = p.A.to_scipy(), p.B.to_scipy(), p.M.to_scipy(), p.C.to_scipy()
    nfg = lowrank_norm2(p.f, p.g)
    tr = true_residual_norm2(A, B, p.f, p.g, Z, gam, Y, Mm, Cm) / nfg
    tr_ref = true_residual_norm2(A, B, p.f, p.g, ref.Z, ref.gamma, ref.Y, Mm, Cm) / nfg
    assert tr <= max(1.5 * tr_ref, 1e-8), (tr, tr_ref)
    dX = factored_diff_fro(Z, gam, Y, ref.Z, ref.gamma, ref.Y) / factored_fro(ref.Z, ref.gamma, ref.Y)
    assert dX <= 1e-6, dX
    if precision == "fp64" and inner == "gmres":
        # u, v of eq. (upd_resgap) use ||M z||, ||C^T y||: the history follows the oracle
        ks = min(len(hist), len(ref.history))
        for i in range(ks):
            assert hist[i][10] == pytest.approx(ref.history[i]["u"], rel=1e-3, abs=1e-20)
            assert hist[i][11] == pytest.approx(ref.history[i]["v"], rel=1e-3, abs=1e-20)
