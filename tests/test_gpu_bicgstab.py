"""Parity of the CUDA BiCGstab inner solver with the oracle's BiCGstab
(Sec. 3.3 "Further implementation aspects", Sec. 4: the paper's inner solver
for unsymmetric systems), through the C ABI: per-step recurrence residuals,
step counts, true residuals and solutions of the shifted systems, then whole
inexact LR-ADI solves with BiCGstab inner solves against the oracle's
Algorithm 1 with the same inner solver, single and batched."""
import numpy as np
import pytest

import paper_2312_02891_gb300 as P
from paper_2312_02891_gb300 import workloads as W
from oracle.gmres import bicgstab as obicg, shifted_apply
from oracle.lradi import lradi
from oracle.residual import factored_diff_fro, factored_fro, lowrank_norm2, true_residual_norm2

pytestmark = pytest.mark.gpu


def _colmajor(torch, M):
    return torch.from_numpy(np.asfortranarray(M).T.copy()).cuda()


def _case(kind):
    if kind == "tiny2d_A":          # n = 144: one chunk
        return W.convdiff(12, 2, "xy", 10.0), -25.0, False
    if kind == "tiny2d_Bt":         # transposed rotational operator
        return W.convdiff(10, 2, "rot2", 5.0), -300.0, True
    if kind == "ragged2d":          # n = 70 x 70 = 4900: several chunks, ragged tail
        return W.convdiff(70, 2, "xy", 40.0), -900.0, False
    if kind == "small3d":           # complex shift, 7-point stencil
        return W.convdiff(8, 3, "zxy", 50.0), -60.0 + 40.0j, False
    raise KeyError(kind)


def _solve(torch, M, tr, sigma, Bm, tol, max_it, jacobi, precision="fp64", rows_hint=None):
    cplx = isinstance(sigma, complex) or np.iscomplexobj(Bm)
    op = P.sylv_op_create(M, transpose=tr)
    try:
        dB = _colmajor(torch, Bm)
        dX = torch.zeros_like(dB)
        rc, iters, res, hist = P.sylv_bicgstab(op, sigma, jacobi, cplx, dB, dX, Bm.shape[1], tol, max_it,
                                               want_hist=True, precision=precision)
        torch.cuda.synchronize()
        X = dX.cpu().numpy().T
    finally:
        P.sylv_op_destroy(op)
    return rc, iters, res, hist, X


@pytest.mark.parametrize("kind", ["tiny2d_A", "tiny2d_Bt", "ragged2d", "small3d"])
@pytest.mark.parametrize("jacobi", [0, 1])
def test_bicgstab_matches_oracle(torch_cuda, kind, jacobi):
    torch = torch_cuda
    M, sigma, tr = _case(kind)
    S = M.to_scipy()
    St = S.T.tocsr() if tr else S
    n = S.shape[0]
    rng = np.random.default_rng(7)
    ncols = 3                                  # one group of three columns
    Bm = rng.standard_normal((n, ncols))
    Bm[:, 2] *= 1e-3
    if isinstance(sigma, complex):
        Bm = Bm + 1j * rng.standard_normal((n, ncols))
    tol = 1e-9
    rc, iters, res, hist, X = _solve(torch, M, tr, sigma, Bm, tol, 4000, jacobi)
    assert rc == 0, P.sylv_last_error()
    for c in range(ncols):
        ref = obicg(St, sigma, Bm[:, c], tol, 4000, bool(jacobi))
        assert ref.converged
        # same recurrences and stop rule: step counts agree up to rounding near the threshold
        assert abs(int(iters[c]) - ref.iters) <= 2, (c, iters[c], ref.iters)
        rr = np.linalg.norm(Bm[:, c] - shifted_apply(St, sigma, X[:, c]))
        assert rr <= tol * (1 + 1e-6)
        assert abs(res[c] - rr) <= 1e-6 * tol + 1e-12 * np.linalg.norm(Bm[:, c])
        # the recurrence residual norms agree step by step over the first steps
        k = min(12, len(ref.history), int(iters[c]))
        assert np.allclose(hist[c, :k], np.array(ref.history[:k]), rtol=1e-6,
                           atol=1e-12 * np.linalg.norm(Bm[:, c]))
        assert np.linalg.norm(X[:, c] - ref.x) <= 1e3 * tol / abs(sigma) * 10 + 1e-12


def test_bicgstab_groups_of_columns(torch_cuda):
    """Six columns form groups of four and two; each column equals its solve
    alone (the group shares only the operator loads, not the recurrences)."""
    torch = torch_cuda
    M, sigma, tr = _case("ragged2d")
    n = M.n
    rng = np.random.default_rng(3)
    Bm = rng.standard_normal((n, 6)) * np.array([1.0, 1e2, 1e-2, 1.0, 3.0, 1e-4])
    tol = 1e-8
    rc, iters, res, hist, X = _solve(torch, M, tr, sigma, Bm, tol, 4000, 1)
    assert rc == 0
    for c in range(6):
        rc1, it1, res1, h1, X1 = _solve(torch, M, tr, sigma, Bm[:, c:c + 1], tol, 4000, 1)
        assert int(it1[0]) == int(iters[c])
        assert np.array_equal(h1[0, :it1[0]], hist[c, :iters[c]])
        assert np.array_equal(X1[:, 0], X[:, c])


@pytest.mark.parametrize("kind", ["tiny2d_A", "ragged2d", "small3d"])
def test_bicgstab_fp32_meets_float64_tolerance(torch_cuda, kind):
    """float32 vectors and products: the float64 restart residual still
    reaches tol (each cycle solves the correction equation)."""
    torch = torch_cuda
    M, sigma, tr = _case(kind)
    S = M.to_scipy()
    St = S.T.tocsr() if tr else S
    n = S.shape[0]
    rng = np.random.default_rng(9)
    Bm = rng.standard_normal((n, 2))
    if isinstance(sigma, complex):
        Bm = Bm + 1j * rng.standard_normal((n, 2))
    tol = 1e-10 * np.linalg.norm(Bm[:, 0])
    rc, iters, res, _, X = _solve(torch, M, tr, sigma, Bm, tol, 6000, 1, precision="fp32")
    assert rc == 0, P.sylv_last_error()
    for c in range(2):
        rr = np.linalg.norm(Bm[:, c] - shifted_apply(St, sigma, X[:, c]))
        assert rr <= tol * (1 + 1e-6)
        ref = obicg(St, sigma, Bm[:, c], tol, 6000, True)
        assert np.linalg.norm(X[:, c] - ref.x) <= 1e3 * tol / abs(sigma) * 10 + 1e-12


def test_bicgstab_zero_rhs_and_step_cap(torch_cuda):
    torch = torch_cuda
    M = W.convdiff(16, 2, "xy", 0.0)
    n = M.n
    B = np.zeros((n, 2))
    B[:, 1] = np.random.default_rng(1).standard_normal(n)
    rc, iters, res, _, X = _solve(torch, M, False, -1.0, B, 1e-30, 5, 0)
    assert rc == -5                                  # INNER_STALL warning
    assert iters[0] == 0 and res[0] == 0.0 and np.all(X[:, 0] == 0)
    assert iters[1] == 5 and res[1] > 0
    ref = obicg(M.to_scipy(), -1.0, B[:, 1], 1e-30, 5, False)
    assert ref.iters == 5
    assert np.allclose(X[:, 1], ref.x, rtol=1e-9, atol=1e-12)


def test_bicgstab_bf16_is_refused(torch_cuda):
    torch = torch_cuda
    M, sigma, tr = _case("tiny2d_A")
    with pytest.raises(P.SylvError, match="UNSUPPORTED"):
        _solve(torch, M, tr, sigma, np.ones((M.n, 1)), 1e-8, 10, 0, precision="bf16")


# ---------------------------------------------------------------- whole solves

_PROB = {}


def problem(name):
    if name not in _PROB:
        _PROB[name] = W.problem_config(name)
    return _PROB[name]


def _adi(p, **opts):
    with P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner="bicgstab", **opts) as s:
        st = s.solve()
        info = s.info()
        hist = s.history()
        Z, Y, gam = s.factors()
    return st, info, hist, Z, Y, gam


@pytest.mark.parametrize("name,strategy,jacobi,precision", [
    ("small2d", "bl_mid", False, "fp64"),
    ("small2d", "nobl_mid", True, "fp64"),
    ("small2d", "fixed", True, "fp64"),
    ("small2d", "nobl_mid", True, "fp32"),
    ("tiny2d", "bl_B", True, "fp32"),
    ("small3d", "nobl_mid", True, "fp64"),
    ("small3d", "nobl_mid", True, "fp32"),
])
def test_lradi_with_bicgstab_matches_oracle(name, strategy, jacobi, precision):
    p = problem(name)
    st, info, hist, Z, Y, gam = _adi(p, strategy=strategy, jacobi=int(jacobi), precision=precision)
    ref = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy=strategy, jacobi=jacobi, inner="bicgstab")
    A, B = p.A.to_scipy(), p.B.to_scipy()
    nfg = lowrank_norm2(p.f, p.g)
    assert st == 0, P.sylv_last_error()
    assert ref.converged
    assert abs(info["steps"] - ref.steps) <= 1, (info["steps"], ref.steps)
    assert info["rel_res_comp"] < p.tau
    tr_gpu = true_residual_norm2(A, B, p.f, p.g, Z, gam, Y) / nfg
    tr_ref = true_residual_norm2(A, B, p.f, p.g, ref.Z, ref.gamma, ref.Y) / nfg
    assert tr_gpu <= max(1.5 * tr_ref, 1e-8), (tr_gpu, tr_ref)
    dX = factored_diff_fro(Z, gam, Y, ref.Z, ref.gamma, ref.Y) / factored_fro(ref.Z, ref.gamma, ref.Y)
    assert dX <= 1e-6, dX
    if precision == "fp64":
        # inner step counts of the whole solve agree closely (same recurrences)
        itg = info["inner_its_A"] + info["inner_its_B"]
        ito = ref.inner_its_A + ref.inner_its_B
        assert abs(itg - ito) <= 0.02 * ito + 4 * info["steps"], (itg, ito)
        # BiCGstab's residual is not monotone: the step that meets the
        # tolerance, and with it the achieved residual, can differ between two
        # roundings of the same recurrences.  Every step meets its requested
        # tolerances; without back-looking the tolerances depend only on
        # ||w||, ||t|| and follow the oracle's (back-looking feeds the achieved
        # residuals into the next tolerances, so there they drift apart)
        ks = min(len(hist), len(ref.history))
        for i in range(ks):
            h, o = hist[i], ref.history[i]
            assert h[6] <= h[3] * (1 + 1e-9) and h[7] <= h[4] * (1 + 1e-9)
            if not strategy.startswith("bl_"):
                assert h[3] == pytest.approx(o["dA"], rel=1e-3) and h[4] == pytest.approx(o["dB"], rel=1e-3)
                assert h[12] == pytest.approx(o["res_comp"], rel=2e-2, abs=1e-3 * p.tau)


def test_graph_and_host_drivers_agree_with_bicgstab():
    p = problem("small2d")
    out = []
    for drv in (0, 1):
        st, info, hist, Z, Y, gam = _adi(p, strategy="nobl_mid", jacobi=1, precision="fp32", driver=drv)
        assert st == 0
        out.append((info["steps"], info["inner_its_A"], info["inner_its_B"], Z, Y))
    assert out[0][:3] == out[1][:3]
    assert np.array_equal(out[0][3], out[1][3]) and np.array_equal(out[0][4], out[1][4])


def test_batch_with_bicgstab_matches_oracle_per_instance():
    probs = W.batch_problems(6, base_seed=2000, n_shifts=6, nmin=8, nmax=20)
    with P.SylvesterADIBatch(probs, strategy="nobl_mid", precision="fp64", jacobi=1, inner="bicgstab") as bt:
        assert bt.solve() == 0, P.sylv_last_error()
        for i, p in enumerate(probs):
            info = bt.info(i)
            Z, Y, gam = bt.factors(i)
            ref = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy="nobl_mid", jacobi=True,
                        inner="bicgstab")
            assert abs(info["steps"] - ref.steps) <= 1
            dX = factored_diff_fro(Z, gam, Y, ref.Z, ref.gamma, ref.Y) / factored_fro(ref.Z, ref.gamma, ref.Y)
            assert dX <= 1e-6, (i, dX)
