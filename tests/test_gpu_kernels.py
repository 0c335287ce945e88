"""Parity of the hot-path kernels with the oracle, element by element, through
the C ABI: shifted SpMM (steps a2/a3), CGS2 (a4), batched GMRES with its
Givens least squares, stop test and restart (a5-a7), controller (a1)."""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_2312_02891_gb300 as P
from paper_2312_02891_gb300 import workloads as W
from oracle import controller as octl
from oracle.gmres import cgs2_step, gmres as ogmres, shifted_apply

pytestmark = pytest.mark.gpu


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _colmajor(torch, M):
    """n x c numpy (complex or real) -> device buffer in column-major order."""
    return _dev(torch, np.asfortranarray(M).T.copy())


def _host(t):
    return t.cpu().numpy()


def _rand_csr(n, density, seed):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr") + sp.eye(n) * 5.0
    M.sort_indices()
    return M.tocsr()


OPS = {
    "stencil2d": lambda: W.convdiff(17, 2, "xy", 10.0),          # n = 289: several chunks, ragged tail
    "stencil3d": lambda: W.convdiff(9, 3, "zxy", 20.0),          # n = 729, 7 diagonals
    "csr_random": lambda: _rand_csr(533, 0.02, 3),               # > 8 diagonals: CSR path
}


@pytest.mark.parametrize("name", list(OPS))
@pytest.mark.parametrize("transpose", [0, 1])
@pytest.mark.parametrize("jacobi", [0, 1])
@pytest.mark.parametrize("cplx", [0, 1])
def test_op_apply_matches_oracle(torch_cuda, name, transpose, jacobi, cplx):
    torch = torch_cuda
    M = OPS[name]()
    S = M.to_scipy() if hasattr(M, "to_scipy") else M
    St = S.T.tocsr() if transpose else S
    n = S.shape[0]
    rng = np.random.default_rng(11)
    ncols = 3
    X = rng.standard_normal((n, ncols))
    sigma = -37.5
    if cplx:
        X = X + 1j * rng.standard_normal((n, ncols))
        sigma = -37.5 + 12.25j
    op = P.sylv_op_create(M if hasattr(M, "rowptr") else S, transpose=bool(transpose))
    try:
        is_st, ndiag, nn = P.sylv_op_format(op)
        assert nn == n and is_st == (0 if name == "csr_random" else 1)
        dX = _colmajor(torch, X)
        dY = torch.zeros_like(dX)
        P.sylv_op_apply(op, sigma, jacobi, cplx, dX, dY, ncols)
        torch.cuda.synchronize()
        Y = _host(dY).T
        pinv = 1.0 / (St.diagonal() + sigma) if jacobi else np.ones(n)
        ref = np.stack([shifted_apply(St, sigma, pinv * X[:, c]) for c in range(ncols)], axis=1)
        scale = (abs(St) @ np.abs(pinv[:, None] * X)) + abs(sigma) * np.abs(pinv[:, None] * X)
        assert np.all(np.abs(Y - ref) <= 1e-14 * scale + 1e-300)
    finally:
        P.sylv_op_destroy(op)


@pytest.mark.parametrize("n,k", [(1, 1), (1000, 1), (4097, 7), (20000, 30)])
@pytest.mark.parametrize("cplx", [0, 1])
def test_cgs2_matches_oracle(torch_cuda, n, k, cplx):
    torch = torch_cuda
    if k > n:
        pytest.skip("k > n")
    rng = np.random.default_rng(n + k)
    V = rng.standard_normal((n, k))
    w = rng.standard_normal(n)
    if cplx:
        V = V + 1j * rng.standard_normal((n, k))
        w = w + 1j * rng.standard_normal(n)
    V, _ = np.linalg.qr(V)
    if n == 1:
        w = np.ones(1, dtype=w.dtype) * 2.0
    dV = _colmajor(torch, V)
    dw = _dev(torch, w)
    h = P.sylv_cgs2(dV, n, k, dw, is_complex=cplx)
    torch.cuda.synchronize()
    h_ref, w2 = cgs2_step(V.T.copy(), w.copy())
    hn = np.linalg.norm(w2)
    assert np.allclose(h[:k], h_ref, rtol=0, atol=1e-13 * np.linalg.norm(w))
    assert abs(h[k] - hn) <= 1e-12 * np.linalg.norm(w) + 1e-300
    if hn > 1e-12 * np.linalg.norm(w):
        v = _host(dw)
        assert np.allclose(v, w2 / hn, atol=1e-10)


def _gmres_case(kind):
    if kind == "tiny2d_A":
        M = W.convdiff(12, 2, "xy", 10.0)
        return M, -25.0, False
    if kind == "tiny2d_Bt":
        M = W.convdiff(10, 2, "rot2", 5.0)
        return M, -300.0, True
    if kind == "small3d":
        M = W.convdiff(8, 3, "zxy", 50.0)
        return M, -60.0 + 40.0j, False
    raise KeyError(kind)


@pytest.mark.parametrize("kind", ["tiny2d_A", "tiny2d_Bt", "small3d"])
@pytest.mark.parametrize("jacobi", [0, 1])
@pytest.mark.parametrize("restart", [30, 7])
def test_gmres_matches_oracle(torch_cuda, kind, jacobi, restart):
    torch = torch_cuda
    M, sigma, tr = _gmres_case(kind)
    S = M.to_scipy()
    St = S.T.tocsr() if tr else S
    n = S.shape[0]
    cplx = isinstance(sigma, complex)
    rng = np.random.default_rng(5)
    ncols = 3
    Bm = rng.standard_normal((n, ncols))
    Bm[:, 2] *= 1e-3                         # columns of different scale
    if cplx:
        Bm = Bm + 1j * rng.standard_normal((n, ncols))
    tol = 1e-9
    max_it = 3000
    op = P.sylv_op_create(M, transpose=tr)
    try:
        dB = _colmajor(torch, Bm)
        dX = torch.zeros_like(dB)
        rc, iters, res, hist = P.sylv_gmres(op, sigma, jacobi, cplx, dB, dX, ncols, tol, restart,
                                            max_it, want_hist=True)
        torch.cuda.synchronize()
        X = _host(dX).T
    finally:
        P.sylv_op_destroy(op)
    assert rc == 0
    for c in range(ncols):
        ref = ogmres(St, sigma, Bm[:, c], tol, restart, max_it, bool(jacobi), "cgs2")
        assert ref.converged
        # same algorithm and stop rule: iteration counts agree up to rounding near the threshold
        assert abs(int(iters[c]) - ref.iters) <= 2, (c, iters[c], ref.iters)
        # true residual recomputed independently
        rr = np.linalg.norm(Bm[:, c] - shifted_apply(St, sigma, X[:, c]))
        assert rr <= tol * (1 + 1e-6)
        assert abs(res[c] - rr) <= 1e-6 * tol + 1e-12 * np.linalg.norm(Bm[:, c])
        # Givens residual estimates agree step by step over the first cycle
        k = min(restart, len(ref.history), int(iters[c]))
        hg = hist[c, :k]
        ho = np.array(ref.history[:k])
        assert np.allclose(hg, ho, rtol=1e-6, atol=1e-12 * np.linalg.norm(Bm[:, c]))
        # solutions agree to the accuracy both reached
        assert np.linalg.norm(X[:, c] - ref.x) <= 1e3 * tol / abs(sigma) * 10 + 1e-12


def test_gmres_zero_rhs_and_iteration_cap(torch_cuda):
    torch = torch_cuda
    M = W.convdiff(16, 2, "xy", 0.0)
    n = M.n
    op = P.sylv_op_create(M)
    try:
        B = np.zeros((n, 2))
        B[:, 1] = np.random.default_rng(1).standard_normal(n)
        dB = _colmajor(torch, B)
        dX = torch.full_like(dB, 7.0)
        # column 0 is zero: done with x = 0 before any Arnoldi step
        # column 1 capped at 5 Arnoldi steps with an unreachable tolerance
        rc, iters, res, _ = P.sylv_gmres(op, -1.0, 0, 0, dB, dX, 2, 1e-30, 30, 5)
        X = _host(dX).T
        assert rc == -5                                  # INNER_STALL warning
        assert iters[0] == 0 and res[0] == 0.0 and np.all(X[:, 0] == 0)
        assert iters[1] == 5 and res[1] > 0
        ref = ogmres(M.to_scipy(), -1.0, B[:, 1], 1e-30, 30, 5, False, "cgs2")
        assert ref.iters == 5
        assert np.allclose(X[:, 1], ref.x, rtol=1e-9, atol=1e-12)
    finally:
        P.sylv_op_destroy(op)


@pytest.mark.parametrize("strategy", list(P.STRATEGIES))
@pytest.mark.parametrize("clamp", [0, 1])
def test_controller_matches_oracle(lib, strategy, clamp):
    rng = np.random.default_rng(3)
    cnt = 400
    k = rng.integers(1, 51, cnt).astype(float)
    kmax = np.full(cnt, 50.0)
    eps = 10.0 ** rng.uniform(-10, -6, cnt)
    xi = rng.uniform(0.1, 1.0, cnt)
    u = 10.0 ** rng.uniform(-14, -7, cnt)
    v = 10.0 ** rng.uniform(-14, -7, cnt)
    Nw = 10.0 ** rng.uniform(-5, 1, cnt)
    Nt = 10.0 ** rng.uniform(-5, 1, cnt)
    fixed = np.full(cnt, 5e-10)
    inp = np.stack([k, kmax, eps, xi, u, v, Nw, Nt, fixed, np.zeros(cnt), np.zeros(cnt)], axis=1)
    o = P.sylv_opts_default(strategy=strategy, bl_clamp=clamp, dmin_A=5e-10, dmin_B=7e-10,
                            dmax_A=0.1, dmax_B=0.05)
    out = P.sylv_controller_eval(o, inp)
    for i in range(cnt):
        if clamp and strategy.startswith("bl_"):
            # clamp variant: max(., 0) in place of |.|
            x = xi[i] * k[i] * eps[i] / (2 * octl.C_BOUND * kmax[i]) - u[i] - v[i]
            ur = max(x, 0.0) / octl.C_BOUND
            sel = {"mid": octl.select_mid, "A": octl.select_prefer_A, "B": octl.select_prefer_B}[strategy.split("_")[1]]
            dA, dB = sel(ur, Nw[i], Nt[i], 5e-10, 0.1, 7e-10, 0.05)
            eh = ur
        else:
            dA, dB, eh = octl.inner_tolerances(strategy, k=int(k[i]), kmax=50, eps=eps[i], xi=xi[i],
                                               u_prev=u[i], v_prev=v[i], N_w=Nw[i], N_t=Nt[i],
                                               dmin_A=5e-10, dmax_A=0.1, dmin_B=7e-10, dmax_B=0.05,
                                               fixed_tol=5e-10)
        assert out[i, 0] == pytest.approx(dA, rel=1e-13, abs=0)
        assert out[i, 1] == pytest.approx(dB, rel=1e-13, abs=0)
        if strategy != "fixed":
            assert out[i, 2] == pytest.approx(eh, rel=1e-13, abs=0)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("kind", ["tiny2d_A", "tiny2d_Bt", "small3d"])
def test_gmres_mixed_precision_meets_tolerance(torch_cuda, precision, kind):
    """float32/bfloat16 basis: the float64 restart residual still reaches tol
    (iterative refinement across restarts) and the solution matches the
    oracle's float64 solve to the accuracy both reached."""
    torch = torch_cuda
    M, sigma, tr = _gmres_case(kind)
    S = M.to_scipy()
    St = S.T.tocsr() if tr else S
    n = S.shape[0]
    cplx = isinstance(sigma, complex)
    rng = np.random.default_rng(8)
    Bm = rng.standard_normal((n, 2))
    if cplx:
        Bm = Bm + 1j * rng.standard_normal((n, 2))
    tol = 1e-10 * np.linalg.norm(Bm[:, 0])
    op = P.sylv_op_create(M, transpose=tr)
    try:
        dB = _colmajor(torch, Bm)
        dX = torch.zeros_like(dB)
        rc, iters, res, _ = P.sylv_gmres(op, sigma, 1, cplx, dB, dX, 2, tol, 30, 6000,
                                         precision=precision)
        X = _host(dX).T
    finally:
        P.sylv_op_destroy(op)
    assert rc == 0
    for c in range(2):
        rr = np.linalg.norm(Bm[:, c] - shifted_apply(St, sigma, X[:, c]))
        assert rr <= tol * (1 + 1e-6)
        ref = ogmres(St, sigma, Bm[:, c], tol, 30, 6000, True, "cgs2")
        assert np.linalg.norm(X[:, c] - ref.x) <= 1e3 * tol / abs(sigma) * 10 + 1e-12
