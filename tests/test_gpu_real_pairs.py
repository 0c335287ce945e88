"""The real double step for complex conjugate shift pairs on the GPU
(Sec. 3.3 "Complex shift parameters") against the oracle's real formulation
(oracle/lradi_real.py) and against the GPU's own complex formulation: outer
steps, the factored solution X = Z G Y^T with real factors and the 2 x 2
cores, the true residual, per-step residual norms of both steps of a pair,
and fewer complex inner steps than the complex formulation."""
import numpy as np
import pytest

import paper_2312_02891_gb300 as P
from paper_2312_02891_gb300 import workloads as W
from oracle.lradi import lradi
from oracle.lradi_real import lradi_real
from oracle.residual import lowrank_fro, lowrank_norm2

pytestmark = pytest.mark.gpu

_PROB = {}


def problem(name):
    if name not in _PROB:
        if name == "t3d":      # n = 1000, m = 512, r = 2, 3 conjugate pairs (real and complex shifts per side)
            _PROB[name] = W.make_problem("t3d", 10, 3, "const3", 100.0, 8, 3, "zxy", 50.0, 2, 4, 6,
                                         real_shifts=False, restart=30, jacobi=True)
        else:
            _PROB[name] = W.problem_config(name)
    return _PROB[name]


def _true_res(p, Z, G, Y):
    """||A X + X B + f g^T||_2 for X = Z G Y^T (eq. adi_res_inexact)."""
    A, B = p.A.to_scipy(), p.B.to_scipy()
    YG = Y @ G.T
    U = np.hstack([A @ Z, Z, p.f])
    Wm = np.hstack([YG, B.T @ YG, p.g])
    return lowrank_norm2(U, Wm)


def _diff(Z1, G1, Y1, Z2, G2, Y2):
    return lowrank_fro(np.hstack([Z1 @ G1, -Z2 @ G2]), np.hstack([Y1, Y2]))


def _gpu(p, **opts):
    with P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, **opts) as s:
        st = s.solve()
        info = s.info()
        hist = s.history()
        Z, Y, G = s.factors()
    return st, info, hist, Z, Y, G


@pytest.mark.parametrize("name,inner,precision,strategy", [
    ("t3d", "gmres", "fp64", "bl_mid"),
    ("t3d", "bicgstab", "fp64", "nobl_mid"),
    ("t3d", "gmres", "fp32", "nobl_mid"),
    ("small3d", "gmres", "fp64", "nobl_mid"),
    ("small3d", "bicgstab", "fp32", "nobl_mid"),
])
def test_real_double_step_matches_oracle(name, inner, precision, strategy):
    p = problem(name)
    st, info, hist, Z, Y, G = _gpu(p, strategy=strategy, jacobi=1, precision=precision, inner=inner,
                                   real_pairs=1)
    assert st == 0, P.sylv_last_error()
    assert info["is_complex"] == 0 and Z.dtype == np.float64 and G.shape == (info["kr"], info["kr"])
    ref = lradi_real(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy=strategy, jacobi=True, inner=inner)
    assert ref.converged
    assert abs(info["steps"] - ref.steps) <= 1, (info["steps"], ref.steps)
    nfg = lowrank_norm2(p.f, p.g)
    assert info["rel_res_comp"] < p.tau
    tr = _true_res(p, Z, G, Y) / nfg
    tr_ref = _true_res(p, ref.Z, ref.Gamma, ref.Y) / nfg
    assert tr <= max(1.5 * tr_ref, 2e-8), (tr, tr_ref)
    dX = _diff(Z, G, Y, ref.Z, ref.Gamma, ref.Y) / lowrank_fro(ref.Z @ ref.Gamma, ref.Y)
    assert dX <= 1e-6, dX
    # the core: 2 x 2 blocks per pair (kron I_r), nothing else off the diagonal
    r = p.r
    c0 = 0
    for h in ref.history:
        s = 2 * r if h["pair"] else r
        blk = G[c0:c0 + s, c0:c0 + s]
        off = G[c0:c0 + s].copy()
        off[:, c0:c0 + s] = 0.0
        assert not off.any()
        if h["pair"]:
            assert np.allclose(blk, np.kron(blk[::r, ::r], np.eye(r)), rtol=1e-12, atol=0)
        c0 += s
    # per step of the equivalent complex formulation: the residual norms of
    # both steps of a pair (the inputs of eq. (upd_resgap)) meet the step's
    # tolerances; with GMRES in float64 they are the oracle's (BiCGstab's
    # achieved residuals differ with the rounding, see test_gpu_bicgstab.py)
    rows = [(h["nrA"][j], h["nrB"][j]) for h in ref.history for j in range(2 if h["pair"] else 1)]
    ks = min(len(rows), len(hist))
    for i in range(ks):
        assert hist[i][6] <= hist[i][3] * (1 + 1e-9) and hist[i][7] <= hist[i][4] * (1 + 1e-9)
    if precision == "fp64" and inner == "gmres":
        for i in range(min(ks, 6)):
            assert hist[i][6] == pytest.approx(rows[i][0], rel=1e-3, abs=1e-3 * p.tau)
            assert hist[i][7] == pytest.approx(rows[i][1], rel=1e-3, abs=1e-3 * p.tau)


def test_real_double_step_agrees_with_complex_formulation_and_saves_solves():
    p = problem("small3d")
    st1, i1, h1, Z1, Y1, g1 = _gpu(p, strategy="nobl_mid", jacobi=1, precision="fp64", real_pairs=0)
    st2, i2, h2, Z2, Y2, G2 = _gpu(p, strategy="nobl_mid", jacobi=1, precision="fp64", real_pairs=1)
    assert st1 == 0 and st2 == 0
    assert i1["is_complex"] == 1 and i2["is_complex"] == 0
    assert abs(i1["steps"] - i2["steps"]) <= 1
    X1U, X1W = Z1 * g1[None, :], Y1.conj()
    dX = lowrank_fro(np.hstack([X1U, -(Z2 @ G2)]), np.hstack([X1W.conj(), Y2])) / lowrank_fro(X1U, Y1)
    assert dX <= 1e-6, dX
    # the second solves of complex-shift sides are derived, not computed
    assert i2["inner_its_A"] + i2["inner_its_B"] < i1["inner_its_A"] + i1["inner_its_B"]


def test_real_pairs_factors_need_the_core_call():
    p = problem("tiny2d")
    al = np.array([-200.0 + 80j, -200.0 - 80j, -500.0 + 0j, -500.0 - 0j])
    be = np.array([-150.0 + 30j, -150.0 - 30j, -700.0 + 10j, -700.0 - 10j])
    with P.SylvesterADI(p.A, p.B, p.f, p.g, al, be, p.tau, jacobi=1, real_pairs=1, strategy="nobl_mid") as s:
        s.solve()
        import ctypes as C
        kr = C.c_int32()
        isc = C.c_int32()
        Z = np.zeros(max(1, s.info()["kr"]) * p.A.n)
        Y = np.zeros(max(1, s.info()["kr"]) * p.B.n)
        g = np.zeros(max(1, s.info()["kr"]))
        rc = P.load().sylv_adi_factors(s.h, Z.ctypes.data, Y.ctypes.data, g.ctypes.data, 0, C.byref(kr),
                                      C.byref(isc))
        assert rc == -1 and "sylv_adi_core" in P.sylv_last_error()
        Zr, Yr, G = s.factors()
        assert Zr.shape[1] == G.shape[0] == s.info()["kr"]


def test_batch_refuses_real_pairs_with_complex_shifts():
    p = problem("small3d")
    with pytest.raises(P.SylvError, match="UNSUPPORTED"):
        P.SylvesterADIBatch([p], real_pairs=1, jacobi=1)
