"""End-to-end parity of the GPU inexact LR-ADI (Algorithm 1) with the oracle
through the C ABI: outer step counts, per-step controller history, the
computed and true residuals, and the factored solution X = Z Gamma Y^*."""
import numpy as np
import pytest

import paper_2312_02891_gb300 as P
from paper_2312_02891_gb300 import workloads as W
from oracle.dense import bartels_stewart
from oracle.lradi import lradi
from oracle.residual import factored_diff_fro, factored_fro, lowrank_norm2, true_residual_norm2

pytestmark = pytest.mark.gpu

_PROB = {}


def problem(name):
    if name not in _PROB:
        _PROB[name] = W.problem_config(name)
    return _PROB[name]


def run_gpu(p, **opts):
    with P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, **opts) as s:
        st = s.solve()
        info = s.info()
        hist = s.history()
        Z, Y, gam = s.factors()
    return st, info, hist, Z, Y, gam


def compare(p, strategy, jacobi, xtol=1e-6, **extra):
    st, info, hist, Z, Y, gam = run_gpu(p, strategy=strategy, jacobi=int(jacobi), **extra)
    ref = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy=strategy, jacobi=jacobi,
                **{k: v for k, v in extra.items() if k in ("kmax", "xi", "fixed_tol", "max_inner", "restart", "ortho",
                                                           "inner")})
    A, B = p.A.to_scipy(), p.B.to_scipy()
    nfg = lowrank_norm2(p.f, p.g)
    assert st == 0, P.sylv_last_error()
    assert ref.converged
    # outer iteration counts within +-1
    assert abs(info["steps"] - ref.steps) <= 1, (info["steps"], ref.steps)
    # computed relative residual below tau on both
    assert info["rel_res_comp"] < p.tau and ref.res_comp < p.tau
    # ||f g^*|| agrees
    assert info["norm_fg"] == pytest.approx(nfg, rel=1e-12)
    # true residuals through the factors, GPU vs oracle
    tr_gpu = true_residual_norm2(A, B, p.f, p.g, Z, gam, Y) / nfg
    tr_ref = true_residual_norm2(A, B, p.f, p.g, ref.Z, ref.gamma, ref.Y) / nfg
    assert tr_gpu <= max(1.5 * tr_ref, 1e-8), (tr_gpu, tr_ref)
    # factored solutions agree
    dX = factored_diff_fro(Z, gam, Y, ref.Z, ref.gamma, ref.Y) / factored_fro(ref.Z, ref.gamma, ref.Y)
    assert dX <= xtol, dX
    # step-by-step history over the common steps: shifts, tolerances, residuals.
    # Mixed precision changes the inner solutions within their tolerances, so
    # the norms of w_k agree to that level rather than to rounding.
    mixed = extra.get("precision", "fp64") != "fp64"
    ks = min(len(hist), len(ref.history))
    for i in range(ks):
        h, o = hist[i], ref.history[i]
        assert h[0] == o["k"]
        assert h[1] == pytest.approx(np.real(o["alpha"])) and h[2] == pytest.approx(np.real(o["beta"]))
        if not mixed:
            assert h[3] == pytest.approx(o["dA"], rel=1e-3) and h[4] == pytest.approx(o["dB"], rel=1e-3)
        elif not strategy.startswith("bl_"):
            # without back-looking the tolerances depend only on ||w||, ||t||
            assert h[3] == pytest.approx(o["dA"], rel=0.05) and h[4] == pytest.approx(o["dB"], rel=0.05)
        # (back-looking tolerances follow the achieved inner residuals, which
        # float32 inner solves change within their tolerances)
        assert h[12] == pytest.approx(o["res_comp"], rel=0.05 if mixed else 1e-3, abs=1e-3 * p.tau)
        assert h[13] == pytest.approx(o["N_w"], rel=1e-2 if mixed else 1e-6)
    return info, ref, tr_gpu, tr_ref, dX


@pytest.mark.parametrize("strategy", ["bl_mid", "nobl_mid", "fixed", "bl_B", "nobl_A"])
def test_small2d_parity(strategy):
    p = problem("small2d")
    info, ref, tr_gpu, tr_ref, dX = compare(p, strategy, jacobi=False)
    # the paper's qualitative point: dynamic tolerances need fewer inner steps than fixed ones
    if strategy == "bl_mid":
        fixed = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy="fixed")
        assert info["inner_its_A"] + info["inner_its_B"] < fixed.inner_its_A + fixed.inner_its_B


def test_small2d_against_bartels_stewart():
    p = problem("small2d")
    st, info, hist, Z, Y, gam = run_gpu(p, strategy="nobl_mid", jacobi=0)
    X = bartels_stewart(p.A.to_scipy(), p.B.to_scipy(), p.f, p.g)
    err = np.linalg.norm(Z @ np.diag(gam) @ Y.T - X) / np.linalg.norm(X)
    assert err < 1e-6


@pytest.mark.parametrize("jacobi", [False, True])
def test_tiny2d_rank2_parity(jacobi):
    compare(problem("tiny2d"), "bl_mid", jacobi)


def test_rank3_ragged_parity():
    p = W.make_problem("r3", 19, 2, "xy", 20.0, 13, 2, "rot2", 8.0, 3, 21, 10)
    compare(p, "bl_mid", True)


def test_complex_shift_pairs_parity():
    # rotational convection on both sides: complex Ritz values, conjugate pairs kept
    p = W.make_problem("cplx", 14, 2, "rot2", 60.0, 12, 2, "rot2", 40.0, 2, 33, 8, real_shifts=False)
    assert np.iscomplexobj(p.alpha) and np.any(np.imag(p.alpha) != 0)
    info, ref, tr_gpu, tr_ref, dX = compare(p, "bl_mid", True)
    assert info["is_complex"] == 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_small3d_complex_parity(precision):
    """3D operators with rotational convection, r = 4, complex conjugate shift
    pairs (the family of the large 3D workloads, at a size the oracle runs)."""
    info, ref, tr_gpu, tr_ref, dX = compare(problem("small3d"), "nobl_mid", True, precision=precision)
    assert info["is_complex"] == 1 and tr_gpu <= 1e-8


def test_zero_rhs_is_solved_by_zero():
    p = problem("tiny2d")
    z = np.zeros_like(p.f)
    with P.SylvesterADI(p.A, p.B, z, p.g, p.alpha, p.beta, p.tau) as s:
        assert s.solve() == 0
        assert s.info()["steps"] == 0


def test_kmax_reached_returns_maxit():
    p = problem("small2d")
    with P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, kmax=3, jacobi=0) as s:
        assert s.solve() == -4
        info = s.info()
        assert info["steps"] == 3 and info["kr"] == 3
        Z, Y, gam = s.factors()
        assert Z.shape == (p.A.n, 3)
    ref = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, kmax=3)
    assert ref.steps == 3 and not ref.converged


def test_resolve_with_new_rhs_is_repeatable():
    p = problem("tiny2d")
    with P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau) as s:
        s.solve()
        Z1, Y1, g1 = s.factors()
        f2, g2 = W.rhs_factors(p.A.n, p.B.n, p.r, 99)
        s.set_rhs(f2, g2)
        s.solve()
        s.set_rhs(p.f, p.g)
        s.solve()
        Z2, Y2, g2_ = s.factors()
    assert np.array_equal(Z1, Z2) and np.array_equal(Y1, Y2) and np.array_equal(g1, g2_)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("name,strategy,jacobi", [("small2d", "nobl_mid", False), ("tiny2d", "bl_mid", True)])
def test_mixed_precision_parity(precision, name, strategy, jacobi):
    """Krylov basis and sweeps in float32 (or a bfloat16 basis), restart
    residuals, least squares and the outer iteration in float64: same outer
    steps as the float64 oracle (+-1) and the same factored solution."""
    compare(problem(name), strategy, jacobi, precision=precision)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_mixed_precision_complex_pairs(precision):
    p = W.make_problem("cplx", 14, 2, "rot2", 60.0, 12, 2, "rot2", 40.0, 2, 33, 8, real_shifts=False)
    info, ref, tr_gpu, tr_ref, dX = compare(p, "bl_mid", True, precision=precision)
    assert info["is_complex"] == 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["tiny2d", "small2d"])
def test_graph_and_host_driven_solves_agree_bitwise(precision, name):
    """The device-driven CUDA graph (conditional nodes set by the kernels) and
    the host-driven loop launch the same kernels in the same order; with the
    fixed-order reductions the factors agree bit for bit."""
    p = problem(name)
    jac = int(p.opts.get("jacobi", False))
    out = []
    for driver in (0, 1):
        st, info, hist, Z, Y, gam = run_gpu(p, strategy="nobl_mid", jacobi=jac, precision=precision,
                                            driver=driver)
        assert st == 0
        out.append((info["steps"], Z, Y, gam, info["launches"]))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    assert np.array_equal(out[0][3], out[1][3])
    # the graph skips the restart kernels in iterations that do not need them
    assert 0 < out[0][4] <= out[1][4]


def test_graph_solve_respects_kmax_and_zero_rhs():
    p = problem("small2d")
    with P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, kmax=2, jacobi=0, driver=0) as s:
        assert s.solve() == -4
        assert s.info()["steps"] == 2
    with P.SylvesterADI(p.A, p.B, np.zeros_like(p.f), p.g, p.alpha, p.beta, p.tau, driver=0) as s:
        assert s.solve() == 0
        assert s.info()["steps"] == 0


# ------------------------------------------------ delayed CGS2 orthogonalisation

@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name,strategy,jacobi", [("small2d", "nobl_mid", False), ("tiny2d", "bl_mid", True)])
def test_dcgs2_parity(precision, name, strategy, jacobi):
    """GMRES with the second Gram-Schmidt pass delayed by one step (two
    sweeps per Arnoldi step) against the oracle running the same
    orthogonalisation: float64 to rounding (history within 1e-3), mixed
    precision within the inner tolerances."""
    compare(problem(name), strategy, jacobi, precision=precision, ortho="dcgs2")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dcgs2_complex_pairs(precision):
    p = W.make_problem("cplx", 14, 2, "rot2", 60.0, 12, 2, "rot2", 40.0, 2, 33, 8, real_shifts=False)
    info, ref, tr_gpu, tr_ref, dX = compare(p, "nobl_mid", True, precision=precision, ortho="dcgs2")
    assert info["is_complex"] == 1


def test_dcgs2_and_cgs2_agree():
    """Both orthogonalisations build the same Krylov bases in exact
    arithmetic: same outer and inner step counts, the same factored X."""
    p = problem("small2d")
    a = run_gpu(p, strategy="nobl_mid", jacobi=0, ortho="cgs2")
    b = run_gpu(p, strategy="nobl_mid", jacobi=0, ortho="dcgs2")
    assert a[0] == b[0] == 0 and a[1]["steps"] == b[1]["steps"]
    assert abs(a[1]["inner_its_A"] - b[1]["inner_its_A"]) <= 2 and abs(a[1]["inner_its_B"] - b[1]["inner_its_B"]) <= 2
    dX = factored_diff_fro(a[3], a[5], a[4], b[3], b[5], b[4]) / factored_fro(a[3], a[5], a[4])
    assert dX <= 1e-7, dX


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dcgs2_graph_and_host_agree_bitwise(precision):
    p = problem("tiny2d")
    out = []
    for driver in (0, 1):
        st, info, hist, Z, Y, gam = run_gpu(p, strategy="nobl_mid", jacobi=1, precision=precision,
                                            driver=driver, ortho="dcgs2")
        assert st == 0
        out.append((info["steps"], Z, Y, gam))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][3], out[1][3])


@pytest.mark.parametrize("ortho", ["cgs2", "dcgs2"])
def test_restart_stride_keeps_results_bitwise(ortho):
    """Host driver with the restart kernels launched every third device
    iteration: systems wait for their restart, their arithmetic is the same,
    so the factors agree bit for bit with the every-iteration launch."""
    p = problem("tiny2d")
    out = []
    for every in (1, 3):
        st, info, hist, Z, Y, gam = run_gpu(p, strategy="nobl_mid", jacobi=1, precision="fp32", driver=1,
                                            ortho=ortho, restart_every=every)
        assert st == 0
        out.append((info["steps"], info["inner_its_A"], Z, gam, info["ticks"]))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2]) and np.array_equal(out[0][3], out[1][3])
    assert out[1][4] >= out[0][4]          # waiting costs device iterations, never saves them
