"""Pins of the real double step for complex conjugate shift pairs
(oracle/lradi_real.py; Sec. 3.3 "Complex shift parameters").

With exact inner solves the double step must reproduce the two steps of the
complex formulation (Algorithm 1 with (alpha, beta), (conj alpha, conj beta))
to rounding: X, w and t, for a complex beta pair, a complex alpha pair and
both.  With inexact solves: real factors, the outer steps of the complex
formulation, the tolerance of every step met by the derived second
solutions, the residual relation r2 = conj(r1) - gamma Im(r1) / Im(beta),
eq. (adi_res_inexact) over the steps of the equivalent complex formulation,
and the residual-gap estimate of eq. (upd_resgap).
"""
import numpy as np
import pytest

from paper_2312_02891_gb300 import workloads as W
from oracle.lradi import lradi
from oracle.lradi_real import lradi_real
from oracle.residual import true_residual_norm2


@pytest.fixture(scope="module")
def tiny():
    return W.problem_config("tiny2d")


@pytest.fixture(scope="module")
def t3d():
    """n = 1000, m = 512, r = 2, 3 conjugate shift pairs (one with a real beta)."""
    return W.make_problem("t3d", 10, 3, "const3", 100.0, 8, 3, "zxy", 50.0, 2, 4, 6,
                          real_shifts=False, restart=30, jacobi=True)


def _pairs(p, complex_alpha, complex_beta):
    a, b = np.real(p.alpha), np.real(p.beta)
    al, be = [], []
    for i in range(3):
        x = a[i] + (0.3j * abs(a[i]) if complex_alpha else 0)
        y = b[i] + (0.2j * abs(b[i]) if complex_beta else 0)
        al += [x, np.conj(x)]
        be += [y, np.conj(y)]
    return np.array(al), np.array(be)


@pytest.mark.parametrize("complex_alpha,complex_beta", [(False, True), (True, False), (True, True)])
def test_double_step_equals_two_complex_steps(tiny, complex_alpha, complex_beta):
    al, be = _pairs(tiny, complex_alpha, complex_beta)
    rc = lradi(tiny.A, tiny.B, tiny.f, tiny.g, al, be, 1e-8, inner="direct", kmax=6)
    rr = lradi_real(tiny.A, tiny.B, tiny.f, tiny.g, al, be, 1e-8, inner="direct", kmax=6)
    assert rc.steps == rr.steps == 6
    assert rr.Z.dtype == rr.Y.dtype == rr.Gamma.dtype == np.float64
    Xc = (rc.Z * rc.gamma[None, :]) @ rc.Y.conj().T
    Xr = rr.Z @ rr.Gamma @ rr.Y.T
    assert np.linalg.norm(Xc - Xr) <= 1e-13 * np.linalg.norm(Xc)
    assert np.linalg.norm(rc.w - rr.w) <= 1e-13 * np.linalg.norm(rc.w)
    assert np.linalg.norm(rc.t - rr.t) <= 1e-13 * np.linalg.norm(rc.t)
    # one complex column solve per pair and column on each side with a complex shift
    r = tiny.r
    assert rr.complex_solves == 3 * r * (int(complex_alpha) + int(complex_beta))
    # Gamma is block diagonal with 2 x 2 blocks (kron I_r)
    G = rr.Gamma
    for q in range(3):
        s = slice(2 * r * q, 2 * r * (q + 1))
        off = G[s].copy()
        off[:, s] = 0.0
        assert not off.any()


@pytest.mark.parametrize("complex_alpha,complex_beta", [(False, True), (True, False)])
def test_double_step_with_a_wrong_relation_fails(tiny, monkeypatch, complex_alpha, complex_beta):
    """The pin above is sensitive: with the sign of the Im(x1) term flipped
    in the derived second solution (a plausible slip in the partial-fraction
    step) the factors no longer reproduce the complex formulation."""
    import oracle.lradi_real as LR
    al, be = _pairs(tiny, complex_alpha, complex_beta)
    rc = lradi(tiny.A, tiny.B, tiny.f, tiny.g, al, be, 1e-8, inner="direct", kmax=2)
    Xc = (rc.Z * rc.gamma[None, :]) @ rc.Y.conj().T
    good = LR._coeffs_complex
    monkeypatch.setattr(LR, "_coeffs_complex", lambda c, im: good(-c, im))
    try:
        rr = LR.lradi_real(tiny.A, tiny.B, tiny.f, tiny.g, al, be, 1e-8, inner="direct", kmax=2)
        differs = np.linalg.norm(Xc - rr.Z @ rr.Gamma @ rr.Y.T) > 1e-6 * np.linalg.norm(Xc)
    except FloatingPointError:
        differs = True
    assert differs


@pytest.mark.parametrize("inner", ["gmres", "bicgstab"])
def test_inexact_real_formulation(t3d, inner):
    p = t3d
    A, B = p.A.to_scipy(), p.B.to_scipy()
    nfg = np.linalg.norm(p.f @ p.g.T, 2)
    rc = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner=inner, strategy="bl_mid", jacobi=True)
    rr = lradi_real(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, inner=inner, strategy="bl_mid",
                    jacobi=True, keep_inner_residuals=True)
    assert rc.converged and rr.converged and abs(rc.steps - rr.steps) <= 1
    Xc = (rc.Z * rc.gamma[None, :]) @ rc.Y.conj().T
    Xr = rr.Z @ rr.Gamma @ rr.Y.T
    assert np.linalg.norm(Xc - Xr) <= 1e-6 * np.linalg.norm(Xc)
    R = A @ Xr + Xr @ B + p.f @ p.g.T
    assert np.linalg.norm(R, 2) <= 3 * p.tau * nfg
    # every step, the derived second ones included, meets its tolerance
    for h in rr.history:
        assert max(h["nrA"]) <= h["dA"] * (1 + 1e-12) and max(h["nrB"]) <= h["dB"] * (1 + 1e-12)
    # eq. (adi_res_inexact) over the steps of the equivalent complex formulation
    gap = sum((s["gamma"] * s["rA"]) @ s["y"].conj().T + (s["gamma"] * s["z"]) @ s["rB"].conj().T
              for s in rr.steps_complex)
    assert np.linalg.norm(R - (rr.w @ rr.t.T - gap)) <= 1e-10 * np.linalg.norm(R) + 1e-14 * nfg
    assert np.linalg.norm(gap, 2) <= rr.history[-1]["u"] + rr.history[-1]["v"] + 1e-20
    # the relation of the derived second solution's residual (complex beta)
    L = len(p.alpha)
    checked = False
    for i in range(0, len(rr.steps_complex) - 1):
        s1, s2 = rr.steps_complex[i], rr.steps_complex[i + 1]
        if np.iscomplexobj(s1["z"]) and np.conj(s1["gamma"]) == s2["gamma"] and np.imag(s1["gamma"]) != 0:
            k = i % L
            b = p.beta[k]
            if np.imag(b) != 0 and np.conj(b) == p.beta[(k + 1) % L]:
                r1, r2 = s1["rA"], s2["rA"]
                pred = np.conj(r1) - s1["gamma"] * r1.imag / np.imag(b)
                assert np.linalg.norm(r2 - pred) <= 1e-6 * np.linalg.norm(r2) + 1e-14 * np.linalg.norm(p.f)
                checked = True
                break
    assert checked
    # one complex column solve per pair and side with a complex shift
    assert rr.complex_solves < 2 * rr.steps * p.r


@pytest.mark.parametrize("complex_alpha,complex_beta", [(False, True), (True, False), (None, None)])
@pytest.mark.parametrize("inner", ["gmres", "bicgstab"])
def test_inexact_pairs_meet_the_column_targets(tiny, complex_alpha, complex_beta, inner):
    """With one side's shift of the pair real (two real solves there, to
    delta / 2 and delta / (2 |gamma|)) and the other complex (one complex
    solve to delta / (1 + |gamma| / |Im shift|)): every column of every step of
    the equivalent complex formulation, the derived second ones included,
    meets the per-column target delta / r of the pair's controller evaluation
    (Sec. 3.3), and u, v accumulate eq. (upd_resgap) over both steps of each
    pair."""
    if complex_alpha is None:
        # real steps between the pairs: the problem's real shifts with one
        # complex-beta pair inserted after the first two
        a, b = np.real(tiny.alpha), np.real(tiny.beta)
        al = np.array([a[0], a[1], a[2], a[2]] + list(a[3:]), dtype=complex)
        be = np.array([b[0], b[1], b[2] + 0.2j * abs(b[2]), b[2] - 0.2j * abs(b[2])] + list(b[3:]))
    else:
        al, be = _pairs(tiny, complex_alpha, complex_beta)
    r = tiny.r
    rr = lradi_real(tiny.A, tiny.B, tiny.f, tiny.g, al, be, 1e-8, inner=inner, strategy="nobl_mid",
                    keep_inner_residuals=True, kmax=30)
    if complex_alpha is None:
        assert any(h["pair"] for h in rr.history) and any(not h["pair"] for h in rr.history)
    assert rr.converged
    j = 0
    u = v = 0.0
    for h in rr.history:
        for _ in range(2 if h["pair"] else 1):
            st = rr.steps_complex[j]
            j += 1
            ca = np.linalg.norm(st["rA"], axis=0)
            cb = np.linalg.norm(st["rB"], axis=0)
            assert np.all(ca <= h["dA"] / r * (1 + 1e-9)), (h["k"], ca, h["dA"] / r)
            assert np.all(cb <= h["dB"] / r * (1 + 1e-9)), (h["k"], cb, h["dB"] / r)
            g = abs(st["gamma"])
            u += g * np.linalg.norm(st["z"], 2) * np.linalg.norm(st["rB"], 2)
            v += g * np.linalg.norm(st["y"], 2) * np.linalg.norm(st["rA"], 2)
        assert h["u"] == pytest.approx(u, rel=1e-10) and h["v"] == pytest.approx(v, rel=1e-10)
    assert j == len(rr.steps_complex)


def test_unpaired_complex_shift_is_rejected(tiny):
    al = np.array([-100.0 + 50j, -200.0])
    be = np.array([-80.0, -90.0])
    with pytest.raises(ValueError):
        lradi_real(tiny.A, tiny.B, tiny.f, tiny.g, al, be, 1e-8, inner="direct", kmax=2)


def test_zero_rhs_and_real_shifts(tiny):
    """f g^* = 0 gives X = 0 without steps; with real shifts only, the
    real formulation is Algorithm 1's real iteration."""
    z = lradi_real(tiny.A, tiny.B, 0 * tiny.f, tiny.g, tiny.alpha, tiny.beta, 1e-8, inner="direct")
    assert z.steps == 0 and z.converged and z.Z.shape[1] == 0
    rc = lradi(tiny.A, tiny.B, tiny.f, tiny.g, tiny.alpha, tiny.beta, 1e-8, inner="direct", kmax=5)
    rr = lradi_real(tiny.A, tiny.B, tiny.f, tiny.g, tiny.alpha, tiny.beta, 1e-8, inner="direct", kmax=5)
    Xc = (rc.Z * rc.gamma[None, :]) @ rc.Y.conj().T
    assert np.linalg.norm(Xc - rr.Z @ rr.Gamma @ rr.Y.T) <= 1e-14 * np.linalg.norm(Xc)
