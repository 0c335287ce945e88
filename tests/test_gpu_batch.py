"""Batched solves: many independent Sylvester equations in one device loop
(sylv_adi_batch_*).  Every instance must match the oracle run of that
instance alone (Algorithm 1 with the same controller, inner GMRES and
options): outer step counts within +-1, computed and true residuals below
tau, and the factored solutions within the parity tolerance."""
import numpy as np
import pytest

import paper_2312_02891_gb300 as P
from paper_2312_02891_gb300 import workloads as W
from oracle.lradi import lradi
from oracle.residual import factored_diff_fro, factored_fro, lowrank_norm2, true_residual_norm2

pytestmark = pytest.mark.gpu

OPTS = dict(strategy="nobl_mid", jacobi=1, restart=30, max_inner=3000)


def small_batch(count, seed=2000, nmin=8, nmax=20, n_shifts=6):
    return W.batch_problems(count, base_seed=seed, n_shifts=n_shifts, nmin=nmin, nmax=nmax)


def check_instance(p, info, Z, Y, gam, xtol=1e-6, mixed=False):
    ref = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy=OPTS["strategy"], jacobi=True,
                restart=OPTS["restart"], max_inner=OPTS["max_inner"])
    assert ref.converged
    assert info["status"] == 0
    assert abs(info["steps"] - ref.steps) <= 1, (info["steps"], ref.steps)
    assert info["kr"] == info["steps"] * p.f.shape[1]
    assert info["rel_res_comp"] < p.tau
    nfg = lowrank_norm2(p.f, p.g)
    A, B = p.A.to_scipy(), p.B.to_scipy()
    tr = true_residual_norm2(A, B, p.f, p.g, Z, gam, Y) / nfg
    tr_ref = true_residual_norm2(A, B, p.f, p.g, ref.Z, ref.gamma, ref.Y) / nfg
    assert tr <= max(1.5 * tr_ref, 1e-8), (tr, tr_ref)
    dX = factored_diff_fro(Z, gam, Y, ref.Z, ref.gamma, ref.Y) / factored_fro(ref.Z, ref.gamma, ref.Y)
    assert dX <= xtol, dX
    return ref


@pytest.mark.parametrize("precision,ortho", [("fp64", "cgs2"), ("fp32", "cgs2"), ("fp32", "dcgs2")])
def test_batch_matches_oracle_per_instance(precision, ortho):
    probs = small_batch(6)
    assert len({(p.A.n, p.B.n, p.f.shape[1]) for p in probs}) > 1    # uneven sizes and ranks
    with P.SylvesterADIBatch(probs, precision=precision, ortho=ortho, **OPTS) as b:
        st = b.solve()
        assert st == 0, P.sylv_last_error()
        for i, p in enumerate(probs):
            Z, Y, gam = b.factors(i)
            check_instance(p, b.info(i), Z, Y, gam, mixed=precision != "fp64")
        stats = b.stats()
        assert stats["launches"] > 0 and stats["ticks"] > 0 and stats["bytes"] > 0


def test_batch_of_one_equals_single_solve():
    """A batch of one instance runs the same arithmetic as the single solver:
    same outer steps, inner iteration counts and controller history."""
    p = small_batch(1, seed=2100)[0]
    with P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, driver=0, **OPTS) as s:
        assert s.solve() == 0
        info1, hist1 = s.info(), s.history()
        Z1, Y1, g1 = s.factors()
    with P.SylvesterADIBatch([p], **OPTS) as b:
        assert b.solve() == 0
        info2, hist2 = b.info(0), b.history(0)
        Z2, Y2, g2 = b.factors(0)
    assert info1["steps"] == info2["steps"]
    assert info1["inner_its_A"] == info2["inner_its_A"] and info1["inner_its_B"] == info2["inner_its_B"]
    np.testing.assert_allclose(hist2, hist1, rtol=1e-9, atol=1e-300)
    assert factored_diff_fro(Z1, g1, Y1, Z2, g2, Y2) <= 1e-12 * factored_fro(Z1, g1, Y1)


def test_batch_mixed_real_and_complex_shifts():
    """One instance with complex conjugate shift pairs makes the whole batch
    complex; the real instances still match their oracle runs and the
    complex one gives a real X."""
    probs = small_batch(3, seed=2200)
    q = W.problem_config("small3d")
    probs.append(q)
    with P.SylvesterADIBatch(probs, **OPTS) as b:
        assert b.solve() == 0, P.sylv_last_error()
        for i, p in enumerate(probs):
            info = b.info(i)
            assert info["is_complex"] == 1
            Z, Y, gam = b.factors(i)
            if i < 3:
                check_instance(p, info, np.real(Z), np.real(Y), np.real(gam))
            else:
                assert info["rel_res_comp"] < p.tau
                X = Z @ (gam[:, None] * Y.conj().T)
                assert np.abs(X.imag).max() <= 1e-6 * np.abs(X.real).max()


def test_batch_zero_rhs_instance_and_resolve():
    """An instance with f g^* = 0 finishes at once (X = 0) without holding up
    the others; a second solve of the same batch repeats the first."""
    probs = small_batch(3, seed=2300)
    z = probs[1]
    probs[1] = W.Problem(z.name, z.A, z.B, np.zeros_like(z.f), z.g, z.alpha, z.beta, z.tau, z.opts)
    with P.SylvesterADIBatch(probs, **OPTS) as b:
        assert b.solve() == 0
        first = [b.info(i) for i in range(3)]
        assert first[1]["steps"] == 0 and first[1]["kr"] == 0
        for i in (0, 2):
            assert first[i]["steps"] > 0 and first[i]["rel_res_comp"] < probs[i].tau
        assert b.solve() == 0
        second = [b.info(i) for i in range(3)]
        for a, c in zip(first, second):
            assert a["steps"] == c["steps"] and a["inner_its_A"] == c["inner_its_A"]


def test_batch_invalid_arguments():
    probs = small_batch(2, seed=2400)
    with P.SylvesterADIBatch(probs, **OPTS) as b:
        with pytest.raises(P.SylvError):
            b.info(2)
        with pytest.raises(P.SylvError):
            P.sylv_adi_batch_info(b.h, -1)
