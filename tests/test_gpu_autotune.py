"""The work-chunk autotuner (opts.autotune): candidates timed at create on
the actual systems, the fastest kept; the solves it configures still match
the oracle (the chunk size changes only the summation order of the
reductions)."""
import numpy as np
import pytest

import paper_2312_02891_gb300 as P
from paper_2312_02891_gb300 import workloads as W
from oracle.lradi import lradi
from oracle.residual import factored_diff_fro, factored_fro

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("inner,ortho", [("bicgstab", "cgs2"), ("gmres", "dcgs2"), ("gmres", "cgs2")])
def test_batch_autotune_picks_a_timed_candidate_and_keeps_parity(inner, ortho):
    probs = W.batch_problems(5, base_seed=2100, n_shifts=6, nmin=12, nmax=40)
    with P.SylvesterADIBatch(probs, strategy="nobl_mid", precision="fp64", jacobi=1, inner=inner, ortho=ortho,
                             autotune=1) as bt:
        tune = bt.tuning()
        assert len(tune["candidates"]) >= 2
        assert tune["rows_per_chunk"] in tune["candidates"]
        assert all(ms > 0 for ms in tune["candidates"].values())
        assert tune["candidates"][tune["rows_per_chunk"]] == min(tune["candidates"].values())
        assert bt.solve() == 0, P.sylv_last_error()
        for i, p in enumerate(probs):
            info = bt.info(i)
            Z, Y, gam = bt.factors(i)
            ref = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy="nobl_mid", jacobi=True, inner=inner,
                        ortho=ortho)
            assert abs(info["steps"] - ref.steps) <= 1
            dX = factored_diff_fro(Z, gam, Y, ref.Z, ref.gamma, ref.Y) / factored_fro(ref.Z, ref.gamma, ref.Y)
            assert dX <= 1e-6, (i, dX)


def test_single_autotune_and_fixed_chunks_agree():
    p = W.problem_config("small2d")
    out = []
    for kw in (dict(autotune=1), dict(rows_per_chunk=256)):
        with P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy="nobl_mid", jacobi=1,
                            inner="bicgstab", **kw) as s:
            assert s.solve() == 0
            out.append((s.info()["steps"], s.factors(), s.tuning()))
    assert len(out[0][2]["candidates"]) >= 1 and not out[1][2]["candidates"]
    assert out[1][2]["rows_per_chunk"] == 256
    assert abs(out[0][0] - out[1][0]) <= 1
    Z1, Y1, g1 = out[0][1]
    Z2, Y2, g2 = out[1][1]
    assert factored_diff_fro(Z1, g1, Y1, Z2, g2, Y2) <= 1e-6 * factored_fro(Z2, g2, Y2)
