"""Write the stored oracle results used by the full-size parity tests and by
the benchmark's CPU-baseline extrapolation.

Calls only the oracle (and the seeded input generator); nothing here comes
from the CUDA path.  Usage:  python tests/golden/make_golden.py mid2d bl_mid
writes tests/golden/<workload>_<strategy>.json with the outer step count,
the per-step controller history, inner iteration totals, the computed and
true relative residuals, and a two-sided sketch S = P^T X Q of the factored
solution (P: n x 16, Q: m x 16 seeded Gaussian, streams 5 and 6).
``python tests/golden/make_golden.py real mid3d nobl_mid bicgstab`` writes the
real double step for complex shift pairs on a named workload, with its shifts.
``python tests/golden/make_golden.py batch64 nobl_mid bicgstab`` writes the
same per instance of the 64-instance batched workload (8 x 8 sketches, and the
shifts each instance was solved with).
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle.lradi import lradi  # noqa: E402
from oracle.residual import lowrank_norm2, true_residual_norm2  # noqa: E402
from paper_2312_02891_gb300 import workloads as W  # noqa: E402

SKETCH = 16


def sketch_mats(n, m):
    P = np.stack([W.normal(12345, 5, c, n) for c in range(SKETCH)], axis=1)
    Q = np.stack([W.normal(12345, 6, c, m) for c in range(SKETCH)], axis=1)
    return P, Q


def sketch(Z, gamma, Y, P, Q):
    """P^T (Z diag(gamma) Y^*) Q, formed through the factors."""
    return (P.T @ Z) @ (gamma[:, None] * (Y.conj().T @ Q))


def main(workload: str, strategy: str, **extra):
    p = W.problem_config(workload)
    opts = dict(strategy=strategy, jacobi=p.opts.get("jacobi", False), restart=p.opts.get("restart", 30))
    opts.update(extra)
    t0 = time.time()
    res = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, **opts)
    wall = time.time() - t0
    A, B = p.A.to_scipy(), p.B.to_scipy()
    nfg = lowrank_norm2(p.f, p.g)
    tr = true_residual_norm2(A, B, p.f, p.g, res.Z, res.gamma, res.Y) / nfg
    P, Q = sketch_mats(p.A.n, p.B.n)
    S = sketch(res.Z, res.gamma, res.Y, P, Q)
    hist = [{k: (float(np.real(v)) if not isinstance(v, (bool, np.bool_)) else bool(v))
             for k, v in h.items()} for h in res.history]
    out = dict(workload=workload, strategy=strategy, opts={k: v for k, v in opts.items()},
               tau=p.tau, n=p.A.n, m=p.B.n, r=p.r, steps=res.steps, converged=bool(res.converged),
               res_comp=res.res_comp, res_true=tr, norm_fg=nfg,
               inner_its_A=res.inner_its_A, inner_its_B=res.inner_its_B,
               sketch=np.real(S).tolist(), sketch_fro=float(np.linalg.norm(S)),
               oracle_wall_s=wall, history=hist)
    suffix = "_".join([strategy] + [f"{k}{v}" for k, v in sorted(extra.items())])
    path = os.path.join(HERE, f"{workload}_{suffix}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, res.steps, res.res_comp, tr, res.inner_its_A, res.inner_its_B, f"{wall:.0f}s")


BATCH_SKETCH = 8


def _batch_one(i, strategy, inner):
    """Oracle solve of instance i of the 64-instance batched workload."""
    p = W.batch_problems(1, base_seed=1000 + i)[0]
    t0 = time.time()
    res = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy=strategy, jacobi=True, inner=inner)
    wall = time.time() - t0
    A, B = p.A.to_scipy(), p.B.to_scipy()
    nfg = lowrank_norm2(p.f, p.g)
    tr = true_residual_norm2(A, B, p.f, p.g, res.Z, res.gamma, res.Y) / nfg
    P = np.stack([W.normal(12345, 5, c, p.A.n) for c in range(BATCH_SKETCH)], axis=1)
    Q = np.stack([W.normal(12345, 6, c, p.B.n) for c in range(BATCH_SKETCH)], axis=1)
    S = sketch(res.Z, res.gamma, res.Y, P, Q)
    # the shifts are stored with the run: the generator's selection compares
    # bounds of nearly equal candidate sets, so another BLAS/LAPACK can pick
    # another set, and the parity test must solve with the shifts used here
    return dict(instance=i, n=p.A.n, m=p.B.n, r=p.r, steps=res.steps, converged=bool(res.converged),
                res_comp=res.res_comp, res_true=tr, inner_its=res.inner_its_A + res.inner_its_B,
                alpha=[[float(np.real(a)), float(np.imag(a))] for a in p.alpha],
                beta=[[float(np.real(b)), float(np.imag(b))] for b in p.beta],
                sketch=np.real(S).tolist(), oracle_wall_s=wall)


def main_batch(strategy: str, inner: str, count: int = 64, workers: int = 8):
    """tests/golden/batch64_<strategy>_<inner>.json: per instance of the
    batched workload the outer steps, residuals and an 8 x 8 sketch of X."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    t0 = time.time()
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        rows = list(ex.map(_batch_one, range(count), [strategy] * count, [inner] * count))
    out = dict(workload="batch64", strategy=strategy, inner=inner, tau=1e-8, sketch_cols=BATCH_SKETCH,
               instances=rows, oracle_wall_s=time.time() - t0)
    path = os.path.join(HERE, f"batch64_{strategy}_{inner}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)
    print(path, sum(r["steps"] for r in rows), f"{time.time() - t0:.0f}s")


def main_real(workload: str, strategy: str, inner: str):
    """tests/golden/<workload>_<strategy>_<inner>_real.json: the real double
    step for complex shift pairs (oracle/lradi_real.py) on a named workload:
    outer steps, computed residual, inner totals, a 16 x 16 sketch of
    X = Z Gamma Y^T and the shifts it was solved with (the generator's
    choice can differ with the host's BLAS/LAPACK)."""
    from oracle.lradi_real import lradi_real
    p = W.problem_config(workload)
    t0 = time.time()
    res = lradi_real(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy=strategy,
                     jacobi=p.opts.get("jacobi", False), restart=p.opts.get("restart", 30), inner=inner)
    wall = time.time() - t0
    P, Q = sketch_mats(p.A.n, p.B.n)
    S = (P.T @ res.Z) @ res.Gamma @ (res.Y.T @ Q)
    hist = [{k: (float(np.real(v)) if not isinstance(v, (bool, np.bool_)) else bool(v))
             for k, v in h.items() if np.isscalar(v)} for h in res.history]
    out = dict(workload=workload, strategy=strategy, inner=inner, real_pairs=True, tau=p.tau,
               n=p.A.n, m=p.B.n, r=p.r, steps=res.steps, converged=bool(res.converged), res_comp=res.res_comp,
               inner_its_A=res.inner_its_A, inner_its_B=res.inner_its_B, complex_solves=res.complex_solves,
               alpha=[[float(np.real(a)), float(np.imag(a))] for a in p.alpha],
               beta=[[float(np.real(b)), float(np.imag(b))] for b in p.beta],
               sketch=np.real(S).tolist(), sketch_fro=float(np.linalg.norm(S)), oracle_wall_s=wall, history=hist)
    path = os.path.join(HERE, f"{workload}_{strategy}_{inner}_real.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, res.steps, res.res_comp, res.inner_its_A, res.inner_its_B, f"{wall:.0f}s")


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "real":
        main_real(sys.argv[2], sys.argv[3] if len(sys.argv) > 3 else "nobl_mid",
                  sys.argv[4] if len(sys.argv) > 4 else "bicgstab")
        sys.exit(0)
    if len(sys.argv) > 1 and sys.argv[1] == "batch64":
        main_batch(sys.argv[2] if len(sys.argv) > 2 else "nobl_mid", sys.argv[3] if len(sys.argv) > 3 else "bicgstab")
        sys.exit(0)
    wl = sys.argv[1] if len(sys.argv) > 1 else "mid2d"
    st = sys.argv[2] if len(sys.argv) > 2 else "bl_mid"
    kw = {}
    for a in sys.argv[3:]:
        k, v = a.split("=")
        for conv in (int, float, str):
            try:
                kw[k] = conv(v)
                break
            except ValueError:
                continue
    main(wl, st, **kw)
