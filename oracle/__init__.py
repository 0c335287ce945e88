"""CPU FP64 oracle for the inexact low-rank Sylvester ADI method.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the package
and the CPU-baseline leg of the benchmark may import this package.  The CUDA
path never calls it and shares no code with it; the two meet only through
the seeded inputs of ``paper_2312_02891_gb300.workloads``.

The oracle is written for a reader who checks it against the paper
(Kuerschner, "Inexact linear solves in the low-rank ADI iteration for large
Sylvester equations"): plain numpy / scipy, float64 (complex128 for complex
shifts), no blocking or fusion.

Modules
-------
controller  eqs. (ADI_relax1_prak), (upd_resgap), (ADI_relax2_prak),
            (simple_tols), (one_side): the inner tolerances delta^A_k, delta^B_k.
gmres       restarted GMRES(m) with right Jacobi preconditioning, the inner
            solver of the shifted systems (Sec. 3.3 "Further implementation
            aspects": per-column solves, ||r(:,l)|| <= delta_k / r).
lradi       Algorithm 1 (inexact LR-ADI) with direct or GMRES inner solves,
            for eq. (sylv) and (with M, C) the generalized eq. (gsylv).
lradi_real  Algorithm 1 with a real double step per complex conjugate shift
            pair (Sec. 3.3 "Complex shift parameters"): one complex solve per
            pair and side, real factors Z, Gamma, Y.
residual    exact norms through low-rank factors: ||w t^*||, the true
            residual of eq. (adi_res_inexact), differences of factored X.
dense       the plain definition of the solution of eq. (sylv): Kronecker
            solve and Bartels-Stewart (scipy), for pinning on small inputs.

Pins: every function is checked in tests/test_oracle_*.py (the
generalized path in tests/test_oracle_generalized.py) against closed
forms, dense solves, the identities of Theorems 1 and 2, and the bound of
Theorem 3.  Functions without such a pin say "parity unpinned" in their
docstring.
"""
