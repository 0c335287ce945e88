"""Kernel-level parity of the Arnoldi cycle of the inner GMRES (steps a2-a4)
in every storage precision and both orthogonalisations, element by element
against the oracle: the float32 and bfloat16 staged (cp.async) sweeps of the
tile-major basis, the stencil product and the last-block tails, at sizes that
span several work chunks with a ragged last 32-row tile, and at the full size
of the 2D benchmark operator."""
import numpy as np
import pytest

import paper_2312_02891_gb300 as P
from paper_2312_02891_gb300 import workloads as W
from oracle.gmres import arnoldi_dcgs2, cgs2_step, shifted_apply

pytestmark = pytest.mark.gpu

_OPS = {}


def _op(N):
    if N not in _OPS:
        _OPS[N] = W.convdiff(N, 2, "xy", 50.0)
    return _OPS[N]


def oracle_cgs2_arnoldi(apply, v0, k):
    """k Arnoldi steps with CGS2 (oracle.gmres.cgs2_step): V (k+1) x n, H (k+1) x k."""
    V = np.zeros((k + 1, v0.shape[0]), v0.dtype)
    H = np.zeros((k + 1, k), v0.dtype)
    V[0] = v0
    for j in range(k):
        h, w = cgs2_step(V[:j + 1], apply(V[j]))
        H[:j + 1, j] = h
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / H[j + 1, j]
    return V, H


TOL = {"fp64": 1e-10, "fp32": 2e-4, "bf16": 4e-2}


@pytest.mark.parametrize("N", [65, 512])             # n = 4225 (17 chunks, ragged tile), 262144
@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("ortho", ["cgs2", "dcgs2"])
@pytest.mark.parametrize("cplx", [False, True])
def test_arnoldi_cycle_matches_oracle(torch_cuda, N, precision, ortho, cplx):
    torch = torch_cuda
    if N == 512 and cplx and precision == "bf16":
        pytest.skip("one complex full-size case per precision pair is enough")
    M = _op(N)
    S = M.to_scipy()
    n = S.shape[0]
    k = 12
    sigma = -3.0e4 + (1.5e4j if cplx else 0.0)
    pinv = 1.0 / (S.diagonal() + sigma)
    apply = lambda x: shifted_apply(S, sigma, pinv * x)
    rng = np.random.default_rng(N)
    v0 = rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0.0)
    v0 = v0 / np.linalg.norm(v0)
    if ortho == "dcgs2":
        Vo, Ho, _ = arnoldi_dcgs2(apply, v0, k)
    else:
        Vo, Ho = oracle_cgs2_arnoldi(apply, v0, k)
    op = P.sylv_op_create(M)
    try:
        dt = torch.complex128 if cplx else torch.float64
        dv0 = torch.from_numpy(v0).to(dt).cuda()
        dV = torch.zeros((k + 1, n), dtype=dt, device="cuda")
        H = P.sylv_arnoldi(op, sigma, 1, cplx, dv0, k, dV, precision=precision, ortho=ortho)
        V = dV.cpu().numpy()
    finally:
        P.sylv_op_destroy(op)
    tol = TOL[precision]
    # the Hessenberg matrix, entry by entry, relative to its size
    assert np.max(np.abs(H - Ho)) <= tol * np.linalg.norm(Ho), np.max(np.abs(H - Ho)) / np.linalg.norm(Ho)
    # the basis vectors v_0 .. v_{k-1} (v_k as well with CGS2), row by row
    last = k if ortho == "cgs2" else k - 1
    for l in range(last + 1):
        assert np.linalg.norm(V[l] - Vo[l]) <= tol, (l, np.linalg.norm(V[l] - Vo[l]))
    if ortho == "dcgs2":
        assert not V[k].any()
    # the Arnoldi relation holds for the GPU's own basis (to the storage precision)
    AV = np.stack([apply(V[l]) for l in range(k)], axis=0)
    if ortho == "cgs2":
        res = np.linalg.norm(AV - H.T @ V) / np.linalg.norm(AV)
        assert res <= 10 * tol, res
