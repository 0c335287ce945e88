"""The allocation-free CGS2 step against the regular one.

sylv_cgs2_noalloc serves callers that cannot let a library allocate GPU
memory at call time (a pool that owns the device budget, loops that must not
allocate after start-up, custom memory managers): its scratch is a static
device array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

import paper_2312_02891_gb300 as P
from oracle.gmres import cgs2_step

pytestmark = pytest.mark.gpu


def _case(torch, n, k, seed):
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((n, k)))
    w = rng.standard_normal(n)
    Vt = torch.from_numpy(np.asfortranarray(V).T.copy()).cuda()
    wt = torch.from_numpy(w).cuda()
    return V, w, Vt, wt


def test_noalloc_cgs2_matches_regular_cgs2_twice_in_a_row(torch_cuda):
    torch = torch_cuda
    # two calls in a row on the shared scratch, different sizes (the second
    # smaller, so leftovers of the first would show), each against sylv_cgs2
    for n, k, seed in ((100003, 17, 1), (4099, 5, 2)):
        V, w, Vt, wt = _case(torch, n, k, seed)
        # regular entry point: w is overwritten with the normalised vector
        w_reg = wt.clone()
        h_reg = P.sylv_cgs2(Vt, n, k, w_reg)
        # allocation-free: V with one more column that receives the result
        Vx = torch.zeros((k + 1, n), dtype=torch.float64, device="cuda")
        Vx[:k] = Vt
        h_na = P.sylv_cgs2_noalloc(Vx, n, k, wt)
        torch.cuda.synchronize()
        nw = np.linalg.norm(w)
        assert np.allclose(h_na, h_reg, rtol=0, atol=1e-13 * nw)
        assert np.allclose(Vx[k].cpu().numpy(), w_reg.cpu().numpy(), atol=1e-12)
        # and against the oracle's CGS2 step (h1 + h2, orthogonalised w)
        h_or, w_or = cgs2_step(V.T, w)
        assert np.allclose(h_na[:k], h_or, rtol=0, atol=1e-12 * nw)
        assert h_na[k] == pytest.approx(np.linalg.norm(w_or), rel=1e-10)
        assert np.allclose(Vx[k].cpu().numpy(), w_or / np.linalg.norm(w_or), atol=1e-10)
        # inputs untouched
        assert np.array_equal(Vx[:k].cpu().numpy(), Vt.cpu().numpy())
        assert np.array_equal(wt.cpu().numpy(), w)


def test_noalloc_cgs2_at_its_limits(torch_cuda):
    """k = 30 (the restart limit, where the state's last column and scale sit
    at the end of the record) and n = the largest row count the scratch
    holds (chunk table and partial sums fill the array), against sylv_cgs2."""
    torch = torch_cuda
    n, k = P.sylv_cgs2_noalloc_max_rows(), 30
    g = torch.Generator(device="cuda").manual_seed(5)
    Q, _ = torch.linalg.qr(torch.randn((n, k), dtype=torch.float64, device="cuda", generator=g))
    Vt = Q.T.contiguous()                                   # column j of V = row j of Vt
    wt = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    w_reg = wt.clone()
    h_reg = P.sylv_cgs2(Vt, n, k, w_reg)
    Vx = torch.zeros((k + 1, n), dtype=torch.float64, device="cuda")
    Vx[:k] = Vt
    h_na = P.sylv_cgs2_noalloc(Vx, n, k, wt)
    torch.cuda.synchronize()
    nw = float(torch.linalg.norm(wt))
    assert np.allclose(h_na, h_reg, rtol=0, atol=1e-13 * nw)
    assert float((Vx[k] - w_reg).abs().max()) <= 1e-12
    del Q, Vt, Vx, w_reg
    torch.cuda.empty_cache()


def test_noalloc_cgs2_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    nmax = P.sylv_cgs2_noalloc_max_rows()
    assert nmax > 1_000_000
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    # integer addresses reach the library unchecked: it refuses n = nmax + 1
    # before touching any memory
    with pytest.raises(P.SylvError, match="static scratch"):
        P.sylv_cgs2_noalloc(dummy.data_ptr(), nmax + 1, 1, dummy.data_ptr())
    # torch tensors that are too small, of another type or on the host are
    # refused by the binding before the library could write past them
    with pytest.raises(P.SylvError, match="holds 2 values"):
        P.sylv_cgs2_noalloc(dummy, 100, 3, dummy)
    with pytest.raises(P.SylvError, match="float64 CUDA tensor"):
        P.sylv_cgs2_noalloc(torch.zeros(8, dtype=torch.float32, device="cuda"), 2, 1, dummy)
    with pytest.raises(P.SylvError, match="float64 CUDA tensor"):
        P.sylv_cgs2_noalloc(torch.zeros(8, dtype=torch.float64), 2, 1, dummy)
