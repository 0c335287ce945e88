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
        # inputs untouched
        assert np.array_equal(Vx[:k].cpu().numpy(), Vt.cpu().numpy())
        assert np.array_equal(wt.cpu().numpy(), w)


def test_noalloc_cgs2_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    nmax = P.sylv_cgs2_noalloc_max_rows()
    assert nmax > 1_000_000
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(P.SylvError, match="static scratch"):
        P.sylv_cgs2_noalloc(dummy, nmax + 1, 1, dummy)
