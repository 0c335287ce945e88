"""The C ABI library loads and exports every entry point declared in
include/sylv_adi.h; host-side argument checks that need no GPU."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

import paper_2312_02891_gb300 as P

HEADER = Path(__file__).resolve().parents[1] / "include" / "sylv_adi.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(sylv_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("sylv_adi_create", "sylv_adi_solve", "sylv_adi_factors", "sylv_op_apply",
                 "sylv_cgs2", "sylv_gmres", "sylv_controller_eval"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(P.EXPORTED) == declared_functions()


def test_opts_default_matches_paper_settings(lib):
    o = P.sylv_opts_default()
    assert o.xi == 1.0 and o.kmax == 50 and o.dmax_A == 0.1 and o.dmax_B == 0.1
    assert o.strategy == P.STRATEGIES["bl_mid"] and o.restart == 30


def _csr_struct(n, rp, ci, v):
    rp = np.asarray(rp, np.int32); ci = np.asarray(ci, np.int32); v = np.asarray(v, np.float64)
    return (rp, ci, v), P.SylvCsr(n, n, int(rp[-1]) if len(rp) else 0, rp.ctypes.data,
                                  ci.ctypes.data, v.ctypes.data, 0)


def test_invalid_arguments_rejected_without_gpu(lib):
    out = C.c_void_p()
    # non-square
    keep, s = _csr_struct(2, [0, 1, 2], [0, 1], [1.0, 1.0])
    s.n_cols = 3
    assert lib.sylv_op_create(C.byref(s), 0, C.byref(out)) == -1
    # column out of range
    keep, s = _csr_struct(2, [0, 1, 2], [0, 5], [1.0, 1.0])
    assert lib.sylv_op_create(C.byref(s), 0, C.byref(out)) == -1
    assert "out of range" in P.sylv_last_error()
    # decreasing rowptr
    keep, s = _csr_struct(2, [0, 2, 1], [0, 1], [1.0, 1.0])
    assert lib.sylv_op_create(C.byref(s), 0, C.byref(out)) == -1
    # null descriptor
    assert lib.sylv_op_create(None, 0, C.byref(out)) == -1
    # adi_create: rank 0 and rank above the build limit
    keep, s = _csr_struct(2, [0, 1, 2], [0, 1], [-1.0, -2.0])
    f = np.ones(2)
    sh = (P.SylvShift * 1)(P.SylvShift(-1.0, 0.0))
    pd = f.ctypes.data_as(C.POINTER(C.c_double))
    assert lib.sylv_adi_create(C.byref(s), C.byref(s), pd, pd, 0, sh, sh, 1, 1e-8, None, None, C.byref(out)) == -1
    assert lib.sylv_adi_create(C.byref(s), C.byref(s), pd, pd, 5, sh, sh, 1, 1e-8, None, None, C.byref(out)) == -8
    # tolerance outside (0, 1)
    assert lib.sylv_adi_create(C.byref(s), C.byref(s), pd, pd, 1, sh, sh, 1, 0.0, None, None, C.byref(out)) == -1
    # unpaired complex shift
    shc = (P.SylvShift * 1)(P.SylvShift(-1.0, 1.0))
    assert lib.sylv_adi_create(C.byref(s), C.byref(s), pd, pd, 1, shc, shc, 1, 1e-8, None, None, C.byref(out)) == -1
    assert "conjugate" in P.sylv_last_error()
    # restart beyond the build limit
    o = P.sylv_opts_default(restart=31)
    assert lib.sylv_adi_create(C.byref(s), C.byref(s), pd, pd, 1, sh, sh, 1, 1e-8, C.byref(o), None, C.byref(out)) == -8
    # batch: empty batch, and a bad instance named in the message
    assert lib.sylv_adi_batch_create(0, None, None, None, C.byref(out)) == -1
    probs = (P.SylvProblem * 2)(
        P.SylvProblem(C.pointer(s), C.pointer(s), f.ctypes.data, f.ctypes.data, 1, C.addressof(sh), C.addressof(sh), 1, 1e-8),
        P.SylvProblem(C.pointer(s), C.pointer(s), f.ctypes.data, f.ctypes.data, 1, C.addressof(shc), C.addressof(shc), 1, 1e-8))
    assert lib.sylv_adi_batch_create(2, probs, None, None, C.byref(out)) == -1
    assert "instance 1" in P.sylv_last_error() and "conjugate" in P.sylv_last_error()
    # a null batch handle
    assert lib.sylv_adi_batch_solve(None) == -1
    assert lib.sylv_adi_batch_destroy(None) == 0


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    """No CPU fallback: a missing shared library is an error."""
    import importlib
    mod = importlib.reload(P)
    monkeypatch.setattr(mod, "lib_path", lambda: tmp_path / "missing.so")
    monkeypatch.setattr(mod, "_LIB", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mod.load()
    importlib.reload(P)


def test_noalloc_entry_point_refuses_bad_sizes_without_gpu(lib):
    """The allocation-free CGS2 step checks its sizes before any device call:
    rows beyond what its static scratch holds, a basis size outside
    1..restart and null pointers are refused with a message.  The pointers
    given here are never dereferenced (the call returns first)."""
    mx = P.sylv_cgs2_noalloc_max_rows()
    assert mx > 100000
    h = np.zeros(8)
    hp = h.ctypes.data_as(C.POINTER(C.c_double))
    fake = C.c_void_p(16)
    assert lib.sylv_cgs2_noalloc(fake, mx + 1, 5, fake, hp, None) == -1
    assert "static scratch" in P.sylv_last_error()
    assert lib.sylv_cgs2_noalloc(fake, 1000, 0, fake, hp, None) == -1
    assert lib.sylv_cgs2_noalloc(fake, 1000, 31, fake, hp, None) == -1
    assert lib.sylv_cgs2_noalloc(None, 1000, 5, fake, hp, None) == -1
    assert lib.sylv_cgs2_noalloc(fake, 0, 5, fake, hp, None) == -1


def test_noalloc_binding_checks_its_tensors():
    """The binding refuses tensors the library must not write into before
    it calls the library: host tensors and other dtypes (the refusal of
    device buffers smaller than n x (k + 1) or n needs device tensors)."""
    torch = pytest.importorskip("torch")
    n, k = 64, 3
    v = torch.zeros(n * (k + 1), dtype=torch.float64)
    w = torch.zeros(n, dtype=torch.float64)
    for V, W_ in ((v, w), (v.float(), w), (v, w.float())):
        with pytest.raises(P.SylvError, match="contiguous float64 CUDA tensor"):
            P.sylv_cgs2_noalloc(V, n, k, W_)
