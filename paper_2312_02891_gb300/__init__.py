"""GB300 inexact low-rank Sylvester ADI: Python binding of libsylv_adi.so.

The functions below carry the names of the C ABI in include/sylv_adi.h and
only marshal arguments (numpy arrays for host data, integer device pointers
or objects with ``data_ptr()`` such as torch CUDA tensors for device data).
Every step of the computation runs in the CUDA library; if the library is
missing the calls raise instead of computing anything on the CPU.

``SylvesterADI`` wraps a solver handle for numpy inputs.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

__all__ = [
    "SylvError", "lib_path", "load", "SylvOpts", "SylvInfo", "SylvShift", "SylvCsr",
    "STRATEGIES", "sylv_opts_default", "sylv_last_error", "sylv_op_create", "sylv_op_create_g",
    "sylv_adi_create_g", "sylv_op_format",
    "sylv_op_apply", "sylv_op_destroy", "sylv_cgs2", "sylv_gmres", "sylv_bicgstab", "sylv_arnoldi",
    "sylv_controller_eval",
    "sylv_adi_create", "sylv_adi_set_rhs", "sylv_adi_set_rhs_device", "sylv_adi_solve",
    "sylv_adi_info", "sylv_adi_history", "sylv_adi_factors", "sylv_adi_destroy", "SylvesterADI",
    "sylv_adi_profile", "sylv_adi_kernel_stats", "sylv_adi_core", "sylv_bicgstab", "sylv_arnoldi",
    "HIST_COLUMNS", "EXPORTED", "KERNELS",
    "SylvProblem", "sylv_adi_batch_create", "sylv_adi_batch_solve", "sylv_adi_batch_info",
    "sylv_adi_batch_history", "sylv_adi_batch_factors", "sylv_adi_batch_stats", "sylv_adi_batch_destroy",
    "SylvesterADIBatch", "sylv_adi_batch_set_rhs", "sylv_adi_batch_profile", "sylv_adi_batch_kernel_stats",
    "sylv_adi_tuning", "sylv_adi_batch_tuning",
]

SYLV_OK = 0
ERRORS = {-1: "INVALID", -2: "CUDA", -3: "NOMEM", -4: "MAXIT", -5: "INNER_STALL",
          -6: "NONFINITE", -7: "NOT_SOLVED", -8: "UNSUPPORTED"}
WARNINGS = (-4, -5)      # solve finished, factors valid
STRATEGIES = {"fixed": 0, "nobl_mid": 1, "bl_mid": 2, "nobl_A": 3, "bl_A": 4, "nobl_B": 5, "bl_B": 6}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2}
ORTHO = {"cgs2": 0, "dcgs2": 1}
INNER = {"gmres": 0, "bicgstab": 1}
HIST_COLUMNS = ("k", "alpha", "beta", "dA", "dB", "eps_hat", "nrA", "nrB", "itsA", "itsB",
                "u", "v", "res_comp", "N_w")
EXPORTED = (
    "sylv_last_error", "sylv_opts_default", "sylv_op_create", "sylv_op_create_g", "sylv_op_format",
    "sylv_op_apply", "sylv_op_destroy", "sylv_cgs2", "sylv_gmres", "sylv_bicgstab", "sylv_arnoldi",
    "sylv_controller_eval", "sylv_adi_create",
    "sylv_adi_create_g", "sylv_adi_set_rhs", "sylv_adi_set_rhs_device", "sylv_adi_solve", "sylv_adi_info",
    "sylv_adi_history", "sylv_adi_factors", "sylv_adi_destroy", "sylv_adi_core", "sylv_adi_profile",
    "sylv_adi_kernel_stats", "sylv_cgs2_noalloc", "sylv_cgs2_noalloc_max_rows",
    "sylv_adi_batch_create", "sylv_adi_batch_solve", "sylv_adi_batch_info", "sylv_adi_batch_history",
    "sylv_adi_batch_factors", "sylv_adi_batch_stats", "sylv_adi_batch_destroy", "sylv_adi_batch_set_rhs",
    "sylv_adi_batch_profile", "sylv_adi_batch_kernel_stats", "sylv_adi_tuning", "sylv_adi_batch_tuning",
)
KERNELS = ("arnoldi_spmv", "cgs_pass2", "cgs_pass3", "restart_update", "restart_residual",
           "adi_controller", "adi_step_init", "adi_gram")


class SylvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SylvCsr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("val", C.c_void_p),
                ("on_device", C.c_int32)]


class SylvShift(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class SylvOpts(C.Structure):
    _fields_ = [("xi", C.c_double), ("dmin_A", C.c_double), ("dmin_B", C.c_double),
                ("dmax_A", C.c_double), ("dmax_B", C.c_double), ("kmax", C.c_int32),
                ("strategy", C.c_int32), ("fixed_tol", C.c_double), ("restart", C.c_int32),
                ("max_inner", C.c_int32), ("precision", C.c_int32), ("jacobi", C.c_int32),
                ("bl_clamp", C.c_int32), ("rows_per_chunk", C.c_int32), ("driver", C.c_int32),
                ("ortho", C.c_int32), ("restart_every", C.c_int32), ("inner", C.c_int32),
                ("real_pairs", C.c_int32), ("autotune", C.c_int32)]


class SylvProblem(C.Structure):
    _fields_ = [("A", C.POINTER(SylvCsr)), ("B", C.POINTER(SylvCsr)), ("f", C.c_void_p),
                ("g", C.c_void_p), ("r", C.c_int32), ("alpha", C.c_void_p), ("beta", C.c_void_p),
                ("n_shifts", C.c_int32), ("tol", C.c_double)]


class SylvInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps", C.c_int32), ("kr", C.c_int32),
                ("is_complex", C.c_int32), ("rel_res_comp", C.c_double), ("norm_fg", C.c_double),
                ("inner_its_A", C.c_int64), ("inner_its_B", C.c_int64),
                ("inner_restarts", C.c_int64), ("stalled_solves", C.c_int32),
                ("ticks", C.c_int32), ("launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def lib_path() -> Path:
    return Path(__file__).resolve().parent / "_lib" / "libsylv_adi.so"


def load():
    """Load libsylv_adi.so (built by _build.build()); raise if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = lib_path()
    if not p.exists():
        raise RuntimeError(f"{p} is not built: run paper_2312_02891_gb300._build.build() "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    L = C.CDLL(str(p))
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    pd, pi32 = C.POINTER(C.c_double), C.POINTER(C.c_int32)
    sig = {
        "sylv_last_error": ([], C.c_char_p),
        "sylv_opts_default": ([C.POINTER(SylvOpts)], C.c_int),
        "sylv_op_create": ([C.POINTER(SylvCsr), i32, C.POINTER(vp)], C.c_int),
        "sylv_op_create_g": ([C.POINTER(SylvCsr), C.POINTER(SylvCsr), i32, C.POINTER(vp)], C.c_int),
        "sylv_op_format": ([vp, pi32, pi32, pi32], C.c_int),
        "sylv_op_apply": ([vp, SylvShift, i32, i32, vp, vp, i32, vp], C.c_int),
        "sylv_op_destroy": ([vp], C.c_int),
        "sylv_cgs2": ([vp, i32, i32, vp, vp, i32, vp], C.c_int),
        "sylv_gmres": ([vp, SylvShift, i32, i32, vp, vp, i32, d, i32, i32, i32, pi32, pd, pd, vp], C.c_int),
        "sylv_bicgstab": ([vp, SylvShift, i32, i32, vp, vp, i32, d, i32, i32, pi32, pd, pd, vp], C.c_int),
        "sylv_arnoldi": ([vp, SylvShift, i32, i32, vp, i32, i32, i32, vp, vp, vp], C.c_int),
        "sylv_controller_eval": ([C.POINTER(SylvOpts), i32, pd, pd], C.c_int),
        "sylv_adi_create": ([C.POINTER(SylvCsr), C.POINTER(SylvCsr), pd, pd, i32,
                             C.POINTER(SylvShift), C.POINTER(SylvShift), i32, d,
                             C.POINTER(SylvOpts), vp, C.POINTER(vp)], C.c_int),
        "sylv_adi_create_g": ([C.POINTER(SylvCsr), C.POINTER(SylvCsr), C.POINTER(SylvCsr),
                               C.POINTER(SylvCsr), pd, pd, i32, C.POINTER(SylvShift), C.POINTER(SylvShift),
                               i32, d, C.POINTER(SylvOpts), vp, C.POINTER(vp)], C.c_int),
        "sylv_adi_set_rhs": ([vp, pd, pd], C.c_int),
        "sylv_adi_set_rhs_device": ([vp, vp, vp], C.c_int),
        "sylv_adi_solve": ([vp], C.c_int),
        "sylv_adi_info": ([vp, C.POINTER(SylvInfo)], C.c_int),
        "sylv_adi_history": ([vp, pd, i32, pi32], C.c_int),
        "sylv_adi_factors": ([vp, vp, vp, vp, i32, pi32, pi32], C.c_int),
        "sylv_adi_destroy": ([vp], C.c_int),
        "sylv_adi_core": ([vp, pd, i32, pi32], C.c_int),
        "sylv_adi_profile": ([vp, i32], C.c_int),
        "sylv_adi_kernel_stats": ([vp, pd, pd, pd, C.POINTER(C.c_int64)], C.c_int),
        "sylv_cgs2_noalloc": ([vp, i32, i32, vp, pd, vp], C.c_int),
        "sylv_cgs2_noalloc_max_rows": ([], C.c_int),
        "sylv_adi_batch_create": ([i32, C.POINTER(SylvProblem), C.POINTER(SylvOpts), vp, C.POINTER(vp)], C.c_int),
        "sylv_adi_batch_solve": ([vp], C.c_int),
        "sylv_adi_batch_info": ([vp, i32, C.POINTER(SylvInfo)], C.c_int),
        "sylv_adi_batch_history": ([vp, i32, pd, i32, pi32], C.c_int),
        "sylv_adi_batch_factors": ([vp, i32, vp, vp, vp, i32, pi32, pi32], C.c_int),
        "sylv_adi_batch_stats": ([vp, C.POINTER(C.c_int64), pd, pd, C.POINTER(C.c_int64)], C.c_int),
        "sylv_adi_batch_destroy": ([vp], C.c_int),
        "sylv_adi_batch_set_rhs": ([vp, i32, pd, pd], C.c_int),
        "sylv_adi_tuning": ([vp, pi32, pi32, pd, i32, pi32], C.c_int),
        "sylv_adi_batch_tuning": ([vp, pi32, pi32, pd, i32, pi32], C.c_int),
        "sylv_adi_batch_profile": ([vp, i32], C.c_int),
        "sylv_adi_batch_kernel_stats": ([vp, pd, pd, pd, C.POINTER(C.c_int64)], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = L
    return L


def sylv_last_error() -> str:
    return load().sylv_last_error().decode()


def _check(rc: int, allow_warn: bool = False) -> int:
    if rc == SYLV_OK or (allow_warn and rc in WARNINGS):
        return rc
    raise SylvError(rc, sylv_last_error())


def _ptr(x) -> int | None:
    """Device or host address of x (int, torch tensor, numpy array) or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return getattr(s, "cuda_stream", None)


def _shift(s) -> SylvShift:
    s = complex(s)
    return SylvShift(s.real, s.imag)


def sylv_opts_default(**overrides) -> SylvOpts:
    o = SylvOpts()
    _check(load().sylv_opts_default(C.byref(o)))
    for k, v in overrides.items():
        if k == "strategy" and isinstance(v, str):
            v = STRATEGIES[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "ortho" and isinstance(v, str):
            v = ORTHO[v]
        if k == "inner" and isinstance(v, str):
            v = INNER[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class _HostCsr:
    """Keeps the contiguous host arrays of a CSR alive while C reads them."""

    def __init__(self, n, rowptr, colind, val):
        self.rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.ci = np.ascontiguousarray(colind, dtype=np.int32)
        self.v = np.ascontiguousarray(val, dtype=np.float64)
        self.s = SylvCsr(n, n, int(self.rp[-1]), self.rp.ctypes.data, self.ci.ctypes.data,
                         self.v.ctypes.data, 0)


def _csr(M) -> _HostCsr:
    if hasattr(M, "rowptr"):
        return _HostCsr(M.n, M.rowptr, M.colind, M.val)
    return _HostCsr(M.shape[0], M.indptr, M.indices, M.data)   # scipy.sparse.csr_matrix


def sylv_op_create(M, transpose: bool = False, mass=None) -> int:
    """Device operator Op (or Op + sigma Mass with a mass matrix, for the
    generalized equation)."""
    h = _csr(M)
    out = C.c_void_p()
    if mass is None:
        _check(load().sylv_op_create(C.byref(h.s), int(transpose), C.byref(out)))
    else:
        hm = _csr(mass)
        _check(load().sylv_op_create_g(C.byref(h.s), C.byref(hm.s), int(transpose), C.byref(out)))
    return out.value


sylv_op_create_g = sylv_op_create


def sylv_op_format(op) -> tuple[int, int, int]:
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().sylv_op_format(op, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def sylv_op_apply(op, sigma, jacobi, is_complex, X, Y, ncols, stream=None) -> None:
    _check(load().sylv_op_apply(op, _shift(sigma), int(jacobi), int(is_complex), _ptr(X), _ptr(Y),
                                int(ncols), _stream(stream)))


def sylv_op_destroy(op) -> None:
    _check(load().sylv_op_destroy(op))


def sylv_cgs2(V, n, k, w, is_complex=False, stream=None) -> np.ndarray:
    """CGS2 of device vector w against k device columns V; returns h (k+1)."""
    h = np.zeros(2 * (k + 1) if is_complex else k + 1)
    _check(load().sylv_cgs2(_ptr(V), int(n), int(k), _ptr(w), h.ctypes.data, int(is_complex),
                            _stream(stream)))
    return h.view(np.complex128) if is_complex else h


def sylv_cgs2_noalloc(V, n, k, w, stream=None) -> np.ndarray:
    """CGS2 step that allocates no GPU memory (static scratch in the library).

    V: device n x (k+1) float64, column-major; column k receives the
    normalised result.  w: device n float64 (read only).  Returns h (k+1).
    Torch tensors are checked (CUDA, float64, contiguous, large enough)
    before the library writes into them; integer addresses are passed on as
    they are."""
    n, k = int(n), int(k)
    for name, x, need in (("V", V, n * (k + 1)), ("w", w, n)):
        if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
            if not x.is_cuda or str(x.dtype) != "torch.float64" or not x.is_contiguous():
                raise SylvError(-1, f"sylv_cgs2_noalloc: {name} must be a contiguous float64 CUDA tensor")
            if x.numel() < need:
                raise SylvError(-1, f"sylv_cgs2_noalloc: {name} holds {x.numel()} values, needs {need}")
    h = np.zeros(k + 1)
    _check(load().sylv_cgs2_noalloc(_ptr(V), int(n), int(k), _ptr(w),
                                    h.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))
    return h


def sylv_cgs2_noalloc_max_rows() -> int:
    return int(load().sylv_cgs2_noalloc_max_rows())


def sylv_gmres(op, sigma, jacobi, is_complex, B, X, ncols, tol, restart, max_iters,
               want_hist=False, stream=None, precision="fp64"):
    """Returns (status, iters[ncols], resnorm[ncols], hist or None)."""
    iters = np.zeros(ncols, dtype=np.int32)
    res = np.zeros(ncols)
    hist = np.zeros((ncols, max_iters)) if want_hist else None
    rc = load().sylv_gmres(op, _shift(sigma), int(jacobi), int(is_complex), _ptr(B), _ptr(X),
                           int(ncols), float(tol), int(restart), int(max_iters),
                           PRECISIONS.get(precision, precision),
                           iters.ctypes.data_as(C.POINTER(C.c_int32)),
                           res.ctypes.data_as(C.POINTER(C.c_double)),
                           hist.ctypes.data_as(C.POINTER(C.c_double)) if want_hist else None,
                           _stream(stream))
    _check(rc, allow_warn=True)
    return rc, iters, res, hist


def sylv_bicgstab(op, sigma, jacobi, is_complex, B, X, ncols, tol, max_iters,
                  want_hist=False, stream=None, precision="fp64"):
    """BiCGstab for ncols columns; returns (status, iters[ncols], resnorm[ncols], hist or None)."""
    iters = np.zeros(ncols, dtype=np.int32)
    res = np.zeros(ncols)
    hist = np.zeros((ncols, max_iters)) if want_hist else None
    rc = load().sylv_bicgstab(op, _shift(sigma), int(jacobi), int(is_complex), _ptr(B), _ptr(X),
                              int(ncols), float(tol), int(max_iters), PRECISIONS.get(precision, precision),
                              iters.ctypes.data_as(C.POINTER(C.c_int32)),
                              res.ctypes.data_as(C.POINTER(C.c_double)),
                              hist.ctypes.data_as(C.POINTER(C.c_double)) if want_hist else None,
                              _stream(stream))
    _check(rc, allow_warn=True)
    return rc, iters, res, hist


def sylv_arnoldi(op, sigma, jacobi, is_complex, v0, k, V_out, precision="fp64", ortho="cgs2", stream=None):
    """One Arnoldi cycle of k steps; V_out (device, n x (k+1)) receives the
    basis; returns the (k+1) x k Hessenberg matrix as formed."""
    H = np.zeros((k, k + 1), dtype=np.complex128 if is_complex else np.float64)   # column-major (k+1) x k
    _check(load().sylv_arnoldi(op, _shift(sigma), int(jacobi), int(is_complex), _ptr(v0), int(k),
                               PRECISIONS.get(precision, precision), ORTHO.get(ortho, ortho), _ptr(V_out),
                               H.ctypes.data, _stream(stream)))
    return H.T.copy()


def sylv_controller_eval(opts: SylvOpts, inputs: np.ndarray) -> np.ndarray:
    inp = np.ascontiguousarray(inputs, dtype=np.float64).reshape(-1, 11)
    out = np.zeros((inp.shape[0], 3))
    _check(load().sylv_controller_eval(C.byref(opts), inp.shape[0],
                                       inp.ctypes.data_as(C.POINTER(C.c_double)),
                                       out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def sylv_adi_create(A, B, f, g, alpha, beta, tau, opts: SylvOpts | None = None, stream=None,
                    M=None, Cm=None) -> int:
    """Solver handle for A X + X B = -f g^*, or with mass matrices M, Cm for the
    generalized A X Cm + M X B = -f g^* (sylv_adi_create_g)."""
    ha, hb = _csr(A), _csr(B)
    hm = _csr(M) if M is not None else None
    hc = _csr(Cm) if Cm is not None else None
    f = np.asfortranarray(f, dtype=np.float64)
    g = np.asfortranarray(g, dtype=np.float64)
    r = f.shape[1]
    if g.shape[1] != r:
        raise ValueError("f and g need the same number of columns")
    al = (SylvShift * len(alpha))(*[_shift(a) for a in alpha])
    be = (SylvShift * len(beta))(*[_shift(b) for b in beta])
    if len(alpha) != len(beta):
        raise ValueError("alpha and beta need the same length")
    out = C.c_void_p()
    if hm is None and hc is None:
        _check(load().sylv_adi_create(C.byref(ha.s), C.byref(hb.s),
                                      f.ctypes.data_as(C.POINTER(C.c_double)),
                                      g.ctypes.data_as(C.POINTER(C.c_double)), r, al, be, len(alpha),
                                      float(tau), C.byref(opts) if opts is not None else None,
                                      _stream(stream), C.byref(out)))
    else:
        _check(load().sylv_adi_create_g(C.byref(ha.s), C.byref(hb.s),
                                        C.byref(hm.s) if hm is not None else None,
                                        C.byref(hc.s) if hc is not None else None,
                                        f.ctypes.data_as(C.POINTER(C.c_double)),
                                        g.ctypes.data_as(C.POINTER(C.c_double)), r, al, be, len(alpha),
                                        float(tau), C.byref(opts) if opts is not None else None,
                                        _stream(stream), C.byref(out)))
    return out.value


def sylv_adi_set_rhs(h, f, g) -> None:
    f = np.asfortranarray(f, dtype=np.float64)
    g = np.asfortranarray(g, dtype=np.float64)
    _check(load().sylv_adi_set_rhs(h, f.ctypes.data_as(C.POINTER(C.c_double)),
                                   g.ctypes.data_as(C.POINTER(C.c_double))))


def sylv_adi_set_rhs_device(h, f, g) -> None:
    _check(load().sylv_adi_set_rhs_device(h, _ptr(f), _ptr(g)))


def sylv_adi_solve(h) -> int:
    """Runs Algorithm 1; returns the status (0, or MAXIT/INNER_STALL warnings)."""
    return _check(load().sylv_adi_solve(h), allow_warn=True)


def sylv_adi_info(h) -> dict:
    info = SylvInfo()
    _check(load().sylv_adi_info(h, C.byref(info)))
    return info.as_dict()


def sylv_adi_history(h, cap: int = 1000) -> np.ndarray:
    buf = np.zeros((cap, len(HIST_COLUMNS)))
    rows = C.c_int32()
    _check(load().sylv_adi_history(h, buf.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(rows)))
    return buf[: rows.value]


def sylv_adi_core(h) -> np.ndarray:
    """The real kr x kr core G of X = Z G Y^T (real factors only)."""
    kr = C.c_int32()
    _check(load().sylv_adi_core(h, None, 0, C.byref(kr)))
    G = np.zeros((kr.value, kr.value))                    # column-major == transposed row-major
    _check(load().sylv_adi_core(h, G.ctypes.data_as(C.POINTER(C.c_double)), max(1, kr.value), C.byref(kr)))
    return G.T.copy()


def sylv_adi_factors(h, n: int, m: int, real_pairs: bool = False):
    """(Z, Y, gamma) as numpy arrays (host copies).  With real double steps
    (real_pairs) the third item is the dense real core G (X = Z G Y^T)."""
    info = sylv_adi_info(h)
    kr, cplx = info["kr"], info["is_complex"]
    if real_pairs:
        Z = np.zeros((kr, n))
        Y = np.zeros((kr, m))
        kro, isc = C.c_int32(), C.c_int32()
        _check(load().sylv_adi_factors(h, Z.ctypes.data, Y.ctypes.data, None, 0, C.byref(kro), C.byref(isc)))
        return Z.T, Y.T, sylv_adi_core(h)
    dt = np.complex128 if cplx else np.float64
    Z = np.zeros((kr, n), dtype=dt)        # column-major n x kr == row-major kr x n
    Y = np.zeros((kr, m), dtype=dt)
    gam = np.zeros(kr, dtype=dt)
    kro, isc = C.c_int32(), C.c_int32()
    _check(load().sylv_adi_factors(h, Z.ctypes.data, Y.ctypes.data, gam.ctypes.data, 0,
                                   C.byref(kro), C.byref(isc)))
    return Z.T, Y.T, gam


def sylv_adi_destroy(h) -> None:
    _check(load().sylv_adi_destroy(h))


def sylv_adi_profile(h, enable: bool) -> None:
    _check(load().sylv_adi_profile(h, int(enable)))


def sylv_adi_kernel_stats(h) -> dict:
    """{kernel: (ms, algorithmic bytes, algorithmic flops, launches)} since the last reset."""
    ms = np.zeros(len(KERNELS))
    by = np.zeros(len(KERNELS))
    fl = np.zeros(len(KERNELS))
    la = np.zeros(len(KERNELS), dtype=np.int64)
    _check(load().sylv_adi_kernel_stats(h, ms.ctypes.data_as(C.POINTER(C.c_double)),
                                        by.ctypes.data_as(C.POINTER(C.c_double)),
                                        fl.ctypes.data_as(C.POINTER(C.c_double)),
                                        la.ctypes.data_as(C.POINTER(C.c_int64))))
    return {k: (float(ms[i]), float(by[i]), float(fl[i]), int(la[i])) for i, k in enumerate(KERNELS)}


class SylvesterADI:
    """A X + X B = -f g^* solved on the GPU by the inexact LR-ADI iteration."""

    def __init__(self, A, B, f, g, alpha, beta, tau=1e-8, stream=None, M=None, Cm=None, **opts):
        """M, Cm: mass matrices of the generalized equation A X Cm + M X B = -f g^*."""
        self.n = A.n if hasattr(A, "n") else A.shape[0]
        self.m = B.n if hasattr(B, "n") else B.shape[0]
        self.r = f.shape[1]
        self.opts = sylv_opts_default(**opts)
        self.h = sylv_adi_create(A, B, f, g, alpha, beta, tau, self.opts, stream, M=M, Cm=Cm)

    def solve(self) -> int:
        return sylv_adi_solve(self.h)

    def set_rhs(self, f, g) -> None:
        sylv_adi_set_rhs(self.h, f, g)

    def info(self) -> dict:
        return sylv_adi_info(self.h)

    def history(self) -> np.ndarray:
        return sylv_adi_history(self.h)

    def factors(self):
        """(Z, Y, gamma); with real double steps (real_pairs=1) (Z, Y, G) with
        the dense real core G, X = Z G Y^T."""
        return sylv_adi_factors(self.h, self.n, self.m, bool(self.opts.real_pairs))

    def profile(self, enable: bool = True) -> None:
        sylv_adi_profile(self.h, enable)

    def kernel_stats(self) -> dict:
        return sylv_adi_kernel_stats(self.h)

    def tuning(self) -> dict:
        return sylv_adi_tuning(self.h)

    def close(self) -> None:
        if self.h:
            sylv_adi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- batched solves ----

def sylv_adi_batch_create(problems, opts: SylvOpts | None = None, stream=None):
    """problems: sequence of (A, B, f, g, alpha, beta, tau).  Returns (handle,
    keep) where keep holds the host arrays alive for the call."""
    keep = []
    arr = (SylvProblem * len(problems))()
    for i, (A, B, f, g, alpha, beta, tau) in enumerate(problems):
        ha, hb = _csr(A), _csr(B)
        f = np.asfortranarray(f, dtype=np.float64)
        g = np.asfortranarray(g, dtype=np.float64)
        if f.shape[1] != g.shape[1] or len(alpha) != len(beta):
            raise ValueError(f"instance {i}: f/g columns or shift counts differ")
        al = (SylvShift * len(alpha))(*[_shift(a) for a in alpha])
        be = (SylvShift * len(beta))(*[_shift(b) for b in beta])
        keep += [ha, hb, f, g, al, be]
        arr[i] = SylvProblem(C.pointer(ha.s), C.pointer(hb.s), f.ctypes.data, g.ctypes.data, f.shape[1],
                             C.addressof(al), C.addressof(be), len(alpha), float(tau))
    out = C.c_void_p()
    _check(load().sylv_adi_batch_create(len(problems), arr, C.byref(opts) if opts is not None else None,
                                        _stream(stream), C.byref(out)))
    return out.value


def sylv_adi_batch_solve(b) -> int:
    """Solves every instance; returns the batch status (0, or MAXIT/INNER_STALL warnings)."""
    return _check(load().sylv_adi_batch_solve(b), allow_warn=True)


def sylv_adi_batch_info(b, i: int) -> dict:
    info = SylvInfo()
    _check(load().sylv_adi_batch_info(b, int(i), C.byref(info)))
    return info.as_dict()


def sylv_adi_batch_history(b, i: int, cap: int = 1000) -> np.ndarray:
    buf = np.zeros((cap, len(HIST_COLUMNS)))
    rows = C.c_int32()
    _check(load().sylv_adi_batch_history(b, int(i), buf.ctypes.data_as(C.POINTER(C.c_double)), cap,
                                         C.byref(rows)))
    return buf[: rows.value]


def sylv_adi_batch_factors(b, i: int, n: int, m: int):
    info = sylv_adi_batch_info(b, i)
    kr, cplx = info["kr"], info["is_complex"]
    dt = np.complex128 if cplx else np.float64
    Z = np.zeros((kr, n), dtype=dt)
    Y = np.zeros((kr, m), dtype=dt)
    gam = np.zeros(kr, dtype=dt)
    kro, isc = C.c_int32(), C.c_int32()
    _check(load().sylv_adi_batch_factors(b, int(i), Z.ctypes.data, Y.ctypes.data, gam.ctypes.data, 0,
                                         C.byref(kro), C.byref(isc)))
    return Z.T, Y.T, gam


def sylv_adi_batch_stats(b) -> dict:
    la, ti = C.c_int64(), C.c_int64()
    by, fl = C.c_double(), C.c_double()
    _check(load().sylv_adi_batch_stats(b, C.byref(la), C.byref(by), C.byref(fl), C.byref(ti)))
    return {"launches": la.value, "bytes": by.value, "flops": fl.value, "ticks": ti.value}


def sylv_adi_batch_destroy(b) -> None:
    _check(load().sylv_adi_batch_destroy(b))


def _tuning(fn, h) -> dict:
    chosen, count = C.c_int32(), C.c_int32()
    cand = np.zeros(16, dtype=np.int32)
    ms = np.zeros(16)
    _check(fn(h, C.byref(chosen), cand.ctypes.data_as(C.POINTER(C.c_int32)),
              ms.ctypes.data_as(C.POINTER(C.c_double)), 16, C.byref(count)))
    k = min(count.value, 16)
    return {"rows_per_chunk": chosen.value,
            "candidates": {int(c): float(m) for c, m in zip(cand[:k], ms[:k])}}


def sylv_adi_tuning(h) -> dict:
    """Chunk size in use and the autotuner's candidates (ms per device iteration)."""
    return _tuning(load().sylv_adi_tuning, h)


def sylv_adi_batch_tuning(b) -> dict:
    return _tuning(load().sylv_adi_batch_tuning, b)


def sylv_adi_batch_set_rhs(b, i: int, f, g) -> None:
    f = np.asfortranarray(f, dtype=np.float64)
    g = np.asfortranarray(g, dtype=np.float64)
    _check(load().sylv_adi_batch_set_rhs(b, int(i), f.ctypes.data_as(C.POINTER(C.c_double)),
                                         g.ctypes.data_as(C.POINTER(C.c_double))))


def sylv_adi_batch_profile(b, enable: bool) -> None:
    _check(load().sylv_adi_batch_profile(b, int(enable)))


def sylv_adi_batch_kernel_stats(b) -> dict:
    """{kernel: (ms, algorithmic bytes, algorithmic flops, launches)} of the batch since the last reset."""
    ms = np.zeros(len(KERNELS))
    by = np.zeros(len(KERNELS))
    fl = np.zeros(len(KERNELS))
    la = np.zeros(len(KERNELS), dtype=np.int64)
    _check(load().sylv_adi_batch_kernel_stats(b, ms.ctypes.data_as(C.POINTER(C.c_double)),
                                              by.ctypes.data_as(C.POINTER(C.c_double)),
                                              fl.ctypes.data_as(C.POINTER(C.c_double)),
                                              la.ctypes.data_as(C.POINTER(C.c_int64))))
    return {k: (float(ms[i]), float(by[i]), float(fl[i]), int(la[i])) for i, k in enumerate(KERNELS)}


class SylvesterADIBatch:
    """Many independent A_i X + X B_i = -f_i g_i^* solved in one device loop.

    problems: objects with fields A, B, f, g, alpha, beta, tau (for example
    workloads.Problem) or tuples in that order."""

    def __init__(self, problems, stream=None, **opts):
        tup = [p if isinstance(p, tuple) else (p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau) for p in problems]
        self.sizes = [(t[0].n if hasattr(t[0], "n") else t[0].shape[0],
                       t[1].n if hasattr(t[1], "n") else t[1].shape[0]) for t in tup]
        self.opts = sylv_opts_default(**opts)
        self.h = sylv_adi_batch_create(tup, self.opts, stream)

    def __len__(self):
        return len(self.sizes)

    def solve(self) -> int:
        return sylv_adi_batch_solve(self.h)

    def info(self, i: int) -> dict:
        return sylv_adi_batch_info(self.h, i)

    def history(self, i: int) -> np.ndarray:
        return sylv_adi_batch_history(self.h, i)

    def factors(self, i: int):
        n, m = self.sizes[i]
        return sylv_adi_batch_factors(self.h, i, n, m)

    def stats(self) -> dict:
        return sylv_adi_batch_stats(self.h)

    def set_rhs(self, i: int, f, g) -> None:
        sylv_adi_batch_set_rhs(self.h, i, f, g)

    def profile(self, enable: bool = True) -> None:
        sylv_adi_batch_profile(self.h, enable)

    def kernel_stats(self) -> dict:
        return sylv_adi_batch_kernel_stats(self.h)

    def tuning(self) -> dict:
        return sylv_adi_batch_tuning(self.h)

    def close(self) -> None:
        if self.h:
            sylv_adi_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
