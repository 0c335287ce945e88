"""Seeded synthetic inputs for the inexact low-rank Sylvester ADI solver.

This module holds the input recipe only: the finite-difference
convection-diffusion operators of the paper's experiments (Sec. 4,
eq. (ex:convdiff)), the Gaussian right-hand-side factors f, g rescaled to
equal norm (Sec. 4), and the ADI shift pairs, which the paper treats as
given inputs computed offline (Sec. 2.1, after eq. (adi_shift); Sec. 4 uses
the heuristic of Benner, Li and Truhar with Ritz and inverse Ritz values).
None of the LR-ADI arithmetic (Algorithm 1, the inner solves, the tolerance
controller) lives here; both the CPU oracle and the CUDA path consume the
arrays this module produces.

Conventions
-----------
* Grid: N interior points per dimension on (0,1)^d, Dirichlet zero boundary,
  h = 1/(N+1), node coordinates x_i = i*h (i = 1..N), lexicographic ordering
  with x fastest.
* L(u) = -Laplace(u) + omega . grad(u): centred differences, diagonal 2d/h^2,
  neighbours -1/h^2 -/+ omega_c(node)/(2h) on the -/+ neighbour in direction c.
* The returned coefficient matrix is A = -L, so its spectrum lies in the open
  left half plane (the paper assumes Lambda(A), Lambda(B) in C_-).
* CSR arrays: int32 row pointers and column indices (columns ascending within
  a row), float64 values.
* Random numbers: a counter-based splitmix64 generator (Steele, Lea, Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014) feeding the
  Box-Muller transform.  It is written out here so that every machine draws
  the same inputs regardless of the numpy version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CSR", "normal", "convdiff", "rhs_factors", "ritz_values",
    "inverse_ritz_values", "select_shift_pairs", "Problem", "make_problem",
    "problem_config", "batch_problems", "mass_matrix", "make_problem_g",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied elementwise to a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int, column: int) -> np.uint64:
    base = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    tag = np.uint64(((stream & 0xFFFFFFFF) << 32) | (column & 0xFFFFFFFF))
    return _mix64(np.array([base ^ tag], dtype=np.uint64))[0]


def _uniform53(seed: int, stream: int, column: int, start: int, count: int) -> np.ndarray:
    """count doubles in (0,1) from counters start..start+count-1 of one stream."""
    key = _stream_key(seed, stream, column)
    ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = _mix64(key + ctr * _GOLDEN)
    return ((x >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, column: int, count: int) -> np.ndarray:
    """count N(0,1) samples (Box-Muller on pairs of counter-based uniforms)."""
    u = _uniform53(seed, stream, column, 0, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# Operators
# ----------------------------------------------------------------------------

@dataclass
class CSR:
    """A square sparse matrix in CSR form (int32 indices, float64 values)."""
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))


def _field(kind: str, mag: float, coords):
    """Convection field omega(node) for the families the experiments use."""
    z0 = np.zeros_like(coords[0])
    if kind == "xy":          # mag * (x, y)
        return [mag * coords[0], mag * coords[1]]
    if kind == "rot2":        # mag * (y, -x)
        return [mag * coords[1], -mag * coords[0]]
    if kind == "zero":
        return [z0 for _ in coords]
    if kind == "const3":      # mag * (1, 1, 1)
        return [z0 + mag, z0 + mag, z0 + mag]
    if kind == "zxy":         # mag * (z, x, y)
        return [mag * coords[2], mag * coords[0], mag * coords[1]]
    if kind == "xyz":         # mag * (x, y, z)
        return [mag * coords[0], mag * coords[1], mag * coords[2]]
    if kind == "rot3":        # mag * (y, -x, 0)
        return [mag * coords[1], -mag * coords[0], z0]
    raise ValueError(f"unknown convection field {kind!r}")


def convdiff(N: int, dim: int, kind: str, mag: float) -> CSR:
    """A = -(FD discretisation of -Laplace(u) + omega.grad(u)), N points per dim."""
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    h = 1.0 / (N + 1)
    n = N ** dim
    idx = np.arange(n, dtype=np.int64)
    sub = [(idx // (N ** c)) % N for c in range(dim)]        # x fastest
    coords = [(s + 1).astype(np.float64) * h for s in sub]
    om = _field(kind, mag, coords)
    inv_h2 = 1.0 / (h * h)
    rows, cols, vals = [], [], []
    # neighbours in ascending column order: -z, -y, -x, centre, +x, +y, +z
    for c in reversed(range(dim)):
        stride = N ** c
        mask = sub[c] > 0
        rows.append(idx[mask]); cols.append(idx[mask] - stride)
        vals.append(-(-inv_h2 - om[c][mask] / (2 * h)))
    rows.append(idx); cols.append(idx); vals.append(np.full(n, -2.0 * dim * inv_h2))
    for c in range(dim):
        stride = N ** c
        mask = sub[c] < N - 1
        rows.append(idx[mask]); cols.append(idx[mask] + stride)
        vals.append(-(-inv_h2 + om[c][mask] / (2 * h)))
    r = np.concatenate(rows); cidx = np.concatenate(cols); v = np.concatenate(vals)
    order = np.lexsort((cidx, r))
    r, cidx, v = r[order], cidx[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr.astype(np.int32), cidx.astype(np.int32), v.astype(np.float64))


def _csr_from_scipy(S) -> CSR:
    S = S.tocsr()
    S.sort_indices()
    return CSR(S.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def mass_matrix(N: int, dim: int) -> CSR:
    """Consistent mass matrix of Q1 (bilinear / trilinear) finite elements on
    the uniform grid of convdiff (N interior nodes per dimension, Dirichlet
    boundary, same node ordering): the Kronecker product of the 1D P1 mass
    matrices (h/6) tridiag(1, 4, 1); symmetric positive definite, 9 (2D) or
    27 (3D) nonzeros per interior row."""
    import scipy.sparse as sp
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    h = 1.0 / (N + 1)
    M1 = sp.diags([np.full(N - 1, h / 6), np.full(N, 4 * h / 6), np.full(N - 1, h / 6)], [-1, 0, 1])
    M = M1
    for _ in range(dim - 1):
        M = sp.kron(M1, M)          # x fastest: the first factor is the slowest index
    return _csr_from_scipy(M)


def rhs_factors(n: int, m: int, r: int, seed: int):
    """f (n x r), g (m x r): N(0,1) columns, each factor rescaled to unit 2-norm.

    The paper draws f, g from a normal distribution and rescales them so that
    ||f|| = ||g|| (Sec. 4); here both are scaled to spectral norm 1.
    """
    f = np.stack([normal(seed, 1, l, n) for l in range(r)], axis=1)
    g = np.stack([normal(seed, 2, l, m) for l in range(r)], axis=1)
    f /= np.linalg.norm(f, 2)
    g /= np.linalg.norm(g, 2)
    return np.asfortranarray(f), np.asfortranarray(g)


# ----------------------------------------------------------------------------
# Shifts (offline input, Sec. 2.1 and Sec. 4)
# ----------------------------------------------------------------------------

def _arnoldi_ritz(matvec, n: int, steps: int) -> np.ndarray:
    """Ritz values of a steps-step Arnoldi process (MGS) from 1/sqrt(n)."""
    V = np.zeros((n, steps + 1))
    H = np.zeros((steps + 1, steps))
    V[:, 0] = 1.0 / math.sqrt(n)
    k = steps
    for j in range(steps):
        w = matvec(V[:, j])
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] < 1e-12 * abs(H[j, j]) + 1e-300:
            k = j + 1
            break
        V[:, j + 1] = w / H[j + 1, j]
    return np.linalg.eigvals(H[:k, :k])


def ritz_values(op: CSR, steps: int = 20) -> np.ndarray:
    S = op.to_scipy()
    return _arnoldi_ritz(lambda x: S @ x, op.n, steps)


def inverse_ritz_values(op: CSR, steps: int = 20) -> np.ndarray:
    """Reciprocals of the Ritz values of op^{-1} (sparse LU applied)."""
    import scipy.sparse.linalg as spla
    lu = spla.splu(op.to_scipy().tocsc())
    mu = _arnoldi_ritz(lu.solve, op.n, steps)
    mu = mu[np.abs(mu) > 0]
    return 1.0 / mu


def generalized_ritz_values(op: CSR, mass: CSR, steps: int = 20) -> np.ndarray:
    """Ritz and inverse Ritz values of the pencil (op, mass), i.e. of
    mass^{-1} op and of op^{-1} mass (sparse LU applied): the spectrum
    Lambda(A, M) that replaces Lambda(A) in the shift problem of the
    generalized equation (Sec. 2, after eq. (lradi_g))."""
    import scipy.sparse.linalg as spla
    S, Mm = op.to_scipy(), mass.to_scipy()
    lum = spla.splu(Mm.tocsc())
    lus = spla.splu(S.tocsc())
    ritz = _arnoldi_ritz(lambda x: lum.solve(S @ x), op.n, steps)
    mu = _arnoldi_ritz(lambda x: lus.solve(Mm @ x), op.n, steps)
    mu = mu[np.abs(mu) > 0]
    return np.concatenate([ritz, 1.0 / mu])


def select_shift_pairs(cand_a: np.ndarray, cand_b: np.ndarray, count: int,
                       real: bool = True):
    """Greedy min-max selection of (alpha_i, beta_i) for eq. (adi_shift).

    alpha approximates Lambda(A) and beta approximates Lambda(B): the factor
    |(lambda-alpha)/(lambda+beta)| vanishes at lambda = alpha.  The first pair
    minimises max |phi_A| * max |phi_B| over the candidate sets; every further
    pair places alpha (beta) where the current rational function of the A
    (B) side is largest on the candidates.  With real=True the real parts of
    the candidates are used and the pairs are real.  With real=False a complex
    alpha or beta is followed immediately by the pair of conjugates, so that
    the conjugate-paired sequence yields a real solution after each pair.
    """
    ca = np.asarray(cand_a, dtype=np.complex128)
    cb = np.asarray(cand_b, dtype=np.complex128)
    if real:
        ca = np.unique(np.round(ca.real, 12)).astype(np.complex128)
        cb = np.unique(np.round(cb.real, 12)).astype(np.complex128)
    else:
        ca = ca[np.imag(ca) >= 0]
        cb = cb[np.imag(cb) >= 0]
    ca = ca[np.real(ca) < 0]
    cb = cb[np.real(cb) < 0]
    if ca.size == 0 or cb.size == 0:
        raise ValueError("shift candidates must lie in the open left half plane")

    def phiA(lam, al, be):
        out = np.ones(lam.shape)
        for a, b in zip(al, be):
            out = out * np.abs((lam - a) / (lam + b))
        return out

    def phiB(mu, al, be):
        out = np.ones(mu.shape)
        for a, b in zip(al, be):
            out = out * np.abs((mu - b) / (mu + a))
        return out

    # first pair: for each alpha, all betas at once (the same elementwise
    # operations as phiA / phiB for one pair, so the values and the first
    # minimum in (alpha, beta) order are those of the plain double loop)
    best = None
    for a in ca:
        ma = np.abs((ca[None, :] - a) / (ca[None, :] + cb[:, None])).max(axis=1)
        mb = np.abs((cb[None, :] - cb[:, None]) / (cb[None, :] + a)).max(axis=1)
        val = ma * mb
        j = int(np.argmin(val))
        if best is None or val[j] < best[0]:
            best = (val[j], a, cb[j])
    al, be = [best[1]], [best[2]]

    def add(a, b):
        al.append(a); be.append(b)
        if not real and (abs(a.imag) > 0 or abs(b.imag) > 0):
            al.append(np.conj(a)); be.append(np.conj(b))

    if not real and (abs(al[0].imag) > 0 or abs(be[0].imag) > 0):
        al.append(np.conj(al[0])); be.append(np.conj(be[0]))
    while len(al) < count:
        a = ca[int(np.argmax(phiA(ca, al, be)))]
        b = cb[int(np.argmax(phiB(cb, al, be)))]
        add(a, b)
    if not real:
        # never cut a conjugate pair in half: drop a dangling first member
        keep, i = 0, 0
        while i < min(count, len(al)):
            if abs(al[i].imag) > 0 or abs(be[i].imag) > 0:
                if i + 1 >= count:
                    break
                i += 2
            else:
                i += 1
            keep = i
        count = keep
    al, be = np.array(al[:count]), np.array(be[:count])
    if real:
        return al.real.copy(), be.real.copy()
    return al, be


def shift_bound(alpha, beta, lam_a, lam_b) -> float:
    """max over lam_a of |prod (lam - alpha_i)/(lam + beta_i)| times the B-side
    maximum: the a-priori contraction of one pass over the shift pairs
    (eq. (adi_shift)) on the sample points."""
    pa = np.ones(np.shape(lam_a))
    pb = np.ones(np.shape(lam_b))
    for a, b in zip(alpha, beta):
        pa = pa * np.abs((lam_a - a) / (lam_a + b))
        pb = pb * np.abs((lam_b - b) / (lam_b + a))
    return float(pa.max() * pb.max())


def select_real_shifts_sampled(cand_a, cand_b, count: int, grids=(0, 12, 25, 50, 100, 200, 400)):
    """Real shift pairs for operators whose candidate sets leave wide gaps
    (Ritz values cluster at both ends of a spectrum spanning many decades).

    For every k in grids the greedy selection runs on the candidates plus k
    log-spaced points between the smallest and the largest |Re| of the
    candidates; the selection with the smallest shift_bound on the
    candidates plus a 400-point log grid is returned."""
    def loggrid(c, k):
        re = np.abs(np.real(np.asarray(c)))
        re = re[re > 0]
        return -np.logspace(np.log10(re.min()), np.log10(re.max()), k)
    sample_a = np.concatenate([np.real(cand_a), loggrid(cand_a, 400)])
    sample_b = np.concatenate([np.real(cand_b), loggrid(cand_b, 400)])
    best = None
    for k in grids:
        xa = cand_a if k == 0 else np.concatenate([cand_a, loggrid(cand_a, k)])
        xb = cand_b if k == 0 else np.concatenate([cand_b, loggrid(cand_b, k)])
        al, be = select_shift_pairs(xa, xb, count, real=True)
        bd = shift_bound(al, be, sample_a, sample_b)
        if best is None or bd < best[0]:
            best = (bd, al, be)
    return best[1], best[2]


# ----------------------------------------------------------------------------
# Problems
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """One Sylvester instance A X + X B = -f g^* (or, with M and C, the
    generalized A X C + M X B = -f g^* of eq. (gsylv)) with shifts and options."""
    name: str
    A: CSR
    B: CSR
    f: np.ndarray
    g: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    tau: float = 1e-8
    opts: dict = field(default_factory=dict)
    M: CSR | None = None
    C: CSR | None = None

    @property
    def r(self) -> int:
        return self.f.shape[1]


INVERSE_RITZ_MAX_N = 600_000     # above this the LU of the operator is too costly


def _inverse_ritz(op: CSR, N: int, dim: int, kind: str, mag: float, steps: int) -> np.ndarray:
    """Inverse Ritz values of the operator, or - when it is too large for a
    sparse LU - of the same convection-diffusion family discretised on a
    coarser grid (the small eigenvalues of the differential operator, which
    these approximate, change little with the grid)."""
    if op.n <= INVERSE_RITZ_MAX_N:
        return inverse_ritz_values(op, steps)
    Nc = int(round(INVERSE_RITZ_MAX_N ** (1.0 / dim) / 2))
    return inverse_ritz_values(convdiff(Nc, dim, kind, mag), steps)


def make_problem(name, NA, dimA, kindA, magA, NB, dimB, kindB, magB, r, seed,
                 n_shifts, real_shifts=True, tau=1e-8, ritz_steps=20, sampled_shifts=False,
                 **opts) -> Problem:
    A = convdiff(NA, dimA, kindA, magA)
    B = convdiff(NB, dimB, kindB, magB)
    f, g = rhs_factors(A.n, B.n, r, seed)
    cand_a = np.concatenate([ritz_values(A, ritz_steps),
                             _inverse_ritz(A, NA, dimA, kindA, magA, ritz_steps)])
    cand_b = np.concatenate([ritz_values(B, ritz_steps),
                             _inverse_ritz(B, NB, dimB, kindB, magB, ritz_steps)])
    if sampled_shifts and real_shifts:
        alpha, beta = select_real_shifts_sampled(cand_a, cand_b, n_shifts)
    else:
        alpha, beta = select_shift_pairs(cand_a, cand_b, n_shifts, real=real_shifts)
    return Problem(name, A, B, f, g, alpha, beta, tau, dict(opts))


def make_problem_g(name, NA, dimA, kindA, magA, NB, dimB, kindB, magB, r, seed, n_shifts,
                   tau=1e-8, ritz_steps=20, **opts) -> Problem:
    """A generalized instance A X C + M X B = -f g^* shaped like a finite
    element discretisation (the paper's Ex. 4 is a finite element model whose
    data is not available): M, C consistent Q1 mass matrices, A = h^d A_fd and
    B = h^d B_fd the convection-diffusion operators of convdiff scaled like
    stiffness matrices, so that Lambda(A, M), Lambda(B, C) lie close to
    Lambda(A_fd), Lambda(B_fd).  Real shift pairs from the Ritz and inverse
    Ritz values of the pencils."""
    hA = (1.0 / (NA + 1)) ** dimA
    hB = (1.0 / (NB + 1)) ** dimB
    Afd = convdiff(NA, dimA, kindA, magA)
    Bfd = convdiff(NB, dimB, kindB, magB)
    A = CSR(Afd.n, Afd.rowptr, Afd.colind, Afd.val * hA)
    B = CSR(Bfd.n, Bfd.rowptr, Bfd.colind, Bfd.val * hB)
    M = mass_matrix(NA, dimA)
    C = mass_matrix(NB, dimB)
    f, g = rhs_factors(A.n, B.n, r, seed)
    cand_a = generalized_ritz_values(A, M, ritz_steps)
    cand_b = generalized_ritz_values(B, C, ritz_steps)
    alpha, beta = select_shift_pairs(cand_a, cand_b, n_shifts, real=True)
    return Problem(name, A, B, f, g, alpha, beta, tau, dict(opts), M, C)


def problem_config(which: str) -> Problem:
    """Named workloads shaped like the paper's experiments.

    * "small2d": A 2D N=32, omega=10(x,y); B 2D N=30, omega=5(y,-x); r=1,
      seed 0, 12 real shift pairs, GMRES(30) without preconditioner.
    * "mid2d": A 2D N=512, omega=50(x,y); B 2D N=400, omega=20(y,-x); r=2,
      seed 1, 12 real shift pairs, right-Jacobi GMRES(30).
    * "tiny2d": A 2D N=12, omega=10(x,y); B 2D N=10, omega=5(y,-x); r=2,
      seed 7 (unit-test size).
    * "mid3d": A 3D N=128 (n = 2097152), omega=100(1,1,1); B 3D N=100
      (m = 1000000), omega=50(z,x,y); r=4, seed 2, 16 shift pairs kept complex
      (conjugate pairs adjacent), right-Jacobi GMRES(30).
    * "large3d": A 3D N=256 (n = 16777216), omega=200(x,y,z); B 3D N=192
      (m = 7077888), omega=100(y,-x,0); r=1, seed 3, 20 complex shift pairs,
      right-Jacobi GMRES(20).
    * "small3d": A 3D N=24, omega=100(1,1,1); B 3D N=20, omega=50(z,x,y);
      r=4, seed 4, 8 complex shift pairs (test size of the 3D family).
    * "tiny2d_g", "small2d_g": the generalized equation (make_problem_g) on
      the grids and fields of "tiny2d" / "small2d" (seeds 8, 5), 8 / 12 real
      shift pairs of the pencils.
    """
    if which == "tiny2d_g":
        return make_problem_g("tiny2d_g", 12, 2, "xy", 10.0, 10, 2, "rot2", 5.0, 2, 8, 8,
                              restart=30, jacobi=False)
    if which == "small2d_g":
        return make_problem_g("small2d_g", 32, 2, "xy", 10.0, 30, 2, "rot2", 5.0, 1, 5, 12,
                              restart=30, jacobi=True)
    if which == "mid3d":
        return make_problem("mid3d", 128, 3, "const3", 100.0, 100, 3, "zxy", 50.0, 4, 2, 16,
                            real_shifts=False, restart=30, jacobi=True)
    if which == "large3d":
        return make_problem("large3d", 256, 3, "xyz", 200.0, 192, 3, "rot3", 100.0, 1, 3, 20,
                            real_shifts=False, restart=20, jacobi=True)
    if which == "small3d":
        return make_problem("small3d", 24, 3, "const3", 100.0, 20, 3, "zxy", 50.0, 4, 4, 8,
                            real_shifts=False, restart=30, jacobi=True)
    if which == "small2d":
        return make_problem("small2d", 32, 2, "xy", 10.0, 30, 2, "rot2", 5.0, 1, 0, 12,
                            restart=30, jacobi=False)
    if which == "mid2d":
        return make_problem("mid2d", 512, 2, "xy", 50.0, 400, 2, "rot2", 20.0, 2, 1, 12,
                            restart=30, jacobi=True)
    if which == "tiny2d":
        return make_problem("tiny2d", 12, 2, "xy", 10.0, 10, 2, "rot2", 5.0, 2, 7, 8,
                            restart=30, jacobi=False)
    raise ValueError(f"unknown workload {which!r}")


def _batch_instance(i: int, base_seed: int, n_shifts: int, nmin: int, nmax: int) -> Problem:
    span = nmax - nmin + 1
    s = base_seed + i
    u = _uniform53(s, 9, 0, 0, 5)
    NA = nmin + int(u[0] * span)
    NB = nmin + int(u[1] * span)
    r = (1, 2, 4)[int(u[2] * 3)]
    magA, magB = 50.0 * u[3], 50.0 * u[4]
    return make_problem(f"batch{i}", NA, 2, "xy", magA, NB, 2, "rot2", magB, r, s,
                        n_shifts, sampled_shifts=True, restart=30, jacobi=True)


def batch_problems(count: int, base_seed: int = 1000, n_shifts: int = 10, nmin: int = 64, nmax: int = 256,
                   workers: int = 1):
    """Independent 2D instances with N_A, N_B ~ U{nmin..nmax} (64..256 for the
    batched workload), r in {1,2,4}, convection magnitudes ~ U[0,50]
    (directions (x,y) for A, (y,-x) for B); instance i uses seed base_seed + i.
    Shifts: select_real_shifts_sampled (with the plain greedy selection six
    of the 64 instances do not reach tau in 50 steps even with exact inner
    solves).  workers > 1 generates the instances in that many spawned
    processes (the same instances: each depends only on its seed)."""
    args = [(i, base_seed, n_shifts, nmin, nmax) for i in range(count)]
    if workers <= 1 or count <= 1:
        return [_batch_instance(*a) for a in args]
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    # one BLAS thread per process (the processes already fill the cores)
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with ProcessPoolExecutor(max_workers=min(workers, count), mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_batch_instance, *zip(*args)))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
