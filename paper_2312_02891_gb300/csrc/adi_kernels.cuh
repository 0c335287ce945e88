// adi_kernels.cuh - outer-iteration kernels of the inexact LR-ADI
// (Algorithm 1, M = I, C = I): the inner-tolerance controller, the per-step
// initialisation of the 2r column solves, and the fused factor update +
// Gram kernel that evaluates the residual norm and the outer stop test.
#pragma once
#include "bicg_kernels.cuh"

namespace sylv {

#define SYLV_MAXR 4
#define SYLV_GSTRIDE (3 * SYLV_MAXR * SYLV_MAXR)   // three r x r Grams per chunk
#define SYLV_HIST_COLS 14

enum Strategy : int { STRAT_FIXED = 0, STRAT_NOBL_MID, STRAT_BL_MID, STRAT_NOBL_A, STRAT_BL_A,
                      STRAT_NOBL_B, STRAT_BL_B };

// Inner tolerances for outer step k (Sec. 3.3).  c = 2 + sqrt(2) bounds the
// constants check-c_k (Crouzeix-Palencia).  Non-back-looking target,
// eq. (ADI_relax1_prak): hat-eps = xi eps / (2 c^2 kmax).  Back-looking,
// eq. (ADI_relax2_prak): hat-eps = |xi k eps / (2 c kmax) - u - v| / c
// (bl_clamp: max(., 0) instead of |.|).  Selection: eq. (simple_tols)
// ("mid"), eq. (one_side) (A preferred) and its mirror (B preferred); every
// value clamped to [delta_min, delta_max] as in eq. (bound_tols).
__host__ __device__ inline void controller_eval(int strategy, int bl_clamp, double k, double kmax,
                                                double eps, double xi, double u, double v,
                                                double Nw, double Nt, double dminA, double dmaxA,
                                                double dminB, double dmaxB, double fixed_tol,
                                                double* dA, double* dB, double* eh) {
    const double c = 2.0 + sqrt(2.0);
    if (strategy == STRAT_FIXED) {
        *dA = fixed_tol; *dB = fixed_tol; *eh = NAN;
        return;
    }
    const bool bl = (strategy == STRAT_BL_MID || strategy == STRAT_BL_A || strategy == STRAT_BL_B);
    double e;
    if (bl) {
        const double x = xi * k * eps / (2.0 * c * kmax) - u - v;
        e = (bl_clamp ? fmax(x, 0.0) : fabs(x)) / c;
    } else {
        e = xi * eps / (2.0 * (c * c) * kmax);
    }
    double a, b;
    if (strategy == STRAT_NOBL_MID || strategy == STRAT_BL_MID) {
        a = fmax(0.5 * (fmin(dmaxA, e / Nt) - dminA), dminA);
        b = fmax(fmin((e - a * Nt) / (2.0 * a + Nw), dmaxB), dminB);
    } else if (strategy == STRAT_NOBL_A || strategy == STRAT_BL_A) {
        a = dminA;
        b = fmax(fmin((e - a * Nt) / (2.0 * a + Nw), dmaxB), dminB);
    } else {
        b = dminB;
        a = fmax(fmin((e - b * Nw) / (2.0 * b + Nt), dmaxA), dminA);
    }
    *dA = a; *dB = b; *eh = e;
}

template <typename T>
struct AdiState {
    int k;                  // current outer step (1-based)
    int done;
    int stage;              // batched solves: where this instance stands (BatchStage)
    int status;             // 0 ok, 1 maxit, 2 nonfinite
    int pair_open;          // inside a conjugate shift pair
    unsigned counter;
    int stalled;            // inner solves that hit their cap
    double nfg;             // ||f g^*||_2
    double eps;             // tau ||f g^*||_2
    double Nw, Nt;          // ||w_{k-1}||, ||t_{k-1}||
    double u, v;            // eq. (upd_resgap)
    double res;             // ||w_{k-1} t_{k-1}^*||_2
    double dA, dB, eh;
    T alpha_k, beta_k, gamma_k;
    long long itsA, itsB, cycles;
    // real double step of a conjugate pair (AdiDev::real_pairs): the step is a
    // pair; the pair's shift on the A side (beta) / B side (alpha) is complex;
    // the second (real-shift) solves are running; inner steps and stalled
    // solves of the pair's first solves
    int pair, cplxA, cplxB, stage2;
    long long pitsA, pitsB;
    int pstalled;
};

template <typename T, typename S, typename C>
struct AdiDev {
    int n, m, r, kmax, nshift, strategy, bl_clamp, max_inner;
    double tau, xi, dminA, dminB, dmaxA, dmaxB, fixed_tol;
    const T* alpha;
    const T* beta;
    const double* f;        // n x r
    const double* g;        // m x r
    T* w;                   // n x r  (w_k)
    T* t;                   // m x r  (t_k)
    T* Z;                   // n x kmax r
    T* Y;                   // m x kmax r
    T* gam;                 // kmax r
    double* hist;           // kmax x SYLV_HIST_COLS
    OpDesc opA, opB;        // A and B^T (float64)
    T* pinvA;               // null: no preconditioner
    T* pinvB;
    C* avalA;               // pre-scaled stencil diagonals for the current shift, or null
    C* avalB;
    const SysDesc<T, S, C>* sd;   // systems 0..r-1: A side, r..2r-1: B side
    SysState<T>* st;
    BatchCtl* ctl;
    T* gpart;               // (nchA + nchB) x SYLV_GSTRIDE
    int nchA, nchB, rpc;
    AdiState<T>* s;
    int* h_done;            // mapped host word
    // real double step of conjugate pairs (Sec. 3.3 "Complex shift parameters"),
    // complex instantiations only: the solves write XA, XB (n x r, m x r,
    // complex); the second solves of a real-shift side write XA2, XB2; the real
    // factors go to Zr, Yr (n x (kmax + 1) r, m x (kmax + 1) r); core holds per
    // step {kind, G00, G01, G10, G11} (kind 1: plain step, G00 = gamma; 2: first
    // step of a pair, G its 2 x 2 real core; 3: second step of a pair); RsA, RsB
    // keep the first residual of a real-shift side (n x r, m x r)
    int real_pairs;
    T* XA;
    T* XB;
    T* XA2;
    T* XB2;
    double* Zr;
    double* Yr;
    double* core;
    double* RsA;
    double* RsB;
    double* pgpart;         // (nchA + nchB) x SYLV_PGSTRIDE Gram partials of the pair update
};

// Largest eigenvalues of small Hermitian matrices (cyclic Jacobi, Golub and
// Van Loan, Matrix Computations, Sec. 8.5, with a phase rotation for the
// complex case).  A, Q: SYLV_MAXR x SYLV_MAXR row-major, top-left r x r used.
template <typename T>
__device__ void herm_jacobi(T* A, T* Q, int r) {
    for (int p = 0; p < SYLV_MAXR; ++p)
        for (int q = 0; q < SYLV_MAXR; ++q) Q[p * SYLV_MAXR + q] = make_scalar<T>(p == q ? 1.0 : 0.0, 0.0);
    for (int sweep = 0; sweep < 20; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int p = 0; p < r; ++p) {
            dg += abs2(A[p * SYLV_MAXR + p]);
            for (int q = p + 1; q < r; ++q) off += abs2(A[p * SYLV_MAXR + q]);
        }
        if (off == 0.0 || off <= 1e-34 * dg) break;
        for (int p = 0; p < r - 1; ++p) {
            for (int q = p + 1; q < r; ++q) {
                const T apq = A[p * SYLV_MAXR + q];
                const double b = absv(apq);
                if (b == 0.0) continue;
                const T e = unit_phase(apq, b);
                const T ec = conjg(e);
                const double app = re(A[p * SYLV_MAXR + p]), aqq = re(A[q * SYLV_MAXR + q]);
                const double theta = (aqq - app) / (2.0 * b);
                const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
                for (int i = 0; i < r; ++i) {       // A <- A W, Q <- Q W
                    const T aip = A[i * SYLV_MAXR + p], aiq = A[i * SYLV_MAXR + q];
                    A[i * SYLV_MAXR + p] = c * aip - s * (ec * aiq);
                    A[i * SYLV_MAXR + q] = s * aip + c * (ec * aiq);
                    const T qip = Q[i * SYLV_MAXR + p], qiq = Q[i * SYLV_MAXR + q];
                    Q[i * SYLV_MAXR + p] = c * qip - s * (ec * qiq);
                    Q[i * SYLV_MAXR + q] = s * qip + c * (ec * qiq);
                }
                for (int i = 0; i < r; ++i) {       // A <- W^* A
                    const T api = A[p * SYLV_MAXR + i], aqi = A[q * SYLV_MAXR + i];
                    A[p * SYLV_MAXR + i] = c * api - s * (e * aqi);
                    A[q * SYLV_MAXR + i] = s * api + c * (e * aqi);
                }
                A[p * SYLV_MAXR + q] = zero<T>();
                A[q * SYLV_MAXR + p] = zero<T>();
            }
        }
    }
}

template <typename T>
__device__ double herm_lmax(const T* G, int r) {
    T A[SYLV_MAXR * SYLV_MAXR], Q[SYLV_MAXR * SYLV_MAXR];
    for (int i = 0; i < SYLV_MAXR * SYLV_MAXR; ++i) A[i] = G[i];
    herm_jacobi(A, Q, r);
    double lm = re(A[0]);
    for (int p = 1; p < r; ++p) lm = fmax(lm, re(A[p * SYLV_MAXR + p]));
    return fmax(lm, 0.0);
}

// ||w t^*||_2 from G_w = w^* w and G_t = t^* t: with G_w = S S^*, S = Q
// Lambda^{1/2}, ||w t^*||^2 = lambda_max(S^* G_t S).
template <typename T>
__device__ double lowrank_norm_from_grams(const T* Gw, const T* Gt, int r) {
    T A[SYLV_MAXR * SYLV_MAXR], Q[SYLV_MAXR * SYLV_MAXR], M[SYLV_MAXR * SYLV_MAXR];
    for (int i = 0; i < SYLV_MAXR * SYLV_MAXR; ++i) A[i] = Gw[i];
    herm_jacobi(A, Q, r);
    double sq[SYLV_MAXR];
    for (int p = 0; p < r; ++p) sq[p] = sqrt(fmax(re(A[p * SYLV_MAXR + p]), 0.0));
    for (int a = 0; a < SYLV_MAXR * SYLV_MAXR; ++a) M[a] = zero<T>();
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            T acc = zero<T>();
            for (int p = 0; p < r; ++p)
                for (int q = 0; q < r; ++q)
                    acc += conjg(Q[p * SYLV_MAXR + a]) * (Gt[p * SYLV_MAXR + q] * Q[q * SYLV_MAXR + b]);
            M[a * SYLV_MAXR + b] = (sq[a] * sq[b]) * acc;
        }
    return sqrt(herm_lmax(M, r));
}

template <typename T>
__device__ __forceinline__ bool is_pair_start(const T* alpha, const T* beta, int idx, int L) {
    const T a = alpha[idx], b = beta[idx];
    if (im(a) == 0.0 && im(b) == 0.0) return false;
    if (idx + 1 >= L) return false;
    const T a1 = alpha[idx + 1], b1 = beta[idx + 1];
    return re(a1) == re(a) && im(a1) == -im(a) && re(b1) == re(b) && im(b1) == -im(b);
}

// Start of outer step k of one instance: tolerances (Sec. 3.3), the shift
// pair and the 2r column systems, left in the restart phase so that their
// first device iteration forms r = b - (Op + sigma I) x with x = 0.
template <typename T, typename S, typename C>
__device__ void adi_begin_step(const AdiDev<T, S, C>& d) {
    AdiState<T>* s = d.s;
    const int r = d.r;
    const int k = s->k;
    const int idx = (k - 1) % d.nshift;
    const T a = d.alpha[idx], b = d.beta[idx];
    double dA, dB, eh;
    controller_eval(d.strategy, d.bl_clamp, (double)k, (double)d.kmax, s->eps, d.xi, s->u, s->v,
                    s->Nw, s->Nt, d.dminA, d.dmaxA, d.dminB, d.dmaxB, d.fixed_tol, &dA, &dB, &eh);
    s->alpha_k = a;
    s->beta_k = b;
    s->gamma_k = -(b + a);
    s->dA = dA; s->dB = dB; s->eh = eh;
    // real double step: one solve per column and side for the pair, to a
    // tolerance divided so that both steps of the pair meet delta / r:
    // 1 + |gamma| / |Im(shift)| for a complex shift (the second solution is
    // derived), 2 for a real shift (two real solves)
    const bool pair = d.real_pairs && is_pair_start(d.alpha, d.beta, idx, d.nshift);
    const double ag = absv(s->gamma_k);
    s->pair = pair ? 1 : 0;
    s->cplxA = im(b) != 0.0;
    s->cplxB = im(a) != 0.0;
    s->stage2 = 0;
    s->pitsA = 0; s->pitsB = 0; s->pstalled = 0;
    const double facA = !pair ? 1.0 : (s->cplxA ? 1.0 + ag / fabs(im(b)) : 2.0);
    const double facB = !pair ? 1.0 : (s->cplxB ? 1.0 + ag / fabs(im(a)) : 2.0);
    for (int q = 0; q < 2 * r; ++q) {
        SysState<T>& st = d.st[q];
        const bool sideA = q < r;
        const int l = sideA ? q : q - r;
        st.phase = PH_RESID;
        st.j = 0; st.iters = 0; st.cycles = 0; st.status = ST_OK; st.nvec = 0; st.counter = 0;
        st.max_iters = d.max_inner;
        st.resnorm = 0.0; st.est = 0.0;
        if (sideA) {
            st.tol = dA / r / facA;
            st.sigma = b;
            st.x = d.real_pairs ? d.XA + (size_t)l * d.n : d.Z + ((size_t)(k - 1) * r + l) * d.n;
            st.b = d.w + (size_t)l * d.n;
        } else {
            st.tol = dB / r / facB;
            st.sigma = conjg(a);
            st.x = d.real_pairs ? d.XB + (size_t)l * d.m : d.Y + ((size_t)(k - 1) * r + l) * d.m;
            st.b = d.t + (size_t)l * d.m;
        }
    }
}

template <typename T, typename S, typename C>
__global__ void k_adi_controller(AdiDev<T, S, C> d) {
    count_launch(d.ctl, K_CTRL);
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    AdiState<T>* s = d.s;
    const int r = d.r;
    // graph-driven solve: no further outer step unless the factor update asks
    if (d.ctl->graph) cudaGraphSetConditional(d.ctl->h_outer, 0u);
    if (s->done) {
        for (int q = 0; q < 2 * r; ++q) d.st[q].phase = PH_DONE;
        d.ctl->n_active = 0;
        if (d.ctl->h_flag) { *(volatile int*)d.ctl->h_flag = 0; __threadfence_system(); }
        if (d.ctl->graph) {
            cudaGraphSetConditional(d.ctl->h_loop, 0u);
            cudaGraphSetConditional(d.ctl->h_outer, 0u);
        }
        return;
    }
    adi_begin_step(d);
    d.ctl->n_active = 2 * r;
    d.ctl->ticks = 0;
    if (d.ctl->graph) cudaGraphSetConditional(d.ctl->h_loop, 1u);
}

// Per-step set-up over the rows of both sides: zero the solution slots of
// Z and Y, form the Jacobi inverse 1 / (diag + sigma) for the new shift and
// the pre-scaled stencil diagonals of (Op + sigma I) P^{-1}.
template <typename T, typename S, typename C>
__device__ __forceinline__ void adi_step_rows(const AdiDev<T, S, C>& d, int bi) {
    const AdiState<T>* s = d.s;
    const bool sideA = bi < d.nchA;
    const int chunk = sideA ? bi : bi - d.nchA;
    const int nn = sideA ? d.n : d.m;
    const int r0 = chunk * d.rpc, r1 = min(nn, r0 + d.rpc);
    const T sigma = sideA ? s->beta_k : conjg(s->alpha_k);
    T* pinv = sideA ? d.pinvA : d.pinvB;
    C* aval = sideA ? d.avalA : d.avalB;
    const OpDesc& op = sideA ? d.opA : d.opB;
    T* X = d.real_pairs ? (sideA ? d.XA : d.XB) : (sideA ? d.Z : d.Y) + (size_t)(s->k - 1) * d.r * nn;
    count_work(d.ctl, K_STEP, chunk,
               (double)d.r * nn * sizeof(T) + (pinv ? (double)nn * (sizeof(T) + sizeof(double)) : 0.0) +
               (aval ? (double)op.ndiag * nn * (sizeof(double) + sizeof(C)) : 0.0),
               FmaFlops<T>::v * (aval ? (double)op.ndiag * nn : 0.0));
    shifted_op_rows<T, C>(op, sigma, pinv, aval, r0, r1);
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
        for (int l = 0; l < d.r; ++l) X[(size_t)l * nn + i] = zero<T>();
}

template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK) k_adi_step_init(AdiDev<T, S, C> d) {
    count_launch(d.ctl, K_STEP);
    if (d.s->done) return;
    adi_step_rows(d, blockIdx.x);
}

// Gram partials of three n x r blocks (P, Q, R): G[a][b] = sum_i conj(P_a) P_b.
template <typename T>
__device__ __forceinline__ void gram_acc(T* G, const T* v, int r) {
#pragma unroll
    for (int a = 0; a < SYLV_MAXR; ++a)
#pragma unroll
        for (int b = 0; b < SYLV_MAXR; ++b)
            if (a < r && b < r) G[a * SYLV_MAXR + b] += cmul(v[a], v[b]);
}

// Fused factor update and Grams (Algorithm 1, update of w_k, t_k, Z, Y,
// Gamma), then the residual norm ||w_k t_k^*|| = sqrt(lambda_max(G_w G_t)),
// eq. (upd_resgap) and the outer stop test ||w_k t_k^*|| < tau ||f g^*||.
// init = 1: w_0 = f, t_0 = g and the norms of the right-hand side.
// Block bi (of nchA + nchB) of one instance; true in the one thread that
// finished the step (thread 0 of the instance's last block).
template <typename T, typename S, typename C>
__device__ bool adi_gram_body(const AdiDev<T, S, C>& d, int init, int bi) {
    AdiState<T>* s = d.s;
    const bool sideA = bi < d.nchA;
    const int chunk = sideA ? bi : bi - d.nchA;
    const int nn = sideA ? d.n : d.m;
    const int r = d.r;
    const int r0 = chunk * d.rpc, r1 = min(nn, r0 + d.rpc);
    T* W = sideA ? d.w : d.t;
    // w, z, r^A read; w written; three r x r Grams
    count_work(d.ctl, K_GRAM, chunk,
               init ? (double)r * nn * (sizeof(double) + sizeof(T)) : 4.0 * r * nn * sizeof(T),
               FmaFlops<T>::v * (init ? 1.0 : 3.0) * r * r * nn);
    T G[3 * SYLV_MAXR * SYLV_MAXR];
#pragma unroll
    for (int q = 0; q < 3 * SYLV_MAXR * SYLV_MAXR; ++q) G[q] = zero<T>();
    if (init) {
        const double* F = sideA ? d.f : d.g;
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            T v[SYLV_MAXR];
#pragma unroll
            for (int l = 0; l < SYLV_MAXR; ++l) {
                if (l < r) {
                    v[l] = make_scalar<T>(F[(size_t)l * nn + i], 0.0);
                    W[(size_t)l * nn + i] = v[l];
                }
            }
            gram_acc(G, v, r);
        }
    } else {
        const T gm = sideA ? s->gamma_k : conjg(s->gamma_k);
        const T* X = (sideA ? d.Z : d.Y) + (size_t)(s->k - 1) * r * nn;
        const SysDesc<T, S, C>* sd = d.sd + (sideA ? 0 : r);
        // generalized equation: w_k = w_{k-1} + gamma M z_k, t_k = t_{k-1} +
        // conj(gamma) C^* y_k (eq. (lradi_g)); u, v use ||M z||, ||C^T y||
        const OpDesc& op = sideA ? d.opA : d.opB;
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            T wv[SYLV_MAXR], zv[SYLV_MAXR], rv[SYLV_MAXR];
#pragma unroll
            for (int l = 0; l < SYLV_MAXR; ++l) {
                if (l < r) {
                    const T* xl = X + (size_t)l * nn;
                    zv[l] = mass_row<T>(op, i, [&](int q) { return xl[q]; });
                    rv[l] = sd[l].rres ? cvt<T>(sd[l].rres[i]) : cvt<T>(sd[l].V[BasisIx<1>::row(sd[l], i)]);
                    wv[l] = W[(size_t)l * nn + i] + gm * zv[l];
                    W[(size_t)l * nn + i] = wv[l];
                }
            }
            gram_acc(G, wv, r);
            gram_acc(G + SYLV_MAXR * SYLV_MAXR, zv, r);
            gram_acc(G + 2 * SYLV_MAXR * SYLV_MAXR, rv, r);
        }
    }
    block_reduce_store<T, T, 3 * SYLV_MAXR * SYLV_MAXR>(G, 3 * SYLV_MAXR * SYLV_MAXR,
                                                      d.gpart + (size_t)bi * SYLV_GSTRIDE);
    if (!last_block(&s->counter, d.nchA + d.nchB)) return false;
    __shared__ T GA[SYLV_GSTRIDE], GB[SYLV_GSTRIDE];
    reduce_chunks(d.gpart, d.nchA, SYLV_GSTRIDE, SYLV_GSTRIDE, GA);
    reduce_chunks(d.gpart + (size_t)d.nchA * SYLV_GSTRIDE, d.nchB, SYLV_GSTRIDE, SYLV_GSTRIDE, GB);
    if (threadIdx.x != 0) return false;
    s->counter = 0;
    const int RR = SYLV_MAXR * SYLV_MAXR;
    if (init) {
        s->nfg = lowrank_norm_from_grams(GA, GB, r);
        s->Nw = sqrt(herm_lmax(GA, r));
        s->Nt = sqrt(herm_lmax(GB, r));
        s->eps = d.tau * s->nfg;
        s->u = 0.0; s->v = 0.0;
        s->res = s->nfg;
        s->k = 1;
        s->pair_open = 0;
        s->status = 0;
        s->stalled = 0;
        s->itsA = 0; s->itsB = 0; s->cycles = 0;
        s->done = (s->nfg > 0.0) ? 0 : 1;   // f g^* = 0: X = 0 solves eq. (sylv)
        if (!isfinite(s->nfg)) { s->done = 1; s->status = 2; }
    } else {
        const int k = s->k;
        const double nz = sqrt(herm_lmax(GA + RR, r));
        const double nrA = sqrt(herm_lmax(GA + 2 * RR, r));
        const double ny = sqrt(herm_lmax(GB + RR, r));
        const double nrB = sqrt(herm_lmax(GB + 2 * RR, r));
        const double ag = absv(s->gamma_k);
        s->u = s->u + ag * nz * nrB;
        s->v = s->v + ag * ny * nrA;
        const double res = lowrank_norm_from_grams(GA, GB, r);
        long long itA = 0, itB = 0, cyc = 0;
        int stalled = 0, nonfin = 0;
        for (int q = 0; q < 2 * r; ++q) {
            const SysState<T>& st = d.st[q];
            if (q < r) itA += st.iters; else itB += st.iters;
            cyc += st.cycles;
            stalled += (st.status == ST_STALL);
            nonfin |= (st.status == ST_NONFINITE);
        }
        double* h = d.hist + (size_t)(k - 1) * SYLV_HIST_COLS;
        h[0] = k; h[1] = re(s->alpha_k); h[2] = re(s->beta_k); h[3] = s->dA; h[4] = s->dB; h[5] = s->eh;
        h[6] = nrA; h[7] = nrB; h[8] = (double)itA; h[9] = (double)itB; h[10] = s->u; h[11] = s->v;
        h[12] = res / s->nfg; h[13] = s->Nw;
        for (int l = 0; l < r; ++l) d.gam[(size_t)(k - 1) * r + l] = s->gamma_k;
        s->itsA += itA; s->itsB += itB; s->cycles += cyc; s->stalled += stalled;
        s->Nw = sqrt(herm_lmax(GA, r));
        s->Nt = sqrt(herm_lmax(GB, r));
        s->res = res;
        const int idx = (k - 1) % d.nshift;
        s->pair_open = (is_pair_start(d.alpha, d.beta, idx, d.nshift) && !s->pair_open) ? 1 : 0;
        s->k = k + 1;
        if (nonfin || !isfinite(res)) { s->done = 1; s->status = 2; }
        else if (!s->pair_open && res < d.tau * s->nfg) { s->done = 1; s->status = 0; }
        else if (s->k > d.kmax) { s->done = 1; s->status = 1; }
    }
    return true;
}

template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK) k_adi_gram(AdiDev<T, S, C> d, int init) {
    count_launch(d.ctl, K_GRAM);
    AdiState<T>* s = d.s;
    if (!init && s->done) return;
    if (!adi_gram_body(d, init, blockIdx.x)) return;
    if (d.h_done) { *(volatile int*)d.h_done = s->done; __threadfence_system(); }
    if (d.ctl->graph) cudaGraphSetConditional(d.ctl->h_outer, s->done ? 0u : 1u);
}

}  // namespace sylv
