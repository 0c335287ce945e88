// pair_kernels.cuh - the real double step of Algorithm 1 for a complex
// conjugate shift pair (Sec. 3.3 "Complex shift parameters"): steps k and
// k + 1 use (alpha, beta) and (conj alpha, conj beta), gamma = -(alpha + beta),
// and the two steps together keep w, t and the factors real.
//
// With w, t real, the partial-fraction identity
//   (A + conj(b) I)^{-1} (A + b I)^{-1} = [(A + conj(b) I)^{-1} - (A + b I)^{-1}] / (b - conj(b))
// gives the second solution of a side from the first:
//   complex shift: z2 = conj(z1) - gamma Im(z1) / Im(beta)        (one complex solve)
//   real shift:    z2 = z1 + gamma q, (A + beta I) q = z1            (two real solves)
// and on the B side (system B^T + conj(alpha) I) y2 = conj(y1) + conj(gamma)
// Im(y1) / Im(alpha), or y2 = y1 + conj(gamma) q.  So [z1, z2] = [a1, a2] P and
// [y1, y2] = [b1, b2] Q with real blocks a1, a2, b1, b2 and 2 x 2 complex P,
// Q; the pair adds [a1 a2] (G kron I_r) [b1 b2]^T to X with the real core
// G = P diag(gamma, conj gamma) Q^*, w += [a1 a2] P [gamma; conj gamma] and
// t += [b1 b2] Q [conj gamma; gamma].  The inner residuals of the second step
// follow the same columns of P and Q (r2 = conj(r1) - gamma Im(r1) / Im(beta),
// or r1 + gamma r_q), so the residual norms of both steps of the equivalent
// complex formulation - the inputs of eq. (upd_resgap) - come from the real
// Gram matrices of [a1 a2] and of the residual pair.
//
// Device flow of a pair (host-driven): controller (tolerances once for the
// pair) -> set-up -> inner solves of the first solutions -> k_adi_pair_mid
// (keeps the first residual of a real-shift side, starts its second solves)
// -> inner solves (only real-shift sides) -> k_adi_pair_update.
#pragma once
#include "adi_kernels.cuh"

namespace sylv {

#define SYLV_PGSTRIDE (9 * SYLV_MAXR * SYLV_MAXR)   // Gram partials per chunk: r x r + two 2r x 2r

// The last true residual of column system sd at row i (float64 type T).
template <typename T, typename S, typename C>
__device__ __forceinline__ T resid_at(const SysDesc<T, S, C>& sd, int i) {
    return sd.rres ? cvt<T>(sd.rres[i]) : cvt<T>(sd.V[BasisIx<1>::row(sd, i)]);
}

// Between the first and the second solves of a pair: a real-shift side keeps
// its first residual (RsA / RsB) and starts the second solves
// (A + beta I) q = z1 to delta / (2 |gamma|) / r; complex-shift sides are
// finished.  Sets the mapped host flag when second solves run.
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK) k_adi_pair_mid(AdiDev<T, S, C> d) {
    AdiState<T>* s = d.s;
    if (s->done || !s->pair) return;
    const int bi = blockIdx.x;
    const bool sideA = bi < d.nchA;
    const int chunk = sideA ? bi : bi - d.nchA;
    const int nn = sideA ? d.n : d.m;
    const int r = d.r;
    const int r0 = chunk * d.rpc, r1 = min(nn, r0 + d.rpc);
    const bool real_side = sideA ? !s->cplxA : !s->cplxB;
    if (real_side) {
        const SysDesc<T, S, C>* sd = d.sd + (sideA ? 0 : r);
        double* Rs = sideA ? d.RsA : d.RsB;
        T* X2 = sideA ? d.XA2 : d.XB2;
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
            for (int l = 0; l < r; ++l) {
                Rs[(size_t)l * nn + i] = re(resid_at(sd[l], i));
                X2[(size_t)l * nn + i] = zero<T>();
            }
    }
    if (!last_block(&s->counter, d.nchA + d.nchB)) return;
    if (threadIdx.x != 0) return;
    s->counter = 0;
    long long itA = 0, itB = 0, cyc = 0;
    int stalled = 0;
    for (int q = 0; q < 2 * r; ++q) {
        const SysState<T>& st = d.st[q];
        if (q < r) itA += st.iters; else itB += st.iters;
        cyc += st.cycles;
        stalled += (st.status == ST_STALL);
    }
    s->pitsA = itA; s->pitsB = itB; s->pstalled = stalled;
    s->cycles += cyc;
    const double ag = absv(s->gamma_k);
    int count = 0;
    for (int q = 0; q < 2 * r; ++q) {
        const bool qa = q < r;
        if (qa ? s->cplxA : s->cplxB) continue;
        const int l = qa ? q : q - r;
        const int nq = qa ? d.n : d.m;
        SysState<T>& st = d.st[q];
        if (st.status == ST_NONFINITE) continue;
        st.phase = PH_RESID;
        st.j = 0; st.iters = 0; st.cycles = 0; st.status = ST_OK; st.nvec = 0; st.counter = 0;
        st.resnorm = 0.0; st.est = 0.0;
        st.tol = (qa ? s->dA : s->dB) / r / (2.0 * ag);
        st.b = (qa ? d.XA : d.XB) + (size_t)l * nq;
        st.x = (qa ? d.XA2 : d.XB2) + (size_t)l * nq;
        ++count;
    }
    s->stage2 = count > 0;
    d.ctl->n_active = count;
    if (count && d.ctl->h_flag) {
        *(volatile int*)d.ctl->h_flag = 1;
        __threadfence_system();
    }
}

// Complex r x r Hermitian Gram of the combination c1 X1 + c2 X2 of two real
// n x r blocks whose joint 2r x 2r Gram is G (row-major, leading dimension 2R).
// Kept out of line: with r = 4 and all eight calls inlined into
// k_adi_pair_finish the kernel returned wrong norms (checked against host
// eigenvalues of the same Grams); out of line it agrees.
template <int R>
__device__ __noinline__ double combo_gram_lmax(const double* G, cplx c1, cplx c2) {
    cplx H[SYLV_MAXR * SYLV_MAXR];
    for (int q = 0; q < SYLV_MAXR * SYLV_MAXR; ++q) H[q] = cplx{0.0, 0.0};
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) {
            const double g11 = G[a * 2 * R + b], g12 = G[a * 2 * R + R + b];
            const double g21 = G[(R + a) * 2 * R + b], g22 = G[(R + a) * 2 * R + R + b];
            // (c1 x1_a + c2 x2_a)^* (c1 x1_b + c2 x2_b)
            H[a * SYLV_MAXR + b] = abs2(c1) * g11 + cmul(c1, c2) * g12 + cmul(c2, c1) * g21 + abs2(c2) * g22;
        }
    return herm_lmax(H, R);
}

// The coefficients of one side's pair: column j of P (A side, shift beta) or
// Q (B side, shift conj(alpha) in the systems): x_j = a1 P[0][j] + a2 P[1][j].
__device__ __forceinline__ void pair_coeffs(bool cplx_side, bool sideA, cplx gam, double im_shift, cplx P[2][2]) {
    const cplx c = sideA ? gam : cplx{-gam.x, gam.y};     // gamma, or -conj(gamma)
    P[0][0] = cplx{1.0, 0.0};
    P[0][1] = cplx{1.0, 0.0};
    if (cplx_side) {
        P[1][0] = cplx{0.0, 1.0};
        P[1][1] = cplx{-c.x / im_shift, -1.0 - c.y / im_shift};   // -i - c / Im(shift)
    } else {
        P[1][0] = cplx{0.0, 0.0};
        P[1][1] = sideA ? gam : conjg(gam);
    }
}

// Factor update of a plain step or of a pair (real double step) with the
// Grams of w (t), of [a1 a2] and of the residual pair; the last block
// evaluates eq. (upd_resgap) for both steps of a pair, the residual norm
// ||w t^*|| and the outer stop test.
template <typename T, typename S, typename C, int R>
__global__ void __launch_bounds__(SYLV_BLOCK) k_adi_pair_update(AdiDev<T, S, C> d) {
    count_launch(d.ctl, K_GRAM);
    AdiState<T>* s = d.s;
    if (s->done) return;
    const int bi = blockIdx.x;
    const bool sideA = bi < d.nchA;
    const int chunk = sideA ? bi : bi - d.nchA;
    const int nn = sideA ? d.n : d.m;
    const int r0 = chunk * d.rpc, r1 = min(nn, r0 + d.rpc);
    const int k = s->k;
    const bool pair = s->pair != 0;
    const bool cside = sideA ? s->cplxA : s->cplxB;
    const T* X = sideA ? d.XA : d.XB;
    const T* X2 = sideA ? d.XA2 : d.XB2;
    const double* Rs = sideA ? d.RsA : d.RsB;
    T* W = sideA ? d.w : d.t;
    double* F = (sideA ? d.Zr : d.Yr) + (size_t)(k - 1) * R * nn;
    const SysDesc<T, S, C>* sd = d.sd + (sideA ? 0 : R);
    const cplx gam = to_cplx(s->gamma_k);
    double c1, c2 = 0.0;
    if (pair) {
        cplx P[2][2];
        const double ims = sideA ? im(s->beta_k) : im(s->alpha_k);
        pair_coeffs(cside, sideA, gam, ims, P);
        // w: P [gamma; conj gamma], t: Q [conj gamma; gamma]
        const cplx g1 = sideA ? gam : conjg(gam), g2 = sideA ? conjg(gam) : gam;
        c1 = re(P[0][0] * g1 + P[0][1] * g2);
        c2 = re(P[1][0] * g1 + P[1][1] * g2);
    } else {
        c1 = gam.x;                          // real shifts: gamma real, conj(gamma) = gamma
    }
    count_work(d.ctl, K_GRAM, chunk, (pair ? 8.0 : 5.0) * R * nn * sizeof(double), 2.0 * 9.0 * R * R * nn);
    // Grams of w (R x R), [a1 a2] (2R x 2R) and of the residual pair (2R x 2R),
    // accumulated cooperatively: a tile of TILE rows is staged in shared
    // memory by the first TILE threads, then thread e adds its Gram entry e
    // over the tile (one accumulator per thread instead of 9 R^2).
    constexpr int NW = R * R, NA = 4 * R * R, NG = NW + 2 * NA;
    constexpr int TILE = 64, NV = 5 * R;                    // per row: a (2R), rv (2R), wv (R)
    static_assert(NG <= SYLV_BLOCK, "one Gram entry per thread");
    __shared__ double tile[TILE][NV];
    const int e = threadIdx.x;
    int e1 = 0, e2 = 0;                                     // the two row values entry e multiplies
    if (e < NW) { e1 = 4 * R + e / R; e2 = 4 * R + e % R; }
    else if (e < NW + NA) { e1 = (e - NW) / (2 * R); e2 = (e - NW) % (2 * R); }
    else if (e < NG) { e1 = 2 * R + (e - NW - NA) / (2 * R); e2 = 2 * R + (e - NW - NA) % (2 * R); }
    double acc = 0.0;
    for (int base = r0; base < r1; base += TILE) {
        const int t = threadIdx.x;
        if (t < TILE) {
            const int i = base + t;
            double* row = tile[t];
            if (i < r1) {
#pragma unroll
                for (int l = 0; l < R; ++l) {
                    const T x = X[(size_t)l * nn + i];
                    const T res = resid_at(sd[l], i);
                    const double a1 = re(x);
                    const double a2 = !pair ? 0.0 : (cside ? im(x) : re(X2[(size_t)l * nn + i]));
                    row[l] = a1;
                    row[R + l] = a2;
                    row[2 * R + l] = pair && !cside ? Rs[(size_t)l * nn + i] : re(res);
                    row[3 * R + l] = !pair ? 0.0 : (cside ? im(res) : re(res));
                    F[(size_t)l * nn + i] = a1;
                    if (pair) F[(size_t)(R + l) * nn + i] = a2;
                    const double wn = re(W[(size_t)l * nn + i]) + c1 * a1 + c2 * a2;
                    row[4 * R + l] = wn;
                    W[(size_t)l * nn + i] = make_scalar<T>(wn, 0.0);
                }
            } else {
#pragma unroll
                for (int q = 0; q < NV; ++q) row[q] = 0.0;
            }
        }
        __syncthreads();
        if (e < NG)
#pragma unroll 8
            for (int q = 0; q < TILE; ++q) acc += tile[q][e1] * tile[q][e2];
        __syncthreads();
    }
    if (e < NG) d.pgpart[(size_t)bi * SYLV_PGSTRIDE + e] = acc;
    if (!last_block(&s->counter, d.nchA + d.nchB)) return;
    // the reduced Grams go to the slots after the chunk partials; the scalar
    // evaluation runs in k_adi_pair_finish (one small block)
    double* GAg = d.pgpart + (size_t)(d.nchA + d.nchB) * SYLV_PGSTRIDE;
    reduce_chunks(d.pgpart, d.nchA, SYLV_PGSTRIDE, NG, GAg);
    reduce_chunks(d.pgpart + (size_t)d.nchA * SYLV_PGSTRIDE, d.nchB, SYLV_PGSTRIDE, NG, GAg + SYLV_PGSTRIDE);
    if (threadIdx.x == 0) s->counter = 0;
}

// The scalar part of the pair update (thread 0): eq. (upd_resgap) for both
// steps of a pair from the reduced Grams, the history rows, the 2 x 2 core,
// the residual norm ||w t^*|| and the outer stop test.
template <typename T, typename S, typename C, int R>
__global__ void k_adi_pair_finish(AdiDev<T, S, C> d) {
    AdiState<T>* s = d.s;
    if (s->done || threadIdx.x != 0) return;
    constexpr int NW = R * R, NA = 4 * R * R;
    const double* GA = d.pgpart + (size_t)(d.nchA + d.nchB) * SYLV_PGSTRIDE;
    const double* GB = GA + SYLV_PGSTRIDE;
    const int k = s->k;
    const bool pair = s->pair != 0;
    const cplx gam = to_cplx(s->gamma_k);
    const double ag = absv(gam);
    // inner steps: the first solves of a pair were counted by k_adi_pair_mid
    long long itA = pair ? s->pitsA : 0, itB = pair ? s->pitsB : 0, cyc = 0;
    int stalled = pair ? s->pstalled : 0, nonfin = 0;
    for (int q = 0; q < 2 * R; ++q) {
        const SysState<T>& st = d.st[q];
        const bool qa = q < R;
        nonfin |= (st.status == ST_NONFINITE);
        const bool counted = !pair || (s->stage2 && !(qa ? s->cplxA : s->cplxB));
        if (!counted) continue;
        if (qa) itA += st.iters; else itB += st.iters;
        cyc += st.cycles;
        stalled += (st.status == ST_STALL);
    }
    // spectral norms of r x r blocks; Grams of a combination of the two halves
    double Gw_A[SYLV_MAXR * SYLV_MAXR], Gw_B[SYLV_MAXR * SYLV_MAXR];
    for (int q = 0; q < SYLV_MAXR * SYLV_MAXR; ++q) { Gw_A[q] = 0.0; Gw_B[q] = 0.0; }
    for (int p = 0; p < R; ++p)
        for (int q = 0; q < R; ++q) {
            Gw_A[p * SYLV_MAXR + q] = GA[p * R + q];
            Gw_B[p * SYLV_MAXR + q] = GB[p * R + q];
        }
    double* hrow = d.hist + (size_t)(k - 1) * SYLV_HIST_COLS;
    double u = s->u, v = s->v;
    const cplx one{1.0, 0.0}, nil{0.0, 0.0};
    if (!pair) {
        const double nz = sqrt((combo_gram_lmax<R>(GA + NW, one, nil)));
        const double nrA = sqrt((combo_gram_lmax<R>(GA + NW + NA, one, nil)));
        const double ny = sqrt((combo_gram_lmax<R>(GB + NW, one, nil)));
        const double nrB = sqrt((combo_gram_lmax<R>(GB + NW + NA, one, nil)));
        u += ag * nz * nrB;
        v += ag * ny * nrA;
        hrow[0] = k; hrow[1] = re(s->alpha_k); hrow[2] = re(s->beta_k); hrow[3] = s->dA; hrow[4] = s->dB;
        hrow[5] = s->eh; hrow[6] = nrA; hrow[7] = nrB; hrow[8] = (double)itA; hrow[9] = (double)itB;
        hrow[10] = u; hrow[11] = v; hrow[13] = s->Nw;
        double* cr = d.core + (size_t)(k - 1) * 5;
        cr[0] = 1.0; cr[1] = gam.x; cr[2] = 0.0; cr[3] = 0.0; cr[4] = 0.0;
    } else {
        cplx P[2][2], Q[2][2];
        pair_coeffs(s->cplxA, true, gam, im(s->beta_k), P);
        pair_coeffs(s->cplxB, false, gam, im(s->alpha_k), Q);
        double nz[2], ny[2], nrA[2], nrB[2];
        for (int j = 0; j < 2; ++j) {
            nz[j] = sqrt((combo_gram_lmax<R>(GA + NW, P[0][j], P[1][j])));
            nrA[j] = sqrt((combo_gram_lmax<R>(GA + NW + NA, P[0][j], P[1][j])));
            ny[j] = sqrt((combo_gram_lmax<R>(GB + NW, Q[0][j], Q[1][j])));
            nrB[j] = sqrt((combo_gram_lmax<R>(GB + NW + NA, Q[0][j], Q[1][j])));
        }
        // G = P diag(gamma, conj gamma) Q^*
        const cplx gd[2] = {gam, conjg(gam)};
        double* cr = d.core + (size_t)(k - 1) * 5;
        cr[0] = 2.0;
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                cplx acc = nil;
                for (int j = 0; j < 2; ++j) acc += P[p][j] * (gd[j] * conjg(Q[q][j]));
                cr[1 + 2 * p + q] = acc.x;
            }
        double* cr2 = cr + 5;
        cr2[0] = 3.0; cr2[1] = cr2[2] = cr2[3] = cr2[4] = 0.0;
        for (int j = 0; j < 2; ++j) {
            double* h = hrow + (size_t)j * SYLV_HIST_COLS;
            u += ag * nz[j] * nrB[j];
            v += ag * ny[j] * nrA[j];
            const T al = j == 0 ? s->alpha_k : conjg(s->alpha_k), be = j == 0 ? s->beta_k : conjg(s->beta_k);
            h[0] = k + j; h[1] = re(al); h[2] = re(be); h[3] = s->dA; h[4] = s->dB; h[5] = s->eh;
            h[6] = nrA[j]; h[7] = nrB[j]; h[8] = j == 0 ? (double)itA : 0.0; h[9] = j == 0 ? (double)itB : 0.0;
            h[10] = u; h[11] = v; h[13] = s->Nw;
        }
    }
    const double res = lowrank_norm_from_grams(Gw_A, Gw_B, R);
    hrow[12] = res / s->nfg;
    if (pair) hrow[SYLV_HIST_COLS + 12] = res / s->nfg;
    s->u = u;
    s->v = v;
    s->itsA += itA; s->itsB += itB; s->cycles += cyc; s->stalled += stalled;
    s->Nw = sqrt(herm_lmax(Gw_A, R));
    s->Nt = sqrt(herm_lmax(Gw_B, R));
    s->res = res;
    s->pair_open = 0;
    s->k = k + (pair ? 2 : 1);
    if (nonfin || !isfinite(res)) { s->done = 1; s->status = 2; }
    else if (res < d.tau * s->nfg) { s->done = 1; s->status = 0; }
    else if (s->k > d.kmax) { s->done = 1; s->status = 1; }
    if (d.h_done) { *(volatile int*)d.h_done = s->done; __threadfence_system(); }
}

}  // namespace sylv
