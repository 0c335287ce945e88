// bicg_kernels.cuh - BiCGstab (van der Vorst, SIAM J. Sci. Stat. Comput. 13,
// 1992) for the shifted inner systems of Algorithm 1, the short-recurrence
// solver the paper runs in its experiments (Sec. 3.3 "Further implementation
// aspects", Sec. 4).  Right Jacobi preconditioning keeps the recurrence
// residual that of the original system; each column l stops at
// ||r(:, l)|| <= delta_k / r, confirmed by the true residual recomputed in
// float64 (a new cycle with a fresh shadow vector starts otherwise).
//
// One step of a column, with Op' = (Op + sigma I) P^{-1}:
//   p = r + beta q,  v = Op' p,  alpha = rho / (rhat^* v)             (k_bicg_a)
//   s = r - alpha v, t = Op' s,  omega = t^* s / t^* t                 (k_bicg_b)
//   x += P^{-1}(alpha p + omega s),  r = s - omega t,  q = p - omega v,
//   rho' = rhat^* r,  beta' = (rho' / rho)(alpha / omega)              (k_bicg_c)
// where q = p - omega v is the part of the next search direction that is
// known before rho' (so k_bicg_a forms p at the stencil neighbours from r and
// q on the fly: no grid-wide barrier between the update of p and its
// product).  Each kernel ends in one grid reduction, finished by the last
// block of each group.
//
// Work is organised by groups: the r column systems of one side of one
// instance share the operator, the shift and the rows, so a work item
// (group, row chunk) applies the stencil to all of the group's active
// columns at once and every stored diagonal value is read once per row for
// all r columns (an SpMM over the right-hand-side columns).
#pragma once
#include "gmres_kernels.cuh"

namespace sylv {

constexpr int BG_MAXCOL = 4;                     // columns of a group (the rank cap)
constexpr int BG_PSTRIDE = 3 * BG_MAXCOL;        // partial sums per chunk (at most 3 per column)
// Resident blocks per SM the step kernels are compiled for: they stream a
// few vectors per row and need many loads in flight, so occupancy comes
// before registers (the counts keep the stencil path of the product free of
// spills for each type).
template <typename C> struct BicgOcc { static constexpr int value = 3; };
template <> struct BicgOcc<float> { static constexpr int value = 4; };
template <> struct BicgOcc<cplx> { static constexpr int value = 2; };

// Vectors of one BiCGstab system, column-major, ldv apart, C precision.
enum BVec : int { BV_R = 0, BV_Q = 1, BV_P = 2, BV_V = 3, BV_T = 4, BV_RH = 5, BV_COUNT = 6 };

// A group: systems sys0 .. sys0 + ncol - 1 (same operator, shift and rows;
// their vectors lie BV_COUNT * ldv apart), its chunk partial sums and its
// completion counter.
template <typename T>
struct BGroup {
    int sys0, ncol, nchunks;
    T* part;                 // nchunks x BG_PSTRIDE
    unsigned* counter;
};

template <typename C> HD C from_real(typename RealOf<C>::type x) { return make_scalar<C>((double)x, 0.0); }
template <> HD double from_real<double>(double x) { return x; }
template <> HD float from_real<float>(float x) { return x; }

// y[q] = ((Op + sigma I) P^{-1} X_q)(i) for the columns q of mask.  Stencil
// operators use the pre-scaled diagonals aval (one load per diagonal for all
// columns); other operators the float64 row with the Jacobi inverse.
template <typename T, typename S, typename C, typename XF>
__device__ __forceinline__ void group_op_row(const SysDesc<T, S, C>& sd, const OpDesc& op, T sigma, int i,
                                             int mask, XF X, C (&y)[BG_MAXCOL]) {
#pragma unroll
    for (int q = 0; q < BG_MAXCOL; ++q) y[q] = zero<C>();
    if (sd.aval) {
        const C* __restrict__ av = sd.aval;
#pragma unroll
        for (int d = 0; d < SYLV_MAXDIAG; ++d) {
            if (d < op.ndiag) {
                const int k = i + op.offs[d];
                if (k >= 0 && k < op.n) {
                    const C a = ldro(av + (size_t)d * op.n + i);
#pragma unroll
                    for (int q = 0; q < BG_MAXCOL; ++q)
                        if (mask >> q & 1) y[q] += a * X(q, k);
                }
            }
        }
    } else {
        const T* __restrict__ pinv = sd.pinv;
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q)
            if (mask >> q & 1)
                y[q] = cvt<C>(op_row<T>(op, i, sigma, [&](int k) {
                    const T x = cvt<T>(X(q, k));
                    return pinv ? pinv[k] * x : x;
                }));
    }
}

// Block sums of NV accumulators (warps combined in A, each sum converted to T
// once) written to out[0..NV).
template <typename T, typename A, int NV>
__device__ __forceinline__ void bg_block_sums(A (&acc)[NV], T* out) {
    __shared__ A red[SYLV_NWARP][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < NV; ++l) {
        const A v = warp_sum(acc[l]);
        if (lane == 0) red[warp][l] = v;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < NV; l += blockDim.x) {
        A s = red[0][l];
#pragma unroll
        for (int w = 1; w < SYLV_NWARP; ++w) s += red[w][l];
        out[l] = cvt<T>(s);
    }
}

// Active columns of a group (phase == ph), as a bit mask.
template <typename T>
__device__ __forceinline__ int group_mask(const SysState<T>* sts, const BGroup<T>& g, int ph) {
    int mask = 0;
    for (int q = 0; q < g.ncol; ++q)
        if (sts[g.sys0 + q].phase == ph) mask |= 1 << q;
    return mask;
}

// End of a BiCGstab cycle: the restart kernel recomputes the true residual.
template <typename T>
__device__ __forceinline__ void bicg_end_cycle(SysState<T>* st) {
    st->bfin = 0;
    st->phase = PH_RESID;
}

// ---------------------------------------------------------------------------
// Step part a: p = r + beta q, v = Op' p, partial rhat^* v.  The last block of
// a group counts the step and sets alpha = rho / (rhat^* v); a zero or
// non-finite denominator ends the cycle (breakdown) without an update.
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK, BicgOcc<C>::value)
k_bicg_a(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts, const OpDesc* __restrict__ ops,
         const BGroup<T>* __restrict__ groups, const Item* __restrict__ items, BatchCtl* ctl) {
    pdl_wait();
    count_launch(ctl, K_SPMV);
    if (ctl->graph && blockIdx.x == 0 && threadIdx.x == 0) {
        cudaGraphSetConditional(ctl->h_loop, 0u);
        if (ctl->bouter) cudaGraphSetConditional(ctl->h_bouter, 0u);
    }
    const Item it = items[blockIdx.x];
    const BGroup<T> g = groups[it.sys];
    const int mask = group_mask(sts, g, PH_ARNOLDI);
    if (!mask) return;
    const SysDesc<T, S, C> sd = sysd[g.sys0];
    const OpDesc op = ops[sd.op];
    const size_t ld = sd.ldv;
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    const int na = __popc(mask);
    count_work(ctl, K_SPMV, it.chunk, (double)op.nnz * sizeof(C) + 5.0 * na * sd.n * sizeof(C),
               FmaFlops<C>::v * na * ((double)op.nnz + 2.0 * sd.n));
    C beta[BG_MAXCOL];
#pragma unroll
    for (int q = 0; q < BG_MAXCOL; ++q)
        beta[q] = (mask >> q & 1) ? cvt<C>(sts[g.sys0 + q].bbeta) : zero<C>();
    // vector v of column q: bv + (q BV_COUNT + v) ld
    C* __restrict__ bv = sd.bv;
    const size_t cs = (size_t)BV_COUNT * ld;
    const T sigma = sts[g.sys0].sigma;
    C acc[BG_MAXCOL];
#pragma unroll
    for (int q = 0; q < BG_MAXCOL; ++q) acc[q] = zero<C>();
    // r, q, rhat and the stencil are not written here: read-only loads
    auto P = [&](int q, int k) {
        const C* c = bv + q * cs + (size_t)k;
        return ldro(c + BV_R * ld) + beta[q] * ldro(c + BV_Q * ld);
    };
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        C y[BG_MAXCOL];
        group_op_row(sd, op, sigma, i, mask, P, y);
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q) {
            if (mask >> q & 1) {
                C* c = bv + q * cs + (size_t)i;
                c[BV_P * ld] = P(q, i);
                c[BV_V * ld] = y[q];
                acc[q] += cmul(ldro(c + BV_RH * ld), y[q]);
            }
        }
    }
    bg_block_sums<T, C, BG_MAXCOL>(acc, g.part + (size_t)it.chunk * BG_PSTRIDE);
    pdl_trigger();
    if (!last_block(g.counter, g.nchunks)) return;
    __shared__ T tot[BG_PSTRIDE];
    reduce_chunks(g.part, g.nchunks, BG_PSTRIDE, BG_MAXCOL, tot);
    const int q = threadIdx.x;
    if (q < g.ncol && (mask >> q & 1)) {
        SysState<T>* st = sts + g.sys0 + q;
        const T den = tot[q];
        st->iters += 1;
        const double ad = absv(den);
        if (!(ad > 0.0) || !isfinite(ad)) {
            bicg_end_cycle(st);
        } else {
            st->balpha = sdiv(st->brho, den);
        }
    }
    if (threadIdx.x == 0) *g.counter = 0;
}

// ---------------------------------------------------------------------------
// Step part b: s = r - alpha v, t = Op' s, partial t^* s, t^* t, s^* s.  The
// last block sets omega = t^* s / t^* t, or ends the step early (omega = 0)
// when ||s|| already meets the tolerance.
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK, BicgOcc<C>::value)
k_bicg_b(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts, const OpDesc* __restrict__ ops,
         const BGroup<T>* __restrict__ groups, const Item* __restrict__ items, BatchCtl* ctl) {
    pdl_wait();
    count_launch(ctl, K_CGS2);
    const Item it = items[blockIdx.x];
    const BGroup<T> g = groups[it.sys];
    const int mask = group_mask(sts, g, PH_ARNOLDI);
    if (!mask) return;
    const SysDesc<T, S, C> sd = sysd[g.sys0];
    const OpDesc op = ops[sd.op];
    const size_t ld = sd.ldv;
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    const int na = __popc(mask);
    count_work(ctl, K_CGS2, it.chunk, (double)op.nnz * sizeof(C) + 3.0 * na * sd.n * sizeof(C),
               FmaFlops<C>::v * na * ((double)op.nnz + 4.0 * sd.n));
    C alpha[BG_MAXCOL];
#pragma unroll
    for (int q = 0; q < BG_MAXCOL; ++q)
        alpha[q] = (mask >> q & 1) ? cvt<C>(sts[g.sys0 + q].balpha) : zero<C>();
    C* __restrict__ bv = sd.bv;
    const size_t cs = (size_t)BV_COUNT * ld;
    const T sigma = sts[g.sys0].sigma;
    C acc[3 * BG_MAXCOL];
#pragma unroll
    for (int q = 0; q < 3 * BG_MAXCOL; ++q) acc[q] = zero<C>();
    // r, v and the stencil are not written here: read-only loads
    auto Sf = [&](int q, int k) {
        const C* c = bv + q * cs + (size_t)k;
        return ldro(c + BV_R * ld) - alpha[q] * ldro(c + BV_V * ld);
    };
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        C y[BG_MAXCOL];
        group_op_row(sd, op, sigma, i, mask, Sf, y);
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q) {
            if (mask >> q & 1) {
                const C si = Sf(q, i);
                bv[q * cs + (size_t)BV_T * ld + i] = y[q];
                acc[3 * q] += cmul(y[q], si);
                acc[3 * q + 1] += from_real<C>(abs2(y[q]));
                acc[3 * q + 2] += from_real<C>(abs2(si));
            }
        }
    }
    bg_block_sums<T, C, 3 * BG_MAXCOL>(acc, g.part + (size_t)it.chunk * BG_PSTRIDE);
    pdl_trigger();
    if (!last_block(g.counter, g.nchunks)) return;
    __shared__ T tot[BG_PSTRIDE];
    reduce_chunks(g.part, g.nchunks, BG_PSTRIDE, 3 * BG_MAXCOL, tot);
    const int q = threadIdx.x;
    if (q < g.ncol && (mask >> q & 1)) {
        SysState<T>* st = sts + g.sys0 + q;
        const T ts = tot[3 * q];
        const double tt = re(tot[3 * q + 1]);
        const double sn = sqrt(re(tot[3 * q + 2]));
        if (sn <= st->tol) {
            st->bomega = zero<T>();
            st->bfin = 1;
            st->est = sn;
        } else {
            const T om = tt > 0.0 ? ts * (1.0 / tt) : zero<T>();
            // a non-finite omega ends the step like a converged s (omega = 0,
            // x += alpha P^{-1} p); the restart then checks the true residual
            const bool ok = isfinite(absv(om));
            st->bomega = ok ? om : zero<T>();
            st->bfin = ok ? 0 : 1;
            st->est = sn;
        }
    }
    if (threadIdx.x == 0) *g.counter = 0;
}

// ---------------------------------------------------------------------------
// Step part c: x += P^{-1}(alpha p + omega s) in float64, r = s - omega t,
// q = p - omega v, partial rhat^* r and r^* r.  The last block records the
// residual norm and ends the cycle when it meets the tolerance, at the step
// cap or at a breakdown (rho' = 0 or omega = 0); otherwise it sets
// beta' = (rho' / rho)(alpha / omega).
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK, BicgOcc<C>::value)
k_bicg_c(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
         const BGroup<T>* __restrict__ groups, const Item* __restrict__ items, BatchCtl* ctl) {
    pdl_wait();
    count_launch(ctl, K_CGS3);
    const Item it = items[blockIdx.x];
    const BGroup<T> g = groups[it.sys];
    const int mask = group_mask(sts, g, PH_ARNOLDI);
    if (mask) {
        const SysDesc<T, S, C> sd = sysd[g.sys0];
        const size_t ld = sd.ldv;
        const int r0 = it.chunk * sd.rows_per_chunk;
        const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
        const int na = __popc(mask);
        count_work(ctl, K_CGS3, it.chunk,
                   7.0 * na * sd.n * sizeof(C) + 2.0 * na * sd.n * sizeof(T) + (sd.pinv ? (double)sd.n * sizeof(T) : 0.0),
                   FmaFlops<C>::v * na * 6.0 * sd.n);
        C alpha[BG_MAXCOL], omega[BG_MAXCOL];
        T* X[BG_MAXCOL];
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q) {
            const bool on = mask >> q & 1;
            alpha[q] = on ? cvt<C>(sts[g.sys0 + q].balpha) : zero<C>();
            omega[q] = on ? cvt<C>(sts[g.sys0 + q].bomega) : zero<C>();
            X[q] = on ? sts[g.sys0 + q].x : nullptr;
        }
        C* __restrict__ bv = sd.bv;
        const size_t cs = (size_t)BV_COUNT * ld;
        const T* __restrict__ pinv = sd.pinv;
        C acc[2 * BG_MAXCOL];
#pragma unroll
        for (int q = 0; q < 2 * BG_MAXCOL; ++q) acc[q] = zero<C>();
        // every element is read and then overwritten by the same thread only:
        // read-only loads, so the next row's loads may pass this row's stores
#pragma unroll 2
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const T pi = pinv ? ldro(pinv + i) : make_scalar<T>(1.0, 0.0);
#pragma unroll
            for (int q = 0; q < BG_MAXCOL; ++q) {
                if (mask >> q & 1) {
                    C* c = bv + q * cs + (size_t)i;
                    const C p = ldro(c + BV_P * ld), v = ldro(c + BV_V * ld), r = ldro(c + BV_R * ld);
                    const C t = ldro(c + BV_T * ld), rh = ldro(c + BV_RH * ld);
                    const T xo = ldro(X[q] + i);
                    const C s = r - alpha[q] * v;
                    X[q][i] = xo + pi * cvt<T>(alpha[q] * p + omega[q] * s);
                    const C rn = s - omega[q] * t;
                    c[BV_R * ld] = rn;
                    c[BV_Q * ld] = p - omega[q] * v;
                    acc[2 * q] += cmul(rh, rn);
                    acc[2 * q + 1] += from_real<C>(abs2(rn));
                }
            }
        }
        bg_block_sums<T, C, 2 * BG_MAXCOL>(acc, g.part + (size_t)it.chunk * BG_PSTRIDE);
        if (last_block(g.counter, g.nchunks)) {
            __shared__ T tot[BG_PSTRIDE];
            reduce_chunks(g.part, g.nchunks, BG_PSTRIDE, 2 * BG_MAXCOL, tot);
            const int q = threadIdx.x;
            if (q < g.ncol && (mask >> q & 1)) {
                SysState<T>* st = sts + g.sys0 + q;
                const SysDesc<T, S, C>& sq = sysd[g.sys0 + q];
                const T rho_new = tot[2 * q];
                const double rnorm = sqrt(re(tot[2 * q + 1]));
                const double est = st->bfin ? st->est : rnorm;
                const int iters = st->iters;
                st->est = est;
                if (sq.hist && iters - 1 < sq.hist_cap && iters >= 1) sq.hist[iters - 1] = est;
                const T om = st->bomega;
                // 32-bit vectors: the recurrence residual drifts from the true
                // one, so a cycle also ends after four orders of magnitude of
                // reduction, or on growth by two (the restart recomputes the
                // residual and the shadow vector in float64, iterative refinement)
                const bool drift = sizeof(typename RealOf<C>::type) == 4 &&
                                   (rnorm < 1e-4 * st->bnorm0 || rnorm > 1e2 * st->bnorm0);
                if (st->bfin || !(est > st->tol) || iters >= st->max_iters || absv(rho_new) == 0.0 ||
                    absv(om) == 0.0 || !isfinite(rnorm) || drift) {
                    bicg_end_cycle(st);
                } else {
                    st->bbeta = sdiv(rho_new, st->brho) * sdiv(st->balpha, om);
                    st->brho = rho_new;
                }
            }
            if (threadIdx.x == 0) *g.counter = 0;
        }
    }
    if (ctl->graph) graph_tail<T>(ctl, sts, K_CGS3);
}

// ---------------------------------------------------------------------------
// Restart: r = b - (Op + sigma I) x in float64 for the columns whose cycle
// ended, stored (C precision) as the new residual and shadow vector, q = 0,
// ||r||; then done (tolerance met, step cap, non-finite) or a new cycle with
// rho = ||r||^2, beta = 0.  Grid-stride over the group work items.
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
__device__ __forceinline__ void bicg_resid_item(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
                                                const OpDesc* __restrict__ ops, const BGroup<T>& g, int chunk,
                                                BatchCtl* ctl) {
    const int mask = group_mask(sts, g, PH_RESID);
    if (!mask) return;
    const SysDesc<T, S, C> sd = sysd[g.sys0];
    const OpDesc op = ops[sd.op];
    const size_t ld = sd.ldv;
    const int r0 = chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    const int na = __popc(mask);
    count_work(ctl, K_RRES, chunk, (double)op.nnz * sizeof(double) + na * sd.n * (2.0 * sizeof(T) + 3.0 * sizeof(C)),
               FmaFlops<T>::v * na * ((double)op.nnz + 2.0 * sd.n));
    const T sigma = sts[g.sys0].sigma;
    double acc[BG_MAXCOL] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < BG_MAXCOL; ++q) {
        if (!(mask >> q & 1)) continue;
        const T* __restrict__ x = sts[g.sys0 + q].x;
        const T* __restrict__ b = sts[g.sys0 + q].b;
        C* base = sd.bv + (size_t)q * BV_COUNT * ld;
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const T r = b[i] - op_row<T>(op, i, sigma, [&](int k) { return x[k]; });
            const C rc = cvt<C>(r);
            base[BV_R * ld + i] = rc;
            base[BV_RH * ld + i] = rc;
            base[BV_Q * ld + i] = zero<C>();
            acc[q] += abs2(r);
        }
    }
    bg_block_sums<double, double, BG_MAXCOL>(acc, reinterpret_cast<double*>(g.part + (size_t)chunk * BG_PSTRIDE));
    if (!last_block(g.counter, g.nchunks)) return;
    __shared__ double tot[BG_MAXCOL];
    reduce_chunks(reinterpret_cast<const double*>(g.part), g.nchunks, BG_PSTRIDE * (int)(sizeof(T) / sizeof(double)),
                  BG_MAXCOL, tot);
    const int q = threadIdx.x;
    if (q < g.ncol && (mask >> q & 1)) {
        SysState<T>* st = sts + g.sys0 + q;
        const double rn = sqrt(tot[q]);
        st->resnorm = rn;
        bool done = false;
        if (st->status == ST_NONFINITE || !isfinite(rn)) {
            st->status = ST_NONFINITE;
            done = true;
        } else if (rn <= st->tol) {
            done = true;
        } else if (st->iters >= st->max_iters) {
            st->status = ST_STALL;
            done = true;
        }
        if (done) {
            mark_done(st, ctl);
        } else {
            st->cycles += 1;
            st->brho = make_scalar<T>(rn * rn, 0.0);
            st->bnorm0 = rn;
            st->bbeta = zero<T>();
            st->balpha = make_scalar<T>(1.0, 0.0);
            st->bomega = make_scalar<T>(1.0, 0.0);
            st->bfin = 0;
            st->phase = PH_ARNOLDI;
        }
    }
    if (threadIdx.x == 0) *g.counter = 0;
}

template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_bicg_resid(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts, const OpDesc* __restrict__ ops,
             const BGroup<T>* __restrict__ groups, const Item* __restrict__ items, int nitems, BatchCtl* ctl) {
    pdl_wait();
    count_launch(ctl, K_RRES);
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const Item it = items[w];
        bicg_resid_item<T, S, C>(sysd, sts, ops, groups[it.sys], it.chunk, ctl);
        __syncthreads();          // shared reduction buffers are reused by the next item
    }
    if (ctl->graph) graph_tail<T>(ctl, sts, K_RRES);
}

}  // namespace sylv
