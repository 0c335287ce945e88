// gmres_kernels.cuh - device kernels of the batched restarted GMRES(m) that
// solves the shifted inner systems of Algorithm 1 (inexact LR-ADI):
//   (A + beta_k I) z = w_{k-1}(:, l)   and   (B^T + conj(alpha_k) I) y = t_{k-1}(:, l),
// each column separately with right Jacobi preconditioning and the stop test
// ||r(:, l)|| <= delta_k / r (Sec. 3.3, "Further implementation aspects").
//
// One launch serves every active system of a batch: the grid is a list of
// (system, chunk) work items, each chunk a contiguous row range.  An Arnoldi
// step is three sweeps over the rows (classical Gram-Schmidt applied twice):
//   k_arnoldi_spmv : w = (Op + sigma I) P^{-1} v_j and h1 = V^* w (fused)
//   k_cgs_pass2    : h2 = V^* (w - V h1)
//   k_cgs_pass3    : v_{j+1} = w - V (h1 + h2), ||v_{j+1}||, then the Givens
//                    update of the Hessenberg least-squares problem
// and a restart is two more:
//   k_restart_update   : x += P^{-1} V y
//   k_restart_residual : r = b - (Op + sigma I) x in float64, ||r||, decision.
// Chunk partial sums are reduced by the last block of each system to finish
// (a completion counter per system), in a fixed order, so results do not
// depend on block scheduling.  Basis vectors are stored unnormalised with a
// scale factor, so no separate normalisation sweep is needed.  Template
// roles: T float64 scalar, S basis storage, C sweep arithmetic (common.cuh).
#pragma once
#include "common.cuh"

namespace sylv {

constexpr int PSTRIDE = SYLV_MAXV + 1;     // partial-sum slots per chunk

// Per-thread accumulators (type A) -> block sums in type T written to out[0..cnt).
template <typename T, typename A, int NV>
__device__ __forceinline__ void block_reduce_store(A (&acc)[NV], int cnt, T* out) {
    __shared__ T red[SYLV_NWARP][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < NV; ++l) {
        if (l < cnt) {
            T v = warp_sum(cvt<T>(acc[l]));
            if (lane == 0) red[warp][l] = v;
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
        T s = zero<T>();
#pragma unroll
        for (int w = 0; w < SYLV_NWARP; ++w) s += red[w][l];
        out[l] = s;
    }
}

// True in exactly one block: the last of nchunks blocks to finish this launch.
__device__ __forceinline__ bool last_block(unsigned* counter, int nchunks) {
    __shared__ int am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == (unsigned)(nchunks - 1));
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last != 0;
}

// tot[l] = sum over chunks c of part[c * stride + l], l < cnt; fixed order.
template <typename T>
__device__ __forceinline__ void reduce_chunks(const T* part, int nchunks, int stride, int cnt, T* tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = warp; l < cnt; l += SYLV_NWARP) {
        T s = zero<T>();
        for (int c = lane; c < nchunks; c += 32) s += ldcg(part + (size_t)c * stride + l);
        s = warp_sum(s);
        if (lane == 0) tot[l] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double absv(double a) { return fabs(a); }
__device__ __forceinline__ double absv(cplx a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double unit_phase(double a, double aa) { return a / aa; }
__device__ __forceinline__ cplx unit_phase(cplx a, double aa) { return {a.x / aa, a.y / aa}; }

// Givens rotation [[c, s], [-conj(s), c]], c real, mapping (a, b) to (rho, 0).
template <typename T>
__device__ __forceinline__ void givens(T a, T b, double& c, T& s) {
    double aa = absv(a), ab = absv(b);
    if (ab == 0.0) { c = 1.0; s = zero<T>(); return; }
    if (aa == 0.0) { c = 0.0; s = conjg(b) * (1.0 / ab); return; }
    double rho = hypot(aa, ab);
    c = aa / rho;
    s = (unit_phase(a, aa) * conjg(b)) * (1.0 / rho);
}

template <typename T>
__device__ void mark_done(SysState<T>* st, BatchCtl* ctl) {
    st->phase = PH_DONE;
    int old = atomicSub(&ctl->n_active, 1);
    if (old == 1 && ctl->h_flag) {
        *(volatile int*)ctl->h_flag = 0;
        __threadfence_system();
    }
}

// Dispatch on the number of basis vectors j + 1 rounded up to a multiple of
// four, so the unrolled per-row loops issue no more than three predicated-off
// multiply-adds (the float64 pipe of this GPU is the bottleneck of the
// float64 sweeps, and predicated-off instructions still occupy it).
#define SYLV_BUCKET_SWITCH(J, CALL)                      \
    switch (((J) + 4) >> 2) {                            \
        case 1: CALL(4); break;                          \
        case 2: CALL(8); break;                          \
        case 3: CALL(12); break;                         \
        case 4: CALL(16); break;                         \
        case 5: CALL(20); break;                         \
        case 6: CALL(24); break;                         \
        case 7: CALL(28); break;                         \
        default: CALL(32); break;                        \
    }

typedef double RedBufD[SYLV_NWARP][PSTRIDE];

// Per-thread accumulators (type A, NV slots) -> block sums in type T written to
// out[0..cnt); red is a shared buffer of SYLV_NWARP x PSTRIDE T.  The warp
// stage adds in A (float32 for the mixed path: float64 adds run at 1/58 of
// the float32 rate on this GPU); warps and chunks are combined in T.
template <typename T, typename A, int NV>
__device__ __forceinline__ void block_reduce_to(A (&acc)[NV], int cnt, T* out, T (*red)[PSTRIDE]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < NV; ++l) {
        if (l < cnt) {
            const A v = warp_sum(acc[l]);
            if (lane == 0) red[warp][l] = cvt<T>(v);
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
        T s = zero<T>();
#pragma unroll
        for (int w = 0; w < SYLV_NWARP; ++w) s += red[w][l];
        out[l] = s;
    }
}

// Row i of w = (Op + sigma I) P^{-1} (sj * V_j): the pre-scaled stencil
// diagonals in C precision, or the generic operator row in float64.
template <int LAY, typename T, typename S, typename C>
__device__ __forceinline__ C spmv_row(const SysDesc<T, S, C>& sd, const OpDesc& op, const SysState<T>* st,
                                      const S* __restrict__ vj, typename RealOf<C>::type sj, int i) {
    typedef BasisIx<LAY> BI;
    const C* __restrict__ av = sd.aval;
    if (av) {
        C a = zero<C>();
#pragma unroll
        for (int d = 0; d < SYLV_MAXDIAG; ++d) {
            if (d < op.ndiag) {
                const int k = i + op.offs[d];
                if (k >= 0 && k < op.n) a += av[(size_t)d * op.n + i] * cvt<C>(vj[BI::row(sd, k)]);
            }
        }
        return sj * a;
    }
    const T sigma = st->sigma;
    const T* __restrict__ pinv = sd.pinv;
    const T acc64 = op_row<T>(op, i, sigma, [&](int k) {
        const T x = (double)sj * cvt<T>(vj[BI::row(sd, k)]);
        return pinv ? pinv[k] * x : x;
    });
    return cvt<C>(acc64);
}

// Rows [r0, r1) of sweep 1 with NV >= j + 1 accumulators.
template <int NV, int LAY, typename T, typename S, typename C>
__device__ __forceinline__ void spmv_rows(const SysDesc<T, S, C>& sd, const OpDesc& op, const SysState<T>* st,
                                          int j, typename RealOf<C>::type sj, int r0, int r1, int mode,
                                          T* out, T (*red)[PSTRIDE]) {
    typedef BasisIx<LAY> BI;
    // the basis, the work vector and the operator never overlap: tell the
    // compiler, so the loads of the next row can overlap this row's store
    const S* __restrict__ V = sd.V;
    C* __restrict__ w = sd.w;
    const S* __restrict__ vj = V + BI::vec(sd, j);
    C acc[NV];
#pragma unroll
    for (int l = 0; l < NV; ++l) acc[l] = zero<C>();
    if constexpr (SweepOcc<C>::value == 1) {
        // float64: one pass, two rows in flight per thread (bound by the
        // float64 pipe, registers are not the limit)
#pragma unroll 2
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            C wi;
            if (mode == 0) {
                wi = spmv_row<LAY>(sd, op, st, vj, sj, i);
                w[i] = wi;
            } else {
                wi = w[i];
            }
            const S* __restrict__ vr = V + BI::row(sd, i);
#pragma unroll
            for (int l = 0; l < NV; ++l)
                if (l <= j) acc[l] += cmul(cvt<C>(vr[BI::vec(sd, l)]), wi);
        }
    } else {
        // 32-bit sweeps: the product rows first, then the dot products over
        // the same rows (each thread re-reads only the w entries it wrote),
        // so neither loop carries the other's registers and more warps stay
        // resident
        if (mode == 0)
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) w[i] = spmv_row<LAY>(sd, op, st, vj, sj, i);
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const C wi = w[i];
            const S* __restrict__ vr = V + BI::row(sd, i);
#pragma unroll
            for (int l = 0; l < NV; ++l)
                if (l <= j) acc[l] += cmul(cvt<C>(vr[BI::vec(sd, l)]), wi);
        }
    }
    block_reduce_to<T, C, NV>(acc, j + 1, out, red);
}

// ---------------------------------------------------------------------------
// Arnoldi step, sweep 1: w = (Op + sigma I) P^{-1} v_j, partial h1 = V^* w.
// Stencil operators use the pre-scaled diagonals aval = (Op + sigma I) P^{-1}
// (formed once per shift), so the product is ndiag fused multiply-adds.
// mode 1: w is given (a plain CGS2 of w against V), no operator product.
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C, int LAY = 1>
__global__ void __launch_bounds__(SYLV_BLOCK, SweepOcc<C>::value)
k_arnoldi_spmv(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
               const OpDesc* __restrict__ ops, const Item* __restrict__ items, BatchCtl* ctl, int mode) {
    typedef typename RealOf<C>::type CR;
    __shared__ T red[SYLV_NWARP][PSTRIDE];
    count_launch(ctl, K_SPMV);
    // graph-driven solve: no further iteration unless sweep 3 or the restart
    // asks for one
    if (ctl->graph && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(ctl->h_loop, 0u);
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    if (st->phase != PH_ARNOLDI) return;
    const SysDesc<T, S, C> sd = sysd[it.sys];
    const OpDesc op = ops[sd.op];
    const int j = st->j;
    const CR sj = (CR)st->scale[j];
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    count_work(ctl, K_SPMV, it.chunk, mode == 0
        ? (double)op.nnz * sizeof(C) + (double)(j + 2) * sd.n * sizeof(S) + (double)sd.n * sizeof(C)
        : (double)(j + 1) * sd.n * sizeof(S) + (double)sd.n * sizeof(C),
        FmaFlops<C>::v * ((mode == 0 ? (double)op.nnz : 0.0) + (double)(j + 1) * sd.n));
    T* out = sd.part + (size_t)it.chunk * PSTRIDE;
#define SYLV_SPMV_CALL(NV) spmv_rows<NV, LAY, T, S, C>(sd, op, st, j, sj, r0, r1, mode, out, red)
    SYLV_BUCKET_SWITCH(j, SYLV_SPMV_CALL)
#undef SYLV_SPMV_CALL
    if (!last_block(&st->counter, sd.nchunks)) return;
    __shared__ T tot[PSTRIDE];
    reduce_chunks(sd.part, sd.nchunks, PSTRIDE, j + 1, tot);
    for (int l = threadIdx.x; l <= j; l += blockDim.x) st->h1[l] = st->scale[l] * tot[l];
    if (threadIdx.x == 0) st->counter = 0;
}

// Rows [r0, r1) of sweep 2 with NV >= j + 1 accumulators.
template <int NV, int LAY, typename T, typename S, typename C>
__device__ __forceinline__ void pass2_rows(const SysDesc<T, S, C>& sd, const C* cc, int j, int r0, int r1,
                                           T* out, T (*red)[PSTRIDE]) {
    typedef BasisIx<LAY> BI;
    const S* __restrict__ V = sd.V;
    const C* __restrict__ w = sd.w;
    C acc[NV];
#pragma unroll
    for (int l = 0; l < NV; ++l) acc[l] = zero<C>();
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        C w1 = w[i];
        const S* __restrict__ vr = V + BI::row(sd, i);
#pragma unroll
        for (int l = 0; l < NV; ++l)
            if (l <= j) w1 -= cc[l] * cvt<C>(vr[BI::vec(sd, l)]);
#pragma unroll
        for (int l = 0; l < NV; ++l)
            if (l <= j) acc[l] += cmul(cvt<C>(vr[BI::vec(sd, l)]), w1);
    }
    block_reduce_to<T, C, NV>(acc, j + 1, out, red);
}

// ---------------------------------------------------------------------------
// Sweep 2: h2 = V^* (w - V h1).  The row of V is read twice; the second read
// hits L1 (or registers).
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C, int LAY = 1>
__global__ void __launch_bounds__(SYLV_BLOCK, SweepOcc<C>::value)
k_cgs_pass2(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
            const Item* __restrict__ items, BatchCtl* ctl) {
    __shared__ T red[SYLV_NWARP][PSTRIDE];
    count_launch(ctl, K_CGS2);
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    if (st->phase != PH_ARNOLDI) return;
    const SysDesc<T, S, C> sd = sysd[it.sys];
    const int j = st->j;
    __shared__ C cc[SYLV_MAXV + 1];
    for (int l = threadIdx.x; l <= j; l += blockDim.x) cc[l] = cvt<C>(st->h1[l] * st->scale[l]);
    count_work(ctl, K_CGS2, it.chunk, (double)(j + 1) * sd.n * sizeof(S) + (double)sd.n * sizeof(C),
               FmaFlops<C>::v * 2.0 * (j + 1) * sd.n);
    __syncthreads();
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    T* out = sd.part + (size_t)it.chunk * PSTRIDE;
#define SYLV_PASS2_CALL(NV) pass2_rows<NV, LAY, T, S, C>(sd, cc, j, r0, r1, out, red)
    SYLV_BUCKET_SWITCH(j, SYLV_PASS2_CALL)
#undef SYLV_PASS2_CALL
    if (!last_block(&st->counter, sd.nchunks)) return;
    __shared__ T tot[PSTRIDE];
    reduce_chunks(sd.part, sd.nchunks, PSTRIDE, j + 1, tot);
    for (int l = threadIdx.x; l <= j; l += blockDim.x) st->h2[l] = st->scale[l] * tot[l];
    if (threadIdx.x == 0) st->counter = 0;
}

// Last block of sweep 3: Hessenberg column j, Givens update, stop test, and
// at the end of a cycle the least-squares solution by back substitution.
// The block stages the rotations and R in shared memory; one warp runs the
// sequential parts.
template <typename T>
__device__ void arnoldi_finish(int restart, double* hist, int hist_cap, SysState<T>* st, double nrm2) {
    __shared__ T s_col[SYLV_MAXV];
    __shared__ T s_sn[SYLV_MR];
    __shared__ double s_cs[SYLV_MR];
    __shared__ T s_R[SYLV_MR * SYLV_MAXV];
    __shared__ T s_g[SYLV_MAXV];
    __shared__ int s_end;
    const int j = st->j;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        s_col[i] = st->h1[i] + st->h2[i];
        s_g[i] = st->g[i];
        if (i < j) { s_cs[i] = st->cs[i]; s_sn[i] = st->sn[i]; }
    }
    // R columns 0..j-1 (needed only when the cycle ends; loaded in parallel)
    for (int q = threadIdx.x; q < j * SYLV_MAXV; q += blockDim.x) s_R[q] = st->R[q];
    __syncthreads();
    const double hn = sqrt(nrm2);
    if (threadIdx.x == 0) {
        T col[SYLV_MAXV];
        for (int i = 0; i <= j; ++i) col[i] = s_col[i];
        col[j + 1] = make_scalar<T>(hn, 0.0);
        st->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
        for (int i = 0; i < j; ++i) {
            const double c = s_cs[i];
            const T s = s_sn[i];
            const T t0 = c * col[i] + s * col[i + 1];
            const T t1 = c * col[i + 1] - conjg(s) * col[i];
            col[i] = t0;
            col[i + 1] = t1;
        }
        double c;
        T s;
        givens(col[j], col[j + 1], c, s);
        st->cs[j] = c;
        st->sn[j] = s;
        col[j] = c * col[j] + s * col[j + 1];
        const T gj = s_g[j];
        const T gj1 = -(conjg(s) * gj);
        st->g[j + 1] = gj1;
        st->g[j] = c * gj;
        s_g[j] = c * gj;
        for (int i = 0; i <= j; ++i) {
            st->R[j * SYLV_MAXV + i] = col[i];
            s_R[j * SYLV_MAXV + i] = col[i];
        }
        const double est = absv(gj1);
        st->est = est;
        st->iters += 1;
        if (hist && st->iters - 1 < hist_cap) hist[st->iters - 1] = est;
        int end;
        if (!isfinite(est) || !isfinite(hn)) {
            st->status = ST_NONFINITE;
            st->nvec = 0;
            st->phase = PH_UPDATE;
            end = 0;
        } else if (est <= st->tol || j + 1 >= restart || st->iters >= st->max_iters) {
            st->nvec = j + 1;
            end = 1;
        } else {
            st->j = j + 1;
            end = 0;
        }
        s_end = end;
    }
    __syncthreads();
    if (!s_end || threadIdx.x >= 32) return;
    // back substitution R y = g by columns, one warp: lane l owns g[l]
    const int k = j + 1;
    const int lane = threadIdx.x;
    T gl = lane < k ? s_g[lane] : zero<T>();
    T yl = zero<T>();
    for (int i = k - 1; i >= 0; --i) {
        const T num = shfl_idx(gl, i);                   // g_i, already updated
        const T rii = s_R[i * SYLV_MAXV + i];
        const T yi = (absv(rii) != 0.0) ? sdiv(num, rii) : zero<T>();
        if (lane == i) yl = yi;
        if (lane < i) gl -= s_R[i * SYLV_MAXV + lane] * yi;
    }
    if (lane < k) st->y[lane] = st->scale[lane] * yl;
    __syncwarp();
    if (lane == 0) st->phase = PH_UPDATE;
}

// ---------------------------------------------------------------------------
// Sweep 3: v_{j+1} = w - V (h1 + h2), ||v_{j+1}||^2; finish the Arnoldi step.
// The norm is taken of the stored (rounded) vector.
// mode 1 (plain CGS2): store the unrotated column and stop the system.
// ---------------------------------------------------------------------------
// Grid-level decision of a device iteration when a CUDA graph drives the
// solve: the last block of the launch scans the systems' phases and sets the
// conditional nodes - whether the restart kernels run in this iteration
// (after sweep 3) and whether another iteration follows.  A cap on the
// iterations of one inner loop ends it in every case (remaining systems are
// reported as stalled), so the loop always terminates.
template <typename T>
__device__ void graph_tail(BatchCtl* ctl, SysState<T>* sts, int kid) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = ((atomicAdd(&ctl->gdone[kid], 1u) + 1u) % gridDim.x) == 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    int pend = 0, act = 0;
    for (int q = threadIdx.x; q < ctl->nsys; q += blockDim.x) {
        const int ph = *(volatile const int*)&sts[q].phase;
        pend |= (ph == PH_UPDATE || ph == PH_RESID);
        act |= (ph != PH_DONE);
    }
    pend = __syncthreads_or(pend);
    act = __syncthreads_or(act);
    // a batch goes on while an instance still has an outer step to take
    act |= (*(volatile int*)&ctl->n_inst_open > 0);
    if (threadIdx.x != 0) return;
    if (kid == K_CGS3) {
        const int t = ++ctl->ticks;
        if (act && t >= ctl->max_ticks) {
            for (int q = 0; q < ctl->nsys; ++q)
                if (sts[q].phase != PH_DONE) { sts[q].status = ST_STALL; sts[q].phase = PH_DONE; }
            ctl->capped += 1;
            ctl->n_active = 0;
            cudaGraphSetConditional(ctl->h_restart, 0u);
            cudaGraphSetConditional(ctl->h_loop, 0u);
            return;
        }
        cudaGraphSetConditional(ctl->h_restart, pend ? 1u : 0u);
        if (!pend) cudaGraphSetConditional(ctl->h_loop, act ? 1u : 0u);
    } else {
        cudaGraphSetConditional(ctl->h_loop, act ? 1u : 0u);
    }
}

template <typename T, typename S, typename C, int LAY>
__device__ __forceinline__ void cgs_pass3_body(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
                                               const Item* __restrict__ items, BatchCtl* ctl, int mode) {
    typedef typename RealOf<C>::type CR;
    count_launch(ctl, K_CGS3);
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    if (st->phase != PH_ARNOLDI) return;
    const SysDesc<T, S, C> sd = sysd[it.sys];
    const int j = st->j;
    __shared__ C cc[SYLV_MAXV + 1];
    for (int l = threadIdx.x; l <= j; l += blockDim.x) cc[l] = cvt<C>((st->h1[l] + st->h2[l]) * st->scale[l]);
    count_work(ctl, K_CGS3, it.chunk, (double)(j + 2) * sd.n * sizeof(S) + (double)sd.n * sizeof(C),
               FmaFlops<C>::v * (double)(j + 2) * sd.n);
    __syncthreads();
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    // vectors 0..j are read, vector j+1 is written: disjoint ranges
    typedef BasisIx<LAY> BI;
    const S* __restrict__ V = sd.V;
    const C* __restrict__ w = sd.w;
    S* __restrict__ vn = sd.V + BI::vec(sd, j + 1);
    CR acc[1] = {(CR)0};
#define SYLV_PASS3_CALL(NV)                                                   \
    _Pragma("unroll 2") for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) { \
        C x = w[i];                                                           \
        const size_t ri = BI::row(sd, i);                                     \
        _Pragma("unroll") for (int l = 0; l < NV; ++l)                        \
            if (l <= j) x -= cc[l] * cvt<C>(V[ri + BI::vec(sd, l)]);          \
        const S xs = cvt<S>(x);                                               \
        vn[ri] = xs;                                                          \
        acc[0] += abs2(cvt<C>(xs));                                           \
    }
    SYLV_BUCKET_SWITCH(j, SYLV_PASS3_CALL)
#undef SYLV_PASS3_CALL
    block_reduce_store<double, CR, 1>(acc, 1, reinterpret_cast<double*>(sd.part + (size_t)it.chunk * PSTRIDE));
    if (!last_block(&st->counter, sd.nchunks)) return;
    __shared__ double tot[1];
    reduce_chunks(reinterpret_cast<const double*>(sd.part), sd.nchunks, PSTRIDE * (int)(sizeof(T) / sizeof(double)), 1, tot);
    if (threadIdx.x == 0) {
        st->counter = 0;
        st->nrm2 = tot[0];
    }
    if (mode == 1) {
        if (threadIdx.x == 0) {
            const double hn = sqrt(tot[0]);
            for (int i = 0; i <= j; ++i) st->R[j * SYLV_MAXV + i] = st->h1[i] + st->h2[i];
            st->R[j * SYLV_MAXV + j + 1] = make_scalar<T>(hn, 0.0);
            st->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
            mark_done(st, ctl);
        }
    } else {
        arnoldi_finish<T>(sd.restart, sd.hist, sd.hist_cap, st, tot[0]);
    }
}

template <typename T, typename S, typename C, int LAY = 1>
__global__ void __launch_bounds__(SYLV_BLOCK, SweepOcc<C>::value)
k_cgs_pass3(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
            const Item* __restrict__ items, BatchCtl* ctl, int mode) {
    cgs_pass3_body<T, S, C, LAY>(sysd, sts, items, ctl, mode);
    if (ctl->graph) graph_tail<T>(ctl, sts, K_CGS3);
}

// ---------------------------------------------------------------------------
// Restart, part 1: x += P^{-1} sum_l y_l V_l  (y already carries the scales).
// The combination is formed in the sweep precision C, the update in float64.
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_restart_update(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
                 const Item* __restrict__ items, BatchCtl* ctl) {
    count_launch(ctl, K_RUPD);
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    if (st->phase != PH_UPDATE) return;
    const SysDesc<T, S, C> sd = sysd[it.sys];
    const int k = st->nvec;
    if (k == 0) return;
    __shared__ C cc[32];
    for (int l = threadIdx.x; l < k; l += blockDim.x) cc[l] = cvt<C>(st->y[l]);
    count_work(ctl, K_RUPD, it.chunk, (double)k * sd.n * sizeof(S) + 2.0 * sd.n * sizeof(T),
               FmaFlops<C>::v * (double)(k + 1) * sd.n);
    __syncthreads();
    T* __restrict__ x = st->x;
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
#define SYLV_RUPD_CALL(NV)                                                    \
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {                 \
        C s = zero<C>();                                                      \
        _Pragma("unroll") for (int l = 0; l < NV; ++l)                        \
            if (l < k) s += cc[l] * cvt<C>(sd.V[BasisIx<1>::row(sd, i) + 32 * l]); \
        const T s64 = cvt<T>(s);                                              \
        x[i] += sd.pinv ? sd.pinv[i] * s64 : s64;                             \
    }
    SYLV_BUCKET_SWITCH(k - 1, SYLV_RUPD_CALL)
#undef SYLV_RUPD_CALL
}

// ---------------------------------------------------------------------------
// Restart, part 2: r = b - (Op + sigma I) x (float64), V_0 = r, ||r||, then
// the decision: converged / iteration cap / non-finite -> done, else a new
// cycle with v_0 = r / ||r||.
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
__device__ __forceinline__ void restart_residual_body(const SysDesc<T, S, C>* __restrict__ sysd,
                                                      SysState<T>* __restrict__ sts,
                                                      const OpDesc* __restrict__ ops,
                                                      const Item* __restrict__ items, BatchCtl* ctl) {
    count_launch(ctl, K_RRES);
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    const int ph = st->phase;
    if (ph != PH_UPDATE && ph != PH_RESID) return;
    const SysDesc<T, S, C> sd = sysd[it.sys];
    const OpDesc op = ops[sd.op];
    const T sigma = st->sigma;
    const T* __restrict__ x = st->x;
    const T* __restrict__ b = st->b;
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    count_work(ctl, K_RRES, it.chunk,
               (double)op.nnz * sizeof(double) + 2.0 * sd.n * sizeof(T) + (double)sd.n * sizeof(S),
               FmaFlops<T>::v * ((double)op.nnz + 2.0 * sd.n));
    double acc[1] = {0.0};
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const T ax = op_row<T>(op, i, sigma, [&](int k) { return x[k]; });
        const T r = b[i] - ax;
        sd.V[BasisIx<1>::row(sd, i)] = cvt<S>(r);
        acc[0] += abs2(r);
    }
    block_reduce_store<double, double, 1>(acc, 1, reinterpret_cast<double*>(sd.part + (size_t)it.chunk * PSTRIDE));
    if (!last_block(&st->counter, sd.nchunks)) return;
    __shared__ double tot[1];
    reduce_chunks(reinterpret_cast<const double*>(sd.part), sd.nchunks, PSTRIDE * (int)(sizeof(T) / sizeof(double)), 1, tot);
    if (threadIdx.x == 0) {
        st->counter = 0;
        const double rn = sqrt(tot[0]);
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
            st->j = 0;
            st->g[0] = make_scalar<T>(rn, 0.0);
            for (int l = 1; l < SYLV_MAXV; ++l) st->g[l] = zero<T>();
            st->scale[0] = 1.0 / rn;
            st->phase = PH_ARNOLDI;
        }
    }
}

template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_restart_residual(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
                   const OpDesc* __restrict__ ops, const Item* __restrict__ items, BatchCtl* ctl) {
    restart_residual_body<T, S, C>(sysd, sts, ops, items, ctl);
    if (ctl->graph) graph_tail<T>(ctl, sts, K_RRES);
}

// x = 0 over the rows of every system (start of a solve).
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_zero_x(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts, const Item* __restrict__ items) {
    const Item it = items[blockIdx.x];
    const SysDesc<T, S, C> sd = sysd[it.sys];
    T* x = sts[it.sys].x;
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) x[i] = zero<T>();
}

// Shift-dependent operator data for rows [r0, r1): pinv = 1 / (diag + sigma)
// (Jacobi, optional) and, for stencil operators with a stored main diagonal,
// the pre-scaled diagonals aval[d][i] = ((Op + sigma I) P^{-1})[i][i + off_d]
// in the sweep precision C.
template <typename T, typename C>
__device__ __forceinline__ void shifted_op_rows(const OpDesc& op, T sigma, T* pinv, C* aval, int r0, int r1) {
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        if (pinv) pinv[i] = sdiv(make_scalar<T>(1.0, 0.0), op.diag[i] + sigma);
        if (!aval) continue;
        for (int d = 0; d < op.ndiag; ++d) {
            const int k = i + op.offs[d];
            T a = zero<T>();
            if (k >= 0 && k < op.n) {
                a = make_scalar<T>(op.dval[(size_t)d * op.n + i], 0.0);
                if (op.offs[d] == 0) a = a + sigma;
                if (pinv) a = a * sdiv(make_scalar<T>(1.0, 0.0), op.diag[k] + sigma);
            }
            aval[(size_t)d * op.n + i] = cvt<C>(a);
        }
    }
}

template <typename T, typename C>
__global__ void k_shifted_op(OpDesc op, T sigma, T* pinv, C* aval) {
    const int rows = (op.n + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * rows, r1 = min(op.n, r0 + rows);
    shifted_op_rows<T, C>(op, sigma, pinv, aval, r0, r1);
}

}  // namespace sylv
