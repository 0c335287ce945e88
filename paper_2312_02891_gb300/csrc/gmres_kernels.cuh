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
// scale factor, so no separate normalisation sweep is needed.
#pragma once
#include "common.cuh"

namespace sylv {

constexpr int PSTRIDE = SYLV_MAXV + 1;     // partial-sum slots per chunk

template <typename T, int NV>
__device__ __forceinline__ void block_reduce_store(T (&acc)[NV], int cnt, T* out) {
    __shared__ T red[SYLV_NWARP][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < NV; ++l) {
        if (l < cnt) {
            T v = warp_sum(acc[l]);
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
__device__ __forceinline__ bool finite_s(double a) { return isfinite(a); }
__device__ __forceinline__ bool finite_s(cplx a) { return isfinite(a.x) && isfinite(a.y); }

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

// ---------------------------------------------------------------------------
// Arnoldi step, sweep 1: w = (Op + sigma I) P^{-1} v_j, partial h1 = V^* w.
// mode 1: w is given (a plain CGS2 of w against V), no operator product.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_arnoldi_spmv(const SysDesc<T>* __restrict__ sysd, SysState<T>* __restrict__ sts,
               const OpDesc* __restrict__ ops, const Item* __restrict__ items, int mode) {
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    if (st->phase != PH_ARNOLDI) return;
    const SysDesc<T> sd = sysd[it.sys];
    const OpDesc op = ops[sd.op];
    const int j = st->j;
    const double sj = st->scale[j];
    const T sigma = st->sigma;
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    const T* __restrict__ vj = sd.V + (size_t)j * sd.ldv;
    const T* __restrict__ pinv = sd.pinv;
    T acc[SYLV_MAXV];
#pragma unroll
    for (int l = 0; l < SYLV_MAXV; ++l) acc[l] = zero<T>();
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        T wi;
        if (mode == 0) {
            if (pinv) wi = op_row<T>(op, i, sigma, [&](int k) { return (sj * pinv[k]) * vj[k]; });
            else      wi = op_row<T>(op, i, sigma, [&](int k) { return sj * vj[k]; });
            sd.w[i] = wi;
        } else {
            wi = sd.w[i];
        }
#pragma unroll
        for (int l = 0; l < SYLV_MAXV; ++l)
            if (l <= j) acc[l] += cmul(sd.V[(size_t)l * sd.ldv + i], wi);
    }
    block_reduce_store<T, SYLV_MAXV>(acc, j + 1, sd.part + (size_t)it.chunk * PSTRIDE);
    if (!last_block(&st->counter, sd.nchunks)) return;
    __shared__ T tot[PSTRIDE];
    reduce_chunks(sd.part, sd.nchunks, PSTRIDE, j + 1, tot);
    for (int l = threadIdx.x; l <= j; l += blockDim.x) st->h1[l] = st->scale[l] * tot[l];
    if (threadIdx.x == 0) st->counter = 0;
}

// ---------------------------------------------------------------------------
// Sweep 2: h2 = V^* (w - V h1).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_cgs_pass2(const SysDesc<T>* __restrict__ sysd, SysState<T>* __restrict__ sts,
            const Item* __restrict__ items) {
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    if (st->phase != PH_ARNOLDI) return;
    const SysDesc<T> sd = sysd[it.sys];
    const int j = st->j;
    __shared__ T cc[SYLV_MAXV];
    for (int l = threadIdx.x; l <= j; l += blockDim.x) cc[l] = st->h1[l] * st->scale[l];
    __syncthreads();
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    T acc[SYLV_MAXV];
#pragma unroll
    for (int l = 0; l < SYLV_MAXV; ++l) acc[l] = zero<T>();
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        if constexpr (sizeof(T) == sizeof(double)) {
            // real: keep the row of V in registers between the two uses
            T v[SYLV_MAXV];
#pragma unroll
            for (int l = 0; l < SYLV_MAXV; ++l)
                v[l] = (l <= j) ? sd.V[(size_t)l * sd.ldv + i] : zero<T>();
            T w1 = sd.w[i];
#pragma unroll
            for (int l = 0; l < SYLV_MAXV; ++l)
                if (l <= j) w1 -= cc[l] * v[l];
#pragma unroll
            for (int l = 0; l < SYLV_MAXV; ++l)
                if (l <= j) acc[l] += cmul(v[l], w1);
        } else {
            // complex: the second use re-reads the row (an L1 hit) to stay in registers
            T w1 = sd.w[i];
#pragma unroll
            for (int l = 0; l < SYLV_MAXV; ++l)
                if (l <= j) w1 -= cc[l] * sd.V[(size_t)l * sd.ldv + i];
#pragma unroll
            for (int l = 0; l < SYLV_MAXV; ++l)
                if (l <= j) acc[l] += cmul(sd.V[(size_t)l * sd.ldv + i], w1);
        }
    }
    block_reduce_store<T, SYLV_MAXV>(acc, j + 1, sd.part + (size_t)it.chunk * PSTRIDE);
    if (!last_block(&st->counter, sd.nchunks)) return;
    __shared__ T tot[PSTRIDE];
    reduce_chunks(sd.part, sd.nchunks, PSTRIDE, j + 1, tot);
    for (int l = threadIdx.x; l <= j; l += blockDim.x) st->h2[l] = st->scale[l] * tot[l];
    if (threadIdx.x == 0) st->counter = 0;
}

// Thread 0 of the last block: Hessenberg column j, Givens update, stop test.
template <typename T>
__device__ void arnoldi_finish(const SysDesc<T>& sd, SysState<T>* st, double nrm2) {
    const int j = st->j;
    const double hn = sqrt(nrm2);
    T col[SYLV_MAXV];
    for (int i = 0; i <= j; ++i) col[i] = st->h1[i] + st->h2[i];
    col[j + 1] = make_scalar<T>(hn, 0.0);
    st->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; ++i) {
        const double c = st->cs[i];
        const T s = st->sn[i];
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
    col[j + 1] = zero<T>();
    const T gj = st->g[j];
    st->g[j + 1] = -(conjg(s) * gj);
    st->g[j] = c * gj;
    for (int i = 0; i <= j; ++i) st->R[j * SYLV_MAXV + i] = col[i];
    const double est = absv(st->g[j + 1]);
    st->est = est;
    st->iters += 1;
    if (sd.hist && st->iters - 1 < sd.hist_cap) sd.hist[st->iters - 1] = est;
    if (!isfinite(est) || !isfinite(hn)) {
        st->status = ST_NONFINITE;
        st->nvec = 0;
        st->phase = PH_UPDATE;
        return;
    }
    if (est <= st->tol || j + 1 >= sd.restart || st->iters >= st->max_iters) {
        const int k = j + 1;
        T y[SYLV_MR];
        for (int i = k - 1; i >= 0; --i) {
            T acc = st->g[i];
            for (int l = i + 1; l < k; ++l) acc -= st->R[l * SYLV_MAXV + i] * y[l];
            const T rii = st->R[i * SYLV_MAXV + i];
            y[i] = (absv(rii) != 0.0) ? sdiv(acc, rii) : zero<T>();
        }
        for (int l = 0; l < k; ++l) st->y[l] = st->scale[l] * y[l];
        st->nvec = k;
        st->phase = PH_UPDATE;
    } else {
        st->j = j + 1;
    }
}

// ---------------------------------------------------------------------------
// Sweep 3: v_{j+1} = w - V (h1 + h2), ||v_{j+1}||^2; finish the Arnoldi step.
// mode 1 (plain CGS2): store the unrotated column and stop the system.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_cgs_pass3(const SysDesc<T>* __restrict__ sysd, SysState<T>* __restrict__ sts,
            const Item* __restrict__ items, BatchCtl* ctl, int mode) {
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    if (st->phase != PH_ARNOLDI) return;
    const SysDesc<T> sd = sysd[it.sys];
    const int j = st->j;
    __shared__ T cc[SYLV_MAXV];
    for (int l = threadIdx.x; l <= j; l += blockDim.x) cc[l] = (st->h1[l] + st->h2[l]) * st->scale[l];
    __syncthreads();
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    T* __restrict__ vn = sd.V + (size_t)(j + 1) * sd.ldv;
    double acc[1] = {0.0};
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        T x = sd.w[i];
#pragma unroll
        for (int l = 0; l < SYLV_MAXV; ++l)
            if (l <= j) x -= cc[l] * sd.V[(size_t)l * sd.ldv + i];
        vn[i] = x;
        acc[0] += abs2(x);
    }
    block_reduce_store<double, 1>(acc, 1, reinterpret_cast<double*>(sd.part + (size_t)it.chunk * PSTRIDE));
    if (!last_block(&st->counter, sd.nchunks)) return;
    __shared__ double tot[1];
    reduce_chunks(reinterpret_cast<const double*>(sd.part), sd.nchunks, PSTRIDE * (int)(sizeof(T) / sizeof(double)), 1, tot);
    if (threadIdx.x == 0) {
        st->counter = 0;
        st->nrm2 = tot[0];
        if (mode == 1) {
            const double hn = sqrt(tot[0]);
            for (int i = 0; i <= j; ++i) st->R[j * SYLV_MAXV + i] = st->h1[i] + st->h2[i];
            st->R[j * SYLV_MAXV + j + 1] = make_scalar<T>(hn, 0.0);
            st->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
            mark_done(st, ctl);
        } else {
            arnoldi_finish(sd, st, tot[0]);
        }
    }
}

// ---------------------------------------------------------------------------
// Restart, part 1: x += P^{-1} sum_l y_l V_l  (y already carries the scales).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_restart_update(const SysDesc<T>* __restrict__ sysd, SysState<T>* __restrict__ sts,
                 const Item* __restrict__ items) {
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    if (st->phase != PH_UPDATE) return;
    const SysDesc<T> sd = sysd[it.sys];
    const int k = st->nvec;
    if (k == 0) return;
    __shared__ T cc[SYLV_MR];
    for (int l = threadIdx.x; l < k; l += blockDim.x) cc[l] = st->y[l];
    __syncthreads();
    T* __restrict__ x = st->x;
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        T s = zero<T>();
#pragma unroll
        for (int l = 0; l < SYLV_MR; ++l)
            if (l < k) s += cc[l] * sd.V[(size_t)l * sd.ldv + i];
        x[i] += sd.pinv ? sd.pinv[i] * s : s;
    }
}

// ---------------------------------------------------------------------------
// Restart, part 2: r = b - (Op + sigma I) x (float64), V_0 = r, ||r||, then
// the decision: converged / iteration cap / non-finite -> done, else a new
// cycle with v_0 = r / ||r||.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_restart_residual(const SysDesc<T>* __restrict__ sysd, SysState<T>* __restrict__ sts,
                   const OpDesc* __restrict__ ops, const Item* __restrict__ items, BatchCtl* ctl) {
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    const int ph = st->phase;
    if (ph != PH_UPDATE && ph != PH_RESID) return;
    const SysDesc<T> sd = sysd[it.sys];
    const OpDesc op = ops[sd.op];
    const T sigma = st->sigma;
    const T* __restrict__ x = st->x;
    const T* __restrict__ b = st->b;
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    double acc[1] = {0.0};
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const T ax = op_row<T>(op, i, sigma, [&](int k) { return x[k]; });
        const T r = b[i] - ax;
        sd.V[i] = r;
        acc[0] += abs2(r);
    }
    block_reduce_store<double, 1>(acc, 1, reinterpret_cast<double*>(sd.part + (size_t)it.chunk * PSTRIDE));
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

// x = 0 over the rows of every system (start of a solve).
template <typename T>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_zero_x(const SysDesc<T>* __restrict__ sysd, SysState<T>* __restrict__ sts, const Item* __restrict__ items) {
    const Item it = items[blockIdx.x];
    const SysDesc<T> sd = sysd[it.sys];
    T* x = sts[it.sys].x;
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) x[i] = zero<T>();
}

// pinv[i] = 1 / (diag[i] + sigma)  (right Jacobi preconditioner).
template <typename T>
__global__ void k_pinv(const double* __restrict__ diag, T sigma, T* __restrict__ pinv, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        pinv[i] = sdiv(make_scalar<T>(1.0, 0.0), diag[i] + sigma);
}

}  // namespace sylv
