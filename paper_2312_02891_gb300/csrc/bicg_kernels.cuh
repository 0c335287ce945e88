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

// ---------------------------------------------------------------------------
// Shared-memory staging of a work item for the stencil product.  The product
// at the rows [r0, r1) reads its input vectors at the rows [r0 - H, r1 + H)
// (H = the largest |offset| of the stored diagonals), its stencil values and
// (kernel a) the shadow vector at [r0, r1).  Each contiguous range is one TMA
// bulk copy (cp.async.bulk) into shared memory, all issued at the start of
// the block and completing on one mbarrier, so a block has its whole input in
// flight at once instead of one row per thread.  Ranges are widened to
// 16-byte boundaries (vectors are 32-row aligned); the unaligned ends of the
// stencil rows are loaded by the threads.  Used when the item fits the
// launch's dynamic shared memory, otherwise the kernels read global memory
// directly.
// ---------------------------------------------------------------------------
// Dynamic shared memory a staged work item may take: two blocks per SM.
#define SYLV_BICG_SMEM_CAP (108 * 1024)
template <typename C> struct StageElems { static constexpr int value = sizeof(C) >= 16 ? 1 : 16 / (int)sizeof(C); };
template <typename C> HD int stage_ls(int rpc, int halo) {
    constexpr int e = StageElems<C>::value;
    return (rpc + 2 * halo + 2 * e + e - 1) / e * e;
}
template <typename C> HD int stage_ds(int rpc) {
    constexpr int e = StageElems<C>::value;
    return (rpc + 2 * e + e - 1) / e * e;
}
template <typename C> HD int stage_hs(int rpc) {
    constexpr int e = StageElems<C>::value;
    return (rpc + e - 1) / e * e;
}
// Bytes of a staged item: the barrier, nvec neighbour-vector slots and nown
// own-row slots per active column, one slot per stored diagonal.
template <typename C> HD size_t stage_bytes(int rpc, int halo, int ndiag, int na, int nvec, int nown) {
    return 16 + ((size_t)nvec * na * stage_ls<C>(rpc, halo) + (size_t)ndiag * stage_ds<C>(rpc) +
                 (size_t)nown * na * stage_hs<C>(rpc)) * sizeof(C);
}
HD int op_halo_of(const int* offs, int ndiag) {
    int h = 0;
    for (int d = 0; d < ndiag; ++d) h = offs[d] < 0 ? (-offs[d] > h ? -offs[d] : h) : (offs[d] > h ? offs[d] : h);
    return h;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned dyn_smem_bytes() {
    unsigned v;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the staged copies; gives up after a bounded number of polls
// (every thread of the block agrees on the outcome).  On failure the fault is
// recorded for the host and the caller poisons its partial sums, so the
// columns end as non-finite instead of the kernel waiting forever.
__device__ __forceinline__ bool stage_wait(unsigned long long* bar, BatchCtl* ctl) {
    bool ok = true;
    for (unsigned it = 0; !mbar_try_wait(bar, 0u); ++it)
        if (it > (1u << 22)) { ok = false; break; }
    ok = __syncthreads_and(ok);
    if (!ok && threadIdx.x == 0) atomicExch(&ctl->stage_fault, 1);
    return ok;
}

// Issues the staging of one work item (slot layout: NV neighbour vectors x na
// active columns of ls elements, ndiag stencil slots of ds, NOWN own-row
// vector x na of hs).  lo is the first staged neighbour row.
template <typename T, typename S, typename C, int NV, int NOWN>
__device__ __forceinline__ void bicg_stage_issue(const SysDesc<T, S, C>& sd, const OpDesc& op, int mask, int r0,
                                                 int r1, int lo, int hi, const int (&vids)[NV], int own_vid, int ls,
                                                 int ds, int hs, unsigned char* smem) {
    constexpr int E = StageElems<C>::value;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem);
    C* sv = reinterpret_cast<C*>(smem + 16);
    const int na = __popc(mask);
    C* sD = sv + (size_t)NV * na * ls;
    C* sH = sD + (size_t)op.ndiag * ds;
    const size_t ld = sd.ldv;
    const size_t cs = (size_t)BV_COUNT * ld;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        // copy lane: neighbour vectors (NV * na), stencil rows (ndiag), own rows (NOWN * na)
        const void* src = nullptr;
        void* dst = nullptr;
        unsigned bytes = 0;
        if (lane < NV * na) {
            const int v = lane / na, j = lane % na;
            int q = 0, c = -1;
            for (; q < BG_MAXCOL; ++q)
                if ((mask >> q & 1) && ++c == j) break;
            src = sd.bv + q * cs + (size_t)vids[v] * ld + lo;
            dst = sv + ((size_t)v * na + j) * ls;
            bytes = (unsigned)((hi - lo) * sizeof(C));
        } else if (lane < NV * na + op.ndiag) {
            const int d = lane - NV * na;
            const size_t g0 = (size_t)d * op.n + r0, base = g0 - g0 % E;
            const size_t a = (g0 + E - 1) / E * E, b = (g0 + (r1 - r0)) / E * E;
            if (b > a) {
                src = sd.aval + a;
                dst = sD + (size_t)d * ds + (a - base);
                bytes = (unsigned)((b - a) * sizeof(C));
            }
        } else if (lane < NV * na + op.ndiag + NOWN * na) {
            const int j = lane - NV * na - op.ndiag;
            int q = 0, c = -1;
            for (; q < BG_MAXCOL; ++q)
                if ((mask >> q & 1) && ++c == j) break;
            src = sd.bv + q * cs + (size_t)own_vid * ld + r0;
            dst = sH + (size_t)j * hs;
            bytes = (unsigned)(((r1 + E - 1) / E * E - r0) * sizeof(C));
        }
        const unsigned total = __reduce_add_sync(0xffffffffu, bytes);
        if (lane == 0) mbar_expect_tx(bar, total);
        __syncwarp();
        if (bytes) bulk_to_smem(dst, src, bytes, bar);
    }
    // unaligned ends of the stencil rows: plain loads
    for (int t = threadIdx.x; t < op.ndiag * 2 * E; t += blockDim.x) {
        const int d = t / (2 * E), u = t % (2 * E);
        const size_t g0 = (size_t)d * op.n + r0, base = g0 - g0 % E, gend = g0 + (r1 - r0);
        const size_t a = (g0 + E - 1) / E * E, b = gend / E * E;
        size_t gi;
        if (b > a) gi = u < E ? g0 + u : b + (u - E);
        else gi = g0 + u;
        const bool in = b > a ? (u < E ? gi < a : gi < gend) : gi < gend;
        if (in) sD[(size_t)d * ds + (gi - base)] = ldro(sd.aval + gi);
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
    const int rpc = sd.rows_per_chunk;
    const int halo = op_halo_of(op.offs, op.ndiag);
    if (sd.aval && stage_bytes<C>(rpc, halo, op.ndiag, na, 2, 1) <= dyn_smem_bytes()) {
        // staged: r, q at [lo, hi), the stencil rows and rhat in shared memory
        extern __shared__ __align__(16) unsigned char bsm[];
        constexpr int E = StageElems<C>::value;
        const int ls = stage_ls<C>(rpc, halo), ds = stage_ds<C>(rpc), hs = stage_hs<C>(rpc);
        const int lo = max(0, r0 - halo) / E * E;
        const int hi = (int)min((size_t)ld, (size_t)((min(sd.n, r1 + halo) + E - 1) / E * E));
        const int vids[2] = {BV_R, BV_Q};
        bicg_stage_issue<T, S, C, 2, 1>(sd, op, mask, r0, r1, lo, hi, vids, BV_RH, ls, ds, hs, bsm);
        const bool ok = stage_wait(reinterpret_cast<unsigned long long*>(bsm), ctl);
        const C* sR = reinterpret_cast<const C*>(bsm + 16);
        const C* sQ = sR + (size_t)na * ls;
        const C* sD = sR + (size_t)2 * na * ls;
        const C* sH = sD + (size_t)op.ndiag * ds;
        int slot[BG_MAXCOL];
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q) slot[q] = __popc(mask & ((1 << q) - 1));
        int dsh[SYLV_MAXDIAG];
#pragma unroll
        for (int d = 0; d < SYLV_MAXDIAG; ++d)
            dsh[d] = d < op.ndiag ? d * ds + (int)(((size_t)d * op.n + r0) % E) - r0 : 0;
        for (int i = r0 + threadIdx.x; ok && i < r1; i += blockDim.x) {
            C y[BG_MAXCOL];
#pragma unroll
            for (int q = 0; q < BG_MAXCOL; ++q) y[q] = zero<C>();
#pragma unroll
            for (int d = 0; d < SYLV_MAXDIAG; ++d) {
                if (d < op.ndiag) {
                    const int k = i + op.offs[d];
                    if (k >= 0 && k < sd.n) {
                        const C a = sD[dsh[d] + i];
#pragma unroll
                        for (int q = 0; q < BG_MAXCOL; ++q)
                            if (mask >> q & 1) {
                                const size_t o = (size_t)slot[q] * ls + (k - lo);
                                y[q] += a * (sR[o] + beta[q] * sQ[o]);
                            }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < BG_MAXCOL; ++q) {
                if (mask >> q & 1) {
                    const size_t o = (size_t)slot[q] * ls + (i - lo);
                    C* c = bv + q * cs + (size_t)i;
                    c[BV_P * ld] = sR[o] + beta[q] * sQ[o];
                    c[BV_V * ld] = y[q];
                    acc[q] += cmul(sH[(size_t)slot[q] * hs + (i - r0)], y[q]);
                }
            }
        }
        if (!ok)
#pragma unroll
            for (int q = 0; q < BG_MAXCOL; ++q) acc[q] = from_real<C>((typename RealOf<C>::type)NAN);
    } else {
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
    const int rpc = sd.rows_per_chunk;
    const int halo = op_halo_of(op.offs, op.ndiag);
    if (sd.aval && stage_bytes<C>(rpc, halo, op.ndiag, na, 2, 0) <= dyn_smem_bytes()) {
        // staged: r, v at [lo, hi) and the stencil rows in shared memory
        extern __shared__ __align__(16) unsigned char bsm[];
        constexpr int E = StageElems<C>::value;
        const int ls = stage_ls<C>(rpc, halo), ds = stage_ds<C>(rpc);
        const int lo = max(0, r0 - halo) / E * E;
        const int hi = (int)min((size_t)ld, (size_t)((min(sd.n, r1 + halo) + E - 1) / E * E));
        const int vids[2] = {BV_R, BV_V};
        bicg_stage_issue<T, S, C, 2, 0>(sd, op, mask, r0, r1, lo, hi, vids, 0, ls, ds, 0, bsm);
        const bool ok = stage_wait(reinterpret_cast<unsigned long long*>(bsm), ctl);
        const C* sR = reinterpret_cast<const C*>(bsm + 16);
        const C* sV = sR + (size_t)na * ls;
        const C* sD = sR + (size_t)2 * na * ls;
        int slot[BG_MAXCOL];
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q) slot[q] = __popc(mask & ((1 << q) - 1));
        int dsh[SYLV_MAXDIAG];
#pragma unroll
        for (int d = 0; d < SYLV_MAXDIAG; ++d)
            dsh[d] = d < op.ndiag ? d * ds + (int)(((size_t)d * op.n + r0) % E) - r0 : 0;
        for (int i = r0 + threadIdx.x; ok && i < r1; i += blockDim.x) {
            C y[BG_MAXCOL];
#pragma unroll
            for (int q = 0; q < BG_MAXCOL; ++q) y[q] = zero<C>();
#pragma unroll
            for (int d = 0; d < SYLV_MAXDIAG; ++d) {
                if (d < op.ndiag) {
                    const int k = i + op.offs[d];
                    if (k >= 0 && k < sd.n) {
                        const C a = sD[dsh[d] + i];
#pragma unroll
                        for (int q = 0; q < BG_MAXCOL; ++q)
                            if (mask >> q & 1) {
                                const size_t o = (size_t)slot[q] * ls + (k - lo);
                                y[q] += a * (sR[o] - alpha[q] * sV[o]);
                            }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < BG_MAXCOL; ++q) {
                if (mask >> q & 1) {
                    const size_t o = (size_t)slot[q] * ls + (i - lo);
                    const C si = sR[o] - alpha[q] * sV[o];
                    bv[q * cs + (size_t)BV_T * ld + i] = y[q];
                    acc[3 * q] += cmul(y[q], si);
                    acc[3 * q + 1] += from_real<C>(abs2(y[q]));
                    acc[3 * q + 2] += from_real<C>(abs2(si));
                }
            }
        }
        if (!ok)
#pragma unroll
            for (int q = 0; q < 3 * BG_MAXCOL; ++q) acc[q] = from_real<C>((typename RealOf<C>::type)NAN);
    } else {
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
