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

// Resident blocks per SM the step kernels are compiled for (their register
// budget): the staged stencil kernels a and b hold three blocks per SM in
// shared memory anyway; the streaming update kernel c keeps more blocks for
// loads in flight.  complex128 needs twice the registers per value: two
// blocks per SM keep its kernels free of large spills.
template <typename C> struct BicgOccAB { static constexpr int value = 3; };
template <> struct BicgOccAB<cplx> { static constexpr int value = 2; };
template <typename C> struct BicgOccC { static constexpr int value = 3; };
template <> struct BicgOccC<float> { static constexpr int value = 4; };
template <> struct BicgOccC<cplx> { static constexpr int value = 2; };

// Vectors of one BiCGstab system, column-major, ldv apart, C precision.
enum BVec : int { BV_R = 0, BV_Q = 1, BV_P = 2, BV_V = 3, BV_T = 4, BV_RH = 5, BV_COUNT = 6 };

// A group: systems sys0 .. sys0 + ncol - 1 (same operator, shift and rows;
// their vectors lie BV_COUNT * ldv apart), its chunk partial sums and its
// completion counter, with copies of the systems' shared descriptor fields
// (one load resolves a work item).
template <typename T, typename C>
struct BGroup {
    int sys0, ncol, nchunks;
    T* part;                 // nchunks x BG_PSTRIDE
    unsigned* counter;
    int n, rpc, ndiag, halo; // rows, rows per chunk, stored diagonals, largest |offset|
    size_t ldv;
    C* bv;                   // vectors of the group's first column
    const C* aval;           // pre-scaled stencil (null: not stored by diagonals)
    const T* pinv;           // Jacobi inverse or null
    int offs[SYLV_MAXDIAG];
    double nnz;              // nonzeros of the operator (byte counts)
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
// Shared-memory staging of a work item for the stencil product (kernels a
// and b).  The block's item [r0, r1) of a group is copied into shared memory
// with TMA bulk copies (cp.async.bulk, issued by the lanes of warp 0, all
// completing on one mbarrier):
//   * the two input vectors of each active column at the neighbour rows
//     [lo, hi) = [r0 - H, r1 + H) rounded out to 16-byte boundaries (H = the
//     largest |offset| of the stored diagonals); rows outside [0, ldv) are
//     zero-filled by warp 0, rows in [n, ldv) are zero in global memory (never
//     written), and the pre-scaled stencil value of a neighbour outside the
//     grid is zero, so the product needs no bounds checks;
//   * the stencil diagonals at the own rows (they may start off a 16-byte
//     boundary: the aligned interior by one bulk copy, the ends by the lane,
//     the value of row i at shift + (i - r0) in the diagonal's slot);
//   * (kernel a) the shadow vector at the own rows.
// Shared-memory indices are 32-bit and the loops over diagonals and columns
// run to the item's counts.  An item that does not fit the launch's stage
// size (or an operator that is not a stencil) reads global memory directly.
// ---------------------------------------------------------------------------
template <typename X> struct StageElems { static constexpr int value = sizeof(X) >= 16 ? 1 : 16 / (int)sizeof(X); };
template <typename X> HD int round_e(int k) {
    constexpr int e = StageElems<X>::value;
    return (k + e - 1) / e * e;
}
// slot lengths (elements; every slot is a multiple of 16 bytes)
template <typename X> HD int slot_nb(int rpc, int halo) {
    return round_e<X>(rpc + 2 * halo + 2 * StageElems<X>::value);
}
template <typename X> HD int slot_ow(int rpc) { return round_e<X>(rpc); }
template <typename X> HD int slot_sh(int rpc) { return round_e<X>(rpc + StageElems<X>::value); }
// bytes of a staged item with na active columns: kernel a (r, q at the
// neighbours, the stencil, rhat), kernel b (r, v at the neighbours, the
// stencil)
template <typename C> HD size_t stage_bytes_a(int rpc, int halo, int ndiag, int na) {
    return ((size_t)2 * na * slot_nb<C>(rpc, halo) + (size_t)ndiag * slot_sh<C>(rpc) + (size_t)na * slot_ow<C>(rpc)) *
           sizeof(C);
}
template <typename C> HD size_t stage_bytes_b(int rpc, int halo, int ndiag, int na) {
    return ((size_t)2 * na * slot_nb<C>(rpc, halo) + (size_t)ndiag * slot_sh<C>(rpc)) * sizeof(C);
}
// Dynamic shared memory a staged work item may take: two blocks per SM.
#define SYLV_BICG_SMEM_CAP (108 * 1024)

HD int op_halo_of(const int* offs, int ndiag) {
    int h = 0;
    for (int d = 0; d < ndiag; ++d) h = offs[d] < 0 ? (-offs[d] > h ? -offs[d] : h) : (offs[d] > h ? offs[d] : h);
    return h;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrival with the bytes the bulk copies will complete (release: warp 0's
// generic stores into the stage are visible to a thread that sees the phase
// complete)
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
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
// recorded for the host, the block waits once more (again bounded) for its
// copies in flight, and the caller poisons its partial sums, so the columns
// end as non-finite instead of the kernel waiting forever.
__device__ __forceinline__ bool stage_wait(unsigned long long* bar, BatchCtl* ctl) {
    bool ok = true;
    for (unsigned it = 0; !mbar_try_wait(bar, 0u); ++it)
        if (it > (1u << 22)) { ok = false; break; }
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(&ctl->stage_fault, 1);
        for (unsigned it = 0; !mbar_try_wait(bar, 0u) && it <= (1u << 22); ++it) {
        }
        __syncthreads();
    }
    return ok;
}

// Column of active slot j of a column mask.
__device__ __forceinline__ int col_of(int mask, int j) {
    int q = 0, c = -1;
    for (; q < BG_MAXCOL; ++q)
        if ((mask >> q & 1) && ++c == j) break;
    return q;
}

// Own rows [r0, r0 + m) of an array that may start off a 16-byte boundary,
// copied into the slot at dst so that element e lands at dst[shift + e]
// (shift = the array's offset from the 16-byte boundary below it, in
// elements): the aligned interior by one bulk copy, the rest by the lane.
template <typename X>
__device__ __forceinline__ int sh_shift(const X* src) { return (int)(((uintptr_t)src & 15) / sizeof(X)); }
template <typename X>
__device__ __forceinline__ void sh_plan(const X* src, int m, X* dst, const void*& csrc, void*& cdst, unsigned& bytes) {
    const uintptr_t s0 = (uintptr_t)src, s1 = s0 + (uintptr_t)m * sizeof(X);
    const uintptr_t a = (s0 + 15) & ~(uintptr_t)15, b = s1 & ~(uintptr_t)15;
    if (b > a) {
        csrc = reinterpret_cast<const void*>(a);
        cdst = reinterpret_cast<unsigned char*>(dst) + (a - (s0 & ~(uintptr_t)15));
        bytes = (unsigned)(b - a);
    }
    const int shift = sh_shift(src);
    for (int e = 0; e < m; ++e) {
        const uintptr_t p = s0 + (uintptr_t)e * sizeof(X);
        if (b > a && p >= a && p < b) {
            e += (int)((b - p) / sizeof(X)) - 1;
            continue;
        }
        dst[shift + e] = ldro(src + e);
    }
}

// Warp 0: issues the staging of the block's item.  KIND 0: kernel a (r and
// q at the neighbours, the stencil, rhat), 1: kernel b (r and v at the
// neighbours, the stencil).  Slot order: neighbour vectors v * na + j, the
// ndiag diagonals, (a) rhat of slot j.
template <typename T, typename C, int KIND>
__device__ __forceinline__ void bicg_stage_issue(const BGroup<T, C>& g, int mask, int na, int r0, int r1, int lo,
                                                 int hi, unsigned char* smem, unsigned long long* bar) {
    const int lane = threadIdx.x & 31;
    const size_t ld = g.ldv, cs = (size_t)BV_COUNT * ld;
    const int ls = slot_nb<C>(g.rpc, g.halo), ds = slot_sh<C>(g.rpc);
    C* const sc = reinterpret_cast<C*>(smem);
    const void* csrc = nullptr;
    void* cdst = nullptr;
    unsigned bytes = 0;
    int u = lane;
    if (u < 2 * na) {
        const int v = u / na, j = u % na;
        const int vid = v == 0 ? BV_R : (KIND == 0 ? BV_Q : BV_V);
        const int a0 = max(lo, 0), a1 = (int)min((size_t)hi, ld);
        if (a1 > a0) {
            csrc = g.bv + col_of(mask, j) * cs + (size_t)vid * ld + a0;
            cdst = sc + (size_t)u * ls + (a0 - lo);
            bytes = (unsigned)((a1 - a0) * sizeof(C));
        }
    } else if ((u -= 2 * na) < g.ndiag) {
        sh_plan(g.aval + (size_t)u * g.n + r0, r1 - r0, sc + (size_t)2 * na * ls + (size_t)u * ds, csrc, cdst, bytes);
    } else if (KIND == 0 && (u -= g.ndiag) < na) {
        csrc = g.bv + col_of(mask, u) * cs + (size_t)BV_RH * ld + r0;
        cdst = sc + (size_t)2 * na * ls + (size_t)g.ndiag * ds + (size_t)u * slot_ow<C>(g.rpc);
        bytes = (unsigned)(round_e<C>(r1 - r0) * sizeof(C));
    }
    // rows of the neighbour ranges outside [0, ldv): zero
    const int z0 = max(0, -lo), z1 = (int)max((long long)0, (long long)hi - (long long)ld);
    if (z0 || z1) {
        for (int v = 0; v < 2 * na; ++v) {
            C* s = sc + (size_t)v * ls;
            for (int e = lane; e < z0; e += 32) s[e] = zero<C>();
            for (int e = lane; e < z1; e += 32) s[(int)(ld - lo) + e] = zero<C>();
        }
    }
    const unsigned total = __reduce_add_sync(0xffffffffu, bytes);
    __syncwarp();
    if (lane == 0) mbar_arrive_tx(bar, total);
    __syncwarp();
    if (bytes) bulk_to_smem(cdst, csrc, bytes, bar);
}

// Block sums of K * BG_MAXCOL accumulators kept per active slot j (warps
// combined in A, each sum converted to T once), written to
// out[col[j] * K + k] for the na active slots.
template <typename T, typename A, int K>
__device__ __forceinline__ void bg_block_sums_slots(A (&acc)[K * BG_MAXCOL], T* out, const int (&col)[BG_MAXCOL],
                                                    int na) {
    __shared__ A red[SYLV_NWARP][K * BG_MAXCOL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < K * BG_MAXCOL; ++l) {
        if (l < K * na) {
            const A v = warp_sum(acc[l]);
            if (lane == 0) red[warp][l] = v;
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < K * na; l += blockDim.x) {
        A s = red[0][l];
#pragma unroll
        for (int w = 1; w < SYLV_NWARP; ++w) s += red[w][l];
        int c = 0;
#pragma unroll
        for (int j = 0; j < BG_MAXCOL; ++j)
            if (j == l / K) c = col[j];
        out[c * K + l % K] = cvt<T>(s);
    }
}

// Block sums of NV accumulators indexed by column (warps combined in A, each
// sum converted to T once) written to out[0..NV).
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
template <typename T, typename C>
__device__ __forceinline__ int group_mask(const SysState<T>* sts, const BGroup<T, C>& g, int ph) {
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
// Work list of a device iteration: the items (group, chunk) of the groups
// with an active column, in group order, and its length ctl->nlist (one
// block).  The step kernels take their items from it; blocks beyond its
// length return at once.  When a graph drives the solve and its step-kernel
// nodes are device-updatable, their grids are set to the list's length, so
// the iterations in which few systems are active launch few blocks.
// ---------------------------------------------------------------------------
template <typename T, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_bicg_list(const BGroup<T, C>* __restrict__ groups, int ngroups, const SysState<T>* __restrict__ sts,
            Item* __restrict__ list, BatchCtl* ctl) {
    pdl_wait();
    __shared__ int wsum[SYLV_NWARP];
    const int per = (ngroups + SYLV_BLOCK - 1) / SYLV_BLOCK;
    const int g0 = min(ngroups, (int)threadIdx.x * per), g1 = min(ngroups, g0 + per);
    auto active = [&](int g) {
        const BGroup<T, C>& gr = groups[g];
        bool on = false;
        for (int q = 0; q < gr.ncol; ++q) on |= sts[gr.sys0 + q].phase == PH_ARNOLDI;
        return on;
    };
    int cnt = 0;
    for (int g = g0; g < g1; ++g)
        if (active(g)) cnt += groups[g].nchunks;
    // exclusive prefix sum of cnt over the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = cnt;
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, m);
        if (lane >= m) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int off = inc - cnt;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    for (int g = g0; g < g1; ++g) {
        if (!active(g)) continue;
        const int nc = groups[g].nchunks;
        for (int c = 0; c < nc; ++c) list[off + c] = Item{g, c};
        off += nc;
    }
    if (threadIdx.x == SYLV_BLOCK - 1) {
        const int total = off;
        ctl->nlist = total;
        if (ctl->graph && ctl->dyn_grid) {
            const dim3 grid(total > 0 ? total : 1);
            for (int k = 0; k < 3; ++k) cudaGraphKernelNodeSetGridDim(ctl->dn_step[k], grid);
        }
    }
}

// ---------------------------------------------------------------------------
// Step part a: p = r + beta q, v = Op' p, partial rhat^* v.  The last block of
// a group counts the step and sets alpha = rho / (rhat^* v); a zero or
// non-finite denominator ends the cycle (breakdown) without an update.
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK, BicgOccAB<C>::value)
k_bicg_a(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts, const OpDesc* __restrict__ ops,
         const BGroup<T, C>* __restrict__ groups, const Item* __restrict__ items, int cap, BatchCtl* ctl) {
    pdl_wait();
    count_launch(ctl, K_SPMV);
    if (ctl->graph && blockIdx.x == 0 && threadIdx.x == 0) {
        cudaGraphSetConditional(ctl->h_loop, 0u);
        if (ctl->bouter) cudaGraphSetConditional(ctl->h_bouter, 0u);
    }
    if ((int)blockIdx.x >= ctl->nlist) return;
    const Item it = items[blockIdx.x];
    const BGroup<T, C>& g = groups[it.sys];
    const int mask = group_mask(sts, g, PH_ARNOLDI);
    if (!mask) return;
    const int na = __popc(mask);
    const int r0 = it.chunk * g.rpc, r1 = min(g.n, r0 + g.rpc);
    count_work(ctl, K_SPMV, it.chunk, g.nnz * sizeof(C) + 5.0 * na * g.n * sizeof(C),
               FmaFlops<C>::v * na * (g.nnz + 2.0 * g.n));
    int col[BG_MAXCOL];
#pragma unroll
    for (int j = 0; j < BG_MAXCOL; ++j) col[j] = j < na ? col_of(mask, j) : 0;
    C acc[BG_MAXCOL];
#pragma unroll
    for (int q = 0; q < BG_MAXCOL; ++q) acc[q] = zero<C>();
    const size_t ld = g.ldv, vcs = (size_t)BV_COUNT * ld;
    if (g.aval && stage_bytes_a<C>(g.rpc, g.halo, g.ndiag, na) <= (size_t)cap) {
        extern __shared__ __align__(128) unsigned char bsm[];
        __shared__ __align__(8) unsigned long long bar;
        constexpr int E = StageElems<C>::value;
        const int ndiag = g.ndiag, halo = g.halo;
        const int lo = ((r0 - halo) >= 0 ? (r0 - halo) / E : -((halo - r0 + E - 1) / E)) * E;   // floor to E
        const int hi = (r1 + halo + E - 1) / E * E;
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x < 32) bicg_stage_issue<T, C, 0>(g, mask, na, r0, r1, lo, hi, bsm, &bar);
        C beta[BG_MAXCOL];
        C* outc[BG_MAXCOL];
#pragma unroll
        for (int j = 0; j < BG_MAXCOL; ++j) {
            beta[j] = j < na ? cvt<C>(sts[g.sys0 + col[j]].bbeta) : zero<C>();
            outc[j] = g.bv + col[j] * vcs;
        }
        const int ls = slot_nb<C>(g.rpc, halo), ds = slot_sh<C>(g.rpc), hs = slot_ow<C>(g.rpc);
        int doff[SYLV_MAXDIAG], koff[SYLV_MAXDIAG];
#pragma unroll
        for (int d = 0; d < SYLV_MAXDIAG; ++d) {
            doff[d] = d < ndiag ? d * ds + sh_shift(g.aval + (size_t)d * g.n + r0) : 0;
            koff[d] = d < ndiag ? r0 - lo + g.offs[d] : 0;
        }
        const bool ok = stage_wait(&bar, ctl);
        const C* sR = reinterpret_cast<const C*>(bsm);
        const C* sQ = sR + na * ls;
        const C* sD = sR + 2 * na * ls;
        const C* sH = sD + ndiag * ds;
        for (int il = threadIdx.x; ok && il < r1 - r0; il += blockDim.x) {
            C y[BG_MAXCOL];
#pragma unroll
            for (int j = 0; j < BG_MAXCOL; ++j) y[j] = zero<C>();
#pragma unroll
            for (int d = 0; d < SYLV_MAXDIAG; ++d) {
                if (d < ndiag) {
                    const C a = sD[doff[d] + il];
                    const int k = il + koff[d];
#pragma unroll
                    for (int j = 0; j < BG_MAXCOL; ++j)
                        if (j < na) y[j] += a * (sR[j * ls + k] + beta[j] * sQ[j * ls + k]);
                }
            }
            const int ko = il + r0 - lo;
#pragma unroll
            for (int j = 0; j < BG_MAXCOL; ++j) {
                if (j < na) {
                    C* c = outc[j] + (size_t)(r0 + il);
                    c[BV_P * ld] = sR[j * ls + ko] + beta[j] * sQ[j * ls + ko];
                    c[BV_V * ld] = y[j];
                    acc[j] += cmul(sH[j * hs + il], y[j]);
                }
            }
        }
        if (!ok)
#pragma unroll
            for (int q = 0; q < BG_MAXCOL; ++q) acc[q] = from_real<C>((typename RealOf<C>::type)NAN);
        bg_block_sums_slots<T, C, 1>(acc, g.part + (size_t)it.chunk * BG_PSTRIDE, col, na);
    } else {
        // r, q, rhat and the stencil are not written here: read-only loads
        const SysDesc<T, S, C> sd = sysd[g.sys0];
        const OpDesc op = ops[sd.op];
        const T sigma = sts[g.sys0].sigma;
        C beta[BG_MAXCOL];
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q)
            beta[q] = (mask >> q & 1) ? cvt<C>(sts[g.sys0 + q].bbeta) : zero<C>();
        C* __restrict__ bv = sd.bv;
        auto P = [&](int q, int k) {
            const C* c = bv + q * vcs + (size_t)k;
            return ldro(c + BV_R * ld) + beta[q] * ldro(c + BV_Q * ld);
        };
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            C y[BG_MAXCOL];
            group_op_row(sd, op, sigma, i, mask, P, y);
#pragma unroll
            for (int q = 0; q < BG_MAXCOL; ++q) {
                if (mask >> q & 1) {
                    C* c = bv + q * vcs + (size_t)i;
                    c[BV_P * ld] = P(q, i);
                    c[BV_V * ld] = y[q];
                    acc[q] += cmul(ldro(c + BV_RH * ld), y[q]);
                }
            }
        }
        bg_block_sums<T, C, BG_MAXCOL>(acc, g.part + (size_t)it.chunk * BG_PSTRIDE);
    }
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
__global__ void __launch_bounds__(SYLV_BLOCK, BicgOccAB<C>::value)
k_bicg_b(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts, const OpDesc* __restrict__ ops,
         const BGroup<T, C>* __restrict__ groups, const Item* __restrict__ items, int cap, BatchCtl* ctl) {
    pdl_wait();
    count_launch(ctl, K_CGS2);
    if ((int)blockIdx.x >= ctl->nlist) return;
    const Item it = items[blockIdx.x];
    const BGroup<T, C>& g = groups[it.sys];
    const int mask = group_mask(sts, g, PH_ARNOLDI);
    if (!mask) return;
    const int na = __popc(mask);
    const int r0 = it.chunk * g.rpc, r1 = min(g.n, r0 + g.rpc);
    count_work(ctl, K_CGS2, it.chunk, g.nnz * sizeof(C) + 3.0 * na * g.n * sizeof(C),
               FmaFlops<C>::v * na * (g.nnz + 4.0 * g.n));
    int col[BG_MAXCOL];
#pragma unroll
    for (int j = 0; j < BG_MAXCOL; ++j) col[j] = j < na ? col_of(mask, j) : 0;
    C acc[3 * BG_MAXCOL];
#pragma unroll
    for (int q = 0; q < 3 * BG_MAXCOL; ++q) acc[q] = zero<C>();
    const size_t ld = g.ldv, vcs = (size_t)BV_COUNT * ld;
    if (g.aval && stage_bytes_b<C>(g.rpc, g.halo, g.ndiag, na) <= (size_t)cap) {
        extern __shared__ __align__(128) unsigned char bsm[];
        __shared__ __align__(8) unsigned long long bar;
        constexpr int E = StageElems<C>::value;
        const int ndiag = g.ndiag, halo = g.halo;
        const int lo = ((r0 - halo) >= 0 ? (r0 - halo) / E : -((halo - r0 + E - 1) / E)) * E;   // floor to E
        const int hi = (r1 + halo + E - 1) / E * E;
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x < 32) bicg_stage_issue<T, C, 1>(g, mask, na, r0, r1, lo, hi, bsm, &bar);
        C alpha[BG_MAXCOL];
        C* outc[BG_MAXCOL];
#pragma unroll
        for (int j = 0; j < BG_MAXCOL; ++j) {
            alpha[j] = j < na ? cvt<C>(sts[g.sys0 + col[j]].balpha) : zero<C>();
            outc[j] = g.bv + col[j] * vcs + (size_t)BV_T * ld;
        }
        const int ls = slot_nb<C>(g.rpc, halo), ds = slot_sh<C>(g.rpc);
        int doff[SYLV_MAXDIAG], koff[SYLV_MAXDIAG];
#pragma unroll
        for (int d = 0; d < SYLV_MAXDIAG; ++d) {
            doff[d] = d < ndiag ? d * ds + sh_shift(g.aval + (size_t)d * g.n + r0) : 0;
            koff[d] = d < ndiag ? r0 - lo + g.offs[d] : 0;
        }
        const bool ok = stage_wait(&bar, ctl);
        const C* sR = reinterpret_cast<const C*>(bsm);
        const C* sV = sR + na * ls;
        const C* sD = sR + 2 * na * ls;
        for (int il = threadIdx.x; ok && il < r1 - r0; il += blockDim.x) {
            C y[BG_MAXCOL];
#pragma unroll
            for (int j = 0; j < BG_MAXCOL; ++j) y[j] = zero<C>();
#pragma unroll
            for (int d = 0; d < SYLV_MAXDIAG; ++d) {
                if (d < ndiag) {
                    const C a = sD[doff[d] + il];
                    const int k = il + koff[d];
#pragma unroll
                    for (int j = 0; j < BG_MAXCOL; ++j)
                        if (j < na) y[j] += a * (sR[j * ls + k] - alpha[j] * sV[j * ls + k]);
                }
            }
            const int ko = il + r0 - lo;
#pragma unroll
            for (int j = 0; j < BG_MAXCOL; ++j) {
                if (j < na) {
                    const C si = sR[j * ls + ko] - alpha[j] * sV[j * ls + ko];
                    outc[j][r0 + il] = y[j];
                    acc[3 * j] += cmul(y[j], si);
                    acc[3 * j + 1] += from_real<C>(abs2(y[j]));
                    acc[3 * j + 2] += from_real<C>(abs2(si));
                }
            }
        }
        if (!ok)
#pragma unroll
            for (int q = 0; q < 3 * BG_MAXCOL; ++q) acc[q] = from_real<C>((typename RealOf<C>::type)NAN);
        bg_block_sums_slots<T, C, 3>(acc, g.part + (size_t)it.chunk * BG_PSTRIDE, col, na);
    } else {
        // r, v and the stencil are not written here: read-only loads
        const SysDesc<T, S, C> sd = sysd[g.sys0];
        const OpDesc op = ops[sd.op];
        const T sigma = sts[g.sys0].sigma;
        C alpha[BG_MAXCOL];
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q)
            alpha[q] = (mask >> q & 1) ? cvt<C>(sts[g.sys0 + q].balpha) : zero<C>();
        C* __restrict__ bv = sd.bv;
        auto Sf = [&](int q, int k) {
            const C* c = bv + q * vcs + (size_t)k;
            return ldro(c + BV_R * ld) - alpha[q] * ldro(c + BV_V * ld);
        };
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            C y[BG_MAXCOL];
            group_op_row(sd, op, sigma, i, mask, Sf, y);
#pragma unroll
            for (int q = 0; q < BG_MAXCOL; ++q) {
                if (mask >> q & 1) {
                    const C si = Sf(q, i);
                    bv[q * vcs + (size_t)BV_T * ld + i] = y[q];
                    acc[3 * q] += cmul(y[q], si);
                    acc[3 * q + 1] += from_real<C>(abs2(y[q]));
                    acc[3 * q + 2] += from_real<C>(abs2(si));
                }
            }
        }
        bg_block_sums<T, C, 3 * BG_MAXCOL>(acc, g.part + (size_t)it.chunk * BG_PSTRIDE);
    }
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
            const bool okw = isfinite(absv(om));
            st->bomega = okw ? om : zero<T>();
            st->bfin = okw ? 0 : 1;
            st->est = sn;
        }
    }
    if (threadIdx.x == 0) *g.counter = 0;
}

// Kernel c with float32 vectors: four consecutive rows per thread, 16-byte
// loads and stores of the vectors (their columns start on 32-row
// boundaries, so a row index that is a multiple of four is 16-byte aligned);
// the rows of a ragged end are stored one by one (rows in [n, ldv) stay
// zero).  Same arithmetic per row as the generic loop.
template <typename T>
__device__ __forceinline__ void bicg_c_rows4(float* __restrict__ bv, size_t ld, const T* __restrict__ pinv, int mask,
                                             const float (&alpha)[BG_MAXCOL], const float (&omega)[BG_MAXCOL],
                                             T* const (&X)[BG_MAXCOL], int r0, int r1, float (&acc)[2 * BG_MAXCOL]) {
    const size_t cs = (size_t)BV_COUNT * ld;
    const int m = r1 - r0;
    auto ld4 = [](const float* a) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(a));
        return v;
    };
    for (int e0 = 4 * (int)threadIdx.x; e0 < m; e0 += 4 * (int)blockDim.x) {
        const int i = r0 + e0;
        const int ne = min(4, m - e0);
        T pi[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) pi[e] = (pinv && e < ne) ? ldro(pinv + i + e) : make_scalar<T>(1.0, 0.0);
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q) {
            if (!(mask >> q & 1)) continue;
            float* c = bv + q * cs + (size_t)i;
            const float4 p4 = ld4(c + BV_P * ld), v4 = ld4(c + BV_V * ld), r4 = ld4(c + BV_R * ld);
            const float4 t4 = ld4(c + BV_T * ld), h4 = ld4(c + BV_RH * ld);
            T xo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) xo[e] = e < ne ? ldro(X[q] + i + e) : zero<T>();
            const float pa[4] = {p4.x, p4.y, p4.z, p4.w}, va[4] = {v4.x, v4.y, v4.z, v4.w};
            const float ra[4] = {r4.x, r4.y, r4.z, r4.w}, ta[4] = {t4.x, t4.y, t4.z, t4.w};
            const float ha[4] = {h4.x, h4.y, h4.z, h4.w};
            float rn[4], qn[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float sv = ra[e] - alpha[q] * va[e];
                if (e < ne) X[q][i + e] = xo[e] + pi[e] * cvt<T>(alpha[q] * pa[e] + omega[q] * sv);
                rn[e] = sv - omega[q] * ta[e];
                qn[e] = pa[e] - omega[q] * va[e];
                if (e < ne) {
                    acc[2 * q] += ha[e] * rn[e];
                    acc[2 * q + 1] += rn[e] * rn[e];
                }
            }
            if (ne == 4) {
                *reinterpret_cast<float4*>(c + BV_R * ld) = make_float4(rn[0], rn[1], rn[2], rn[3]);
                *reinterpret_cast<float4*>(c + BV_Q * ld) = make_float4(qn[0], qn[1], qn[2], qn[3]);
            } else {
                for (int e = 0; e < ne; ++e) {
                    c[BV_R * ld + e] = rn[e];
                    c[BV_Q * ld + e] = qn[e];
                }
            }
        }
    }
}
template <typename T, typename C> struct BicgRows4 { static constexpr bool value = false; };
template <typename T> struct BicgRows4<T, float> { static constexpr bool value = true; };

// ---------------------------------------------------------------------------
// Step part c: x += P^{-1}(alpha p + omega s) in float64, r = s - omega t,
// q = p - omega v, partial rhat^* r and r^* r.  The last block records the
// residual norm and ends the cycle when it meets the tolerance, at the step
// cap or at a breakdown (rho' = 0 or omega = 0); otherwise it sets
// beta' = (rho' / rho)(alpha / omega).
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK, BicgOccC<C>::value)
k_bicg_c(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
         const BGroup<T, C>* __restrict__ groups, const Item* __restrict__ items, BatchCtl* ctl) {
    pdl_wait();
    count_launch(ctl, K_CGS3);
    const bool inlist = (int)blockIdx.x < ctl->nlist;
    const Item it = inlist ? items[blockIdx.x] : Item{0, 0};
    const BGroup<T, C>& g = groups[it.sys];
    const int mask = inlist ? group_mask(sts, g, PH_ARNOLDI) : 0;
    if (mask) {
        const int na = __popc(mask);
        const int r0 = it.chunk * g.rpc, r1 = min(g.n, r0 + g.rpc);
        count_work(ctl, K_CGS3, it.chunk,
                   7.0 * na * g.n * sizeof(C) + 2.0 * na * g.n * sizeof(T) + (g.pinv ? (double)g.n * sizeof(T) : 0.0),
                   FmaFlops<C>::v * na * 6.0 * g.n);
        C alpha[BG_MAXCOL], omega[BG_MAXCOL];
        T* X[BG_MAXCOL];
#pragma unroll
        for (int q = 0; q < BG_MAXCOL; ++q) {
            const bool on = mask >> q & 1;
            alpha[q] = on ? cvt<C>(sts[g.sys0 + q].balpha) : zero<C>();
            omega[q] = on ? cvt<C>(sts[g.sys0 + q].bomega) : zero<C>();
            X[q] = on ? sts[g.sys0 + q].x : nullptr;
        }
        C* __restrict__ bv = g.bv;
        const size_t ld = g.ldv, cs = (size_t)BV_COUNT * ld;
        const T* __restrict__ pinv = g.pinv;
        C acc[2 * BG_MAXCOL];
#pragma unroll
        for (int q = 0; q < 2 * BG_MAXCOL; ++q) acc[q] = zero<C>();
        // every element is read and then overwritten by the same thread only:
        // read-only loads, so the next row's loads may pass this row's stores
        if constexpr (BicgRows4<T, C>::value) {
            bicg_c_rows4<T>(bv, ld, pinv, mask, alpha, omega, X, r0, r1, acc);
        } else {
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
                                                const OpDesc* __restrict__ ops, const BGroup<T, C>& g, int chunk,
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
             const BGroup<T, C>* __restrict__ groups, const Item* __restrict__ items, int nitems, BatchCtl* ctl) {
    pdl_wait();
    count_launch(ctl, K_RRES);
    // this block's items w = blockIdx.x + i * gridDim.x: the threads examine
    // up to SYLV_BLOCK of them at once, then the block restarts the active ones
    __shared__ int wl[SYLV_BLOCK];
    __shared__ int wn;
    for (int base = blockIdx.x; base < nitems; base += SYLV_BLOCK * gridDim.x) {
        if (threadIdx.x == 0) wn = 0;
        __syncthreads();
        const int w = base + (int)threadIdx.x * (int)gridDim.x;
        if (w < nitems && group_mask(sts, groups[items[w].sys], PH_RESID)) wl[atomicAdd(&wn, 1)] = w;
        __syncthreads();
        const int nw = wn;
        for (int e = 0; e < nw; ++e) {
            // any order: each item writes its own partial sums
            const Item it = items[wl[e]];
            bicg_resid_item<T, S, C>(sysd, sts, ops, groups[it.sys], it.chunk, ctl);
            __syncthreads();      // shared reduction buffers are reused by the next item
        }
    }
    if (ctl->graph) graph_tail<T>(ctl, sts, K_RRES);
}

}  // namespace sylv
