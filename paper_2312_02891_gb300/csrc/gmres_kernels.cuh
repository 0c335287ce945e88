// gmres_kernels.cuh - device kernels of the batched restarted GMRES(m) that
// solves the shifted inner systems of Algorithm 1 (inexact LR-ADI):
//   (A + beta_k I) z = w_{k-1}(:, l)   and   (B^T + conj(alpha_k) I) y = t_{k-1}(:, l),
// each column separately with right Jacobi preconditioning and the stop test
// ||r(:, l)|| <= delta_k / r (Sec. 3.3, "Further implementation aspects").
//
// One launch serves every active system of a batch: the grid is a list of
// (system, chunk) work items, each chunk a contiguous row range.  With
// classical Gram-Schmidt applied twice an Arnoldi step is three sweeps over
// the rows:
//   k_arnoldi_spmv : w = (Op + sigma I) P^{-1} v_j and h1 = V^* w (fused)
//   k_cgs_pass2    : h2 = V^* (w - V h1)
//   k_cgs_pass3    : v_{j+1} = w - V (h1 + h2), ||v_{j+1}||, then the Givens
//                    update of the Hessenberg least-squares problem
// and with the second pass delayed by one step (DCGS2) two:
//   k_dcgs_a : the product and every dot product of the step; the last
//              block of each system forms beta and the coefficients of sweep b
//   k_dcgs_b : the basis update, beside one Givens block per system (Givens
//              update, stop test, first pass of the next column);
// a restart is two more:
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

constexpr int PSTRIDE = 2 * SYLV_MAXV + 2; // partial-sum slots per chunk (delayed CGS2: 2j + 2 sums)

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
// The block's stores (its partial sums) are ordered before thread 0's
// increment by the barrier; the increment is a release (for this block's
// stores) and an acquire (for the stores of the blocks counted before it),
// and the second barrier passes that on to the block's other threads, whose
// loads of the partial sums bypass L1.  No thread of the block needs a full
// fence of its own.
__device__ __forceinline__ bool last_block(unsigned* counter, int nchunks) {
    __shared__ int am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(counter) : "memory");
        am_last = (prev == (unsigned)(nchunks - 1));
    }
    __syncthreads();
    return am_last != 0;
}

// Programmatic dependent launch.  A kernel of the device iteration first
// waits until the previous kernel of the stream has completed and its stores
// are visible (a no-op when it was launched without the attribute, e.g. in a
// graph).  The next kernel may be scheduled once every block of this one has
// called pdl_trigger() or exited: k_dcgs_a triggers after its sweep, so the
// blocks of k_dcgs_b take the SM slots freed during the sequential tail and
// start the moment it ends; the other kernels trigger by exiting.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// tot[l] = sum over chunks c of part[c * stride + l], l < cnt, in a fixed
// order.  Thread t takes sum l = t mod W and the chunks c = g, g + G, ...
// of group g = t / W (W = 32 or 64 sums per pass, G = blockDim / W groups),
// eight loads in flight at a time; the G group sums are then added in group
// order.  A warp reads 32 consecutive partial sums of one chunk (coalesced),
// and the float64 adds are spread over all lanes instead of repeated per
// warp and sum.
template <typename T>
__device__ __forceinline__ void reduce_chunks(const T* part, int nchunks, int stride, int cnt, T* tot) {
    __shared__ T rsum[SYLV_BLOCK];
    const int W = cnt > 32 ? 64 : 32;
    const int G = SYLV_BLOCK / W;
    for (int l0 = 0; l0 < cnt; l0 += W) {
        const int l = l0 + (int)threadIdx.x % W, g = (int)threadIdx.x / W;
        T sum = zero<T>();
        if (l < cnt) {
            for (int c0 = g; c0 < nchunks; c0 += 8 * G) {
                T v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int c = c0 + u * G;
                    v[u] = c < nchunks ? ldcg(part + (size_t)c * stride + l) : zero<T>();
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) sum += v[u];
            }
        }
        rsum[threadIdx.x] = sum;
        __syncthreads();
        if ((int)threadIdx.x < W && l0 + (int)threadIdx.x < cnt) {
            T t = rsum[threadIdx.x];
            for (int q = 1; q < G; ++q) t += rsum[q * W + threadIdx.x];
            tot[l0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
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
    if (ctl->graph && ctl->bouter) cudaGraphSetConditional(ctl->h_bouter, 1u);
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
// out[0..cnt); red is a shared buffer of SYLV_NWARP x PSTRIDE T (used as A).
// The warps of the block are combined in A (float32 for the mixed path) and
// each sum is converted to T once: on this GPU every float64 instruction,
// conversions included, occupies the small float64 pipe for a whole warp
// even with one active lane, so a conversion per warp and sum (lane 0 of
// each warp) had cost more than the sweep's own arithmetic.  Chunks are
// combined in T.
template <typename T, typename A, int NV>
__device__ __forceinline__ void block_reduce_to(A (&acc)[NV], int cnt, T* out, T (*red)[PSTRIDE]) {
    static_assert(sizeof(A) <= sizeof(T), "the reduction buffer holds T");
    A (*ra)[PSTRIDE] = reinterpret_cast<A (*)[PSTRIDE]>(red);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < NV; ++l) {
        if (l < cnt) {
            const A v = warp_sum(acc[l]);
            if (lane == 0) ra[warp][l] = v;
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
        A s = ra[0][l];
#pragma unroll
        for (int w = 1; w < SYLV_NWARP; ++w) s += ra[w][l];
        out[l] = cvt<T>(s);
    }
}

// ---------------------------------------------------------------------------
// Staged sweeps (real 32-bit and 16-bit basis storage).  Each warp streams
// its row tiles of the block's chunk (tiles t0 + warp, t0 + warp + NWARP, ...)
// through a ring of shared-memory stages: the tile's vectors 0..nv-1 (one
// contiguous range in the tile-major basis) and its 32 rows of the work
// vector are copied with cp.async, NST - 1 tiles ahead of use.  No register
// holds an in-flight basis value, so the accumulators alone set the register
// count, and every warp keeps several KB of loads in flight.
// ---------------------------------------------------------------------------
constexpr int SWEEP_WARP_SMEM = 8192;                         // staging bytes per warp
constexpr int SWEEP_SMEM = SWEEP_WARP_SMEM * SYLV_NWARP;      // dynamic shared memory per block

template <typename S, typename C> struct Staged {
    static constexpr bool value = sizeof(S) <= 4 && sizeof(C) == 4;   // real float32 / bfloat16 basis
};
template <typename S, typename C> constexpr int sweep_smem_bytes() { return Staged<S, C>::value ? SWEEP_SMEM : 0; }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory");
}

// The stage pipeline: tile_body(t, sv, sw) runs, by the whole warp, for
// every tile t of the warp in [t0, t1), with sv[32 l + r] = V_l(32 t + r)
// (l < nv) and sw[r] = w(32 t + r) in shared memory.
template <int NV, typename S, typename C, typename TileBody>
__device__ __forceinline__ void stream_tile_stages(const S* __restrict__ V, size_t tstride, const C* __restrict__ w,
                                                   int t0, int t1, int nv, TileBody tile_body) {
    extern __shared__ __align__(16) unsigned char sweep_dsm[];
    constexpr int NVS = NV < SYLV_MAXV ? NV : SYLV_MAXV;               // vectors a stage must hold
    constexpr int VB = NVS * 32 * (int)sizeof(S);                       // basis bytes of a tile
    constexpr int TB = VB + 32 * (int)sizeof(C);                        // + the work vector rows
    constexpr int NST0 = SWEEP_WARP_SMEM / TB;
    constexpr int NST = NST0 > 8 ? 8 : NST0;
    static_assert(NST >= 2, "a warp needs two stages");
    constexpr int P = NST - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wsm = sweep_dsm + warp * SWEEP_WARP_SMEM;
    const int ntile = t1 - t0;
    const int mine = ntile > warp ? (ntile - warp + SYLV_NWARP - 1) / SYLV_NWARP : 0;
    const int vchunks = nv * 32 * (int)sizeof(S) / 16;
    constexpr int WCH = 32 * (int)sizeof(C) / 16;
    auto issue = [&](int q) {
        const size_t t = (size_t)(t0 + warp + q * SYLV_NWARP);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(V + t * tstride);
        unsigned char* dst = wsm + (q % NST) * TB;
        for (int c = lane; c < vchunks; c += 32) cp_async16(dst + 16 * c, src + 16 * c);
        if (lane < WCH) cp_async16(dst + VB + 16 * lane, reinterpret_cast<const unsigned char*>(w + t * 32) + 16 * lane);
    };
#pragma unroll
    for (int q = 0; q < P; ++q) {
        if (q < mine) issue(q);
        cp_async_commit();
    }
    for (int q = 0; q < mine; ++q) {
        if (q + P < mine) issue(q + P);
        cp_async_commit();
        cp_async_wait<P>();
        __syncwarp();
        const unsigned char* st = wsm + (q % NST) * TB;
        tile_body(t0 + warp + q * SYLV_NWARP, reinterpret_cast<const S*>(st), reinterpret_cast<const C*>(st + VB));
        __syncwarp();
    }
}

// Runs body(i, sv, wv) for every row i < r1 of the warp's tiles in [t0, t1),
// lane = row of the tile, with sv[32 l] = V_l(i) (l < nv) and wv = w(i) read
// from the stage.
template <int NV, typename S, typename C, typename Body>
__device__ __forceinline__ void stream_tiles(const S* __restrict__ V, size_t tstride, const C* __restrict__ w,
                                             int t0, int t1, int r1, int nv, Body body) {
    const int lane = threadIdx.x & 31;
    stream_tile_stages<NV, S, C>(V, tstride, w, t0, t1, nv, [&](int t, const S* sv, const C* sw) {
        const int i = t * 32 + lane;
        if (i < r1) body(i, sv + lane, sw[lane]);
    });
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
    } else if constexpr (Staged<S, C>::value && LAY == 1) {
        // 32-bit and 16-bit real bases: the product rows first, in the
        // warp-tile order of the staged sweep (each warp then stages only
        // rows it wrote itself), then the dot products from shared memory
        if (mode == 0) {
            // two row tiles per warp in flight: the stencil gathers of
            // independent rows overlap (four spill at 80 registers)
            const int lane = threadIdx.x & 31;
#pragma unroll 2
            for (int t = (r0 >> 5) + (int)(threadIdx.x >> 5); t < ((r1 + 31) >> 5); t += SYLV_NWARP) {
                const int i = t * 32 + lane;
                if (i < r1) w[i] = spmv_row<LAY>(sd, op, st, vj, sj, i);
            }
            __syncwarp();
        }
        stream_tiles<NV, S, C>(V, sd.tstride, w, r0 >> 5, (r1 + 31) >> 5, r1, j + 1,
                               [&](int, const S* sv, C wv) {
#pragma unroll
                                   for (int l = 0; l < NV; ++l)
                                       if (l <= j) acc[l] += cmul(cvt<C>(sv[32 * l]), wv);
                               });
    } else {
        // other 32-bit sweeps: the product rows first, then the dot products
        // over the same rows (each thread re-reads only the w entries it
        // wrote), so neither loop carries the other's registers
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
    if (ctl->graph && blockIdx.x == 0 && threadIdx.x == 0) {
        cudaGraphSetConditional(ctl->h_loop, 0u);
        if (ctl->bouter) cudaGraphSetConditional(ctl->h_bouter, 0u);
    }
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
    if constexpr (Staged<S, C>::value && LAY == 1) {
        stream_tiles<NV, S, C>(V, sd.tstride, w, r0 >> 5, (r1 + 31) >> 5, r1, j + 1, [&](int, const S* sv, C wv) {
            C w1 = wv;
#pragma unroll
            for (int l = 0; l < NV; ++l)
                if (l <= j) w1 -= cc[l] * cvt<C>(sv[32 * l]);
#pragma unroll
            for (int l = 0; l < NV; ++l)
                if (l <= j) acc[l] += cmul(cvt<C>(sv[32 * l]), w1);
        });
    } else {
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

// Column c of the Hessenberg matrix is complete: s_col[0..c] (shared
// memory) and the subdiagonal hn.  Applies the previous rotations and a new
// one, updates g and the residual estimate, counts the Arnoldi step and
// decides whether the cycle ends (estimate below tol, restart length, step
// cap, non-finite value); at the end of a cycle the least-squares solution
// y is formed by back substitution and the system moves to the update
// phase.  Returns the (block-uniform) end decision.  One warp runs the
// sequential parts.
template <typename T>
__device__ int hess_column_finish(int restart, double* hist, int hist_cap, SysState<T>* st, int c, const T* s_col,
                                  double hn, T* s_R /* shared, SYLV_MR * SYLV_MAXV */) {
    __shared__ T s_sn[SYLV_MR];
    __shared__ double s_cs[SYLV_MR];
    __shared__ T s_g[SYLV_MAXV];
    __shared__ int s_end;
    for (int i = threadIdx.x; i <= c; i += blockDim.x) {
        s_g[i] = st->g[i];
        if (i < c) { s_cs[i] = st->cs[i]; s_sn[i] = st->sn[i]; }
    }
    // R columns 0..c-1 (needed only when the cycle ends; loaded in parallel)
    for (int q = threadIdx.x; q < c * SYLV_MAXV; q += blockDim.x) s_R[q] = st->R[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        T col[SYLV_MAXV];
        for (int i = 0; i <= c; ++i) col[i] = s_col[i];
        col[c + 1] = make_scalar<T>(hn, 0.0);
        for (int i = 0; i < c; ++i) {
            const double cc_ = s_cs[i];
            const T sn_ = s_sn[i];
            const T t0 = cc_ * col[i] + sn_ * col[i + 1];
            const T t1 = cc_ * col[i + 1] - conjg(sn_) * col[i];
            col[i] = t0;
            col[i + 1] = t1;
        }
        double cr;
        T sr;
        givens(col[c], col[c + 1], cr, sr);
        st->cs[c] = cr;
        st->sn[c] = sr;
        col[c] = cr * col[c] + sr * col[c + 1];
        const T gc = s_g[c];
        const T gc1 = -(conjg(sr) * gc);
        st->g[c + 1] = gc1;
        st->g[c] = cr * gc;
        s_g[c] = cr * gc;
        for (int i = 0; i <= c; ++i) {
            st->R[c * SYLV_MAXV + i] = col[i];
            s_R[c * SYLV_MAXV + i] = col[i];
        }
        const double est = absv(gc1);
        st->est = est;
        st->iters += 1;
        if (hist && st->iters - 1 < hist_cap) hist[st->iters - 1] = est;
        int end;
        if (!isfinite(est) || !isfinite(hn)) {
            st->status = ST_NONFINITE;
            st->nvec = 0;
            st->phase = PH_UPDATE;
            end = 2;
        } else if (est <= st->tol || c + 1 >= restart || st->iters >= st->max_iters || hn == 0.0) {
            st->nvec = c + 1;
            end = 1;
        } else {
            end = 0;
        }
        s_end = end;
    }
    __syncthreads();
    const int end = s_end;
    if (end != 1 || threadIdx.x >= 32) return end;
    // back substitution R y = g by columns, one warp: lane l owns g[l]
    const int k = c + 1;
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
    return end;
}

// Last block of sweep 3 (CGS2): Hessenberg column j = h1 + h2 with
// subdiagonal ||v_{j+1}||; the next step when the cycle goes on.
template <typename T>
__device__ void arnoldi_finish(int restart, double* hist, int hist_cap, SysState<T>* st, double nrm2) {
    __shared__ T s_col[SYLV_MAXV];
    __shared__ T s_R[SYLV_MR * SYLV_MAXV];
    const int j = st->j;
    const double hn = sqrt(nrm2);
    // column j as formed (unrotated) is kept in Hr, as in the delayed variant
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) {
        const T hi = i <= j ? st->h1[i] + st->h2[i] : make_scalar<T>(hn, 0.0);
        if (i <= j) s_col[i] = hi;
        st->Hr[j * SYLV_MAXV + i] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) st->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    const int end = hess_column_finish<T>(restart, hist, hist_cap, st, j, s_col, hn, s_R);
    if (end == 0 && threadIdx.x == 0) st->j = j + 1;
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
    if (threadIdx.x == 0) {
        s_last = atomicAdd(&ctl->gdone[kid], 1u) + 1u == gridDim.x;
        // the last block resets the count: the next launch may have another grid
        if (s_last) ctl->gdone[kid] = 0u;
    }
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
#define SYLV_PASS3_STAGED(NV)                                                 \
    stream_tiles<NV, S, C>(V, sd.tstride, w, r0 >> 5, (r1 + 31) >> 5, r1, j + 1,     \
                           [&](int i, const S* sv, C wv) {                    \
                               C x = wv;                                      \
                               _Pragma("unroll") for (int l = 0; l < NV; ++l) \
                                   if (l <= j) x -= cc[l] * cvt<C>(sv[32 * l]); \
                               const S xs = cvt<S>(x);                        \
                               vn[BI::row(sd, i)] = xs;                       \
                               acc[0] += abs2(cvt<C>(xs));                    \
                           });
    if constexpr (Staged<S, C>::value && LAY == 1) {
        SYLV_BUCKET_SWITCH(j, SYLV_PASS3_STAGED)
    } else {
        SYLV_BUCKET_SWITCH(j, SYLV_PASS3_CALL)
    }
#undef SYLV_PASS3_STAGED
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
// Arnoldi with delayed reorthogonalisation (DCGS2; Swirydowicz et al.,
// Numer. Linear Algebra Appl. 28 (2021)).  Step j works on u_j, the
// once-orthogonalised candidate for v_j, stored (unnormalised, scale sj) in
// basis slot j; slots 0..j-1 hold v_0..v_{j-1}.  Two sweeps per step:
//   k_dcgs_a : y = (Op + sigma I) P^{-1} u_j and, in the same pass,
//              s = V_<j^* u_j, alpha = u_j^* u_j, z = V_<j^* y, gamma = u_j^* y
//              (one grid reduction).  Its last block sets beta = ||u_j - V s||
//              = sqrt(alpha - |s|^2), completes Hessenberg column j-1 (first
//              pass of the previous step + s, subdiagonal beta), runs the
//              Givens update and stop test, and otherwise the coefficients of
//              sweep b and the first pass of column j:
//                h1 = ([z; v_j^* y] - H s) / beta,  v_j^* y = (gamma - s^* z) / beta
//   k_dcgs_b : v_j = (u_j - V_<j s) / beta, u_{j+1} = (y - V_<j z - v_j v_j^* y) / beta
//              (no reduction).
// Relative to CGS2 (three sweeps, three reductions per step) one sweep and
// two reductions go, for one extra product per restart cycle (the step that
// completes the last column).
// ---------------------------------------------------------------------------


// w = (Op + sigma I) P^{-1} (sj u) over the warp's row tiles of [r0, r1)
// (tiles t0 + warp, t0 + warp + NWARP, ...) for a stencil-stored operator
// (pre-scaled diagonals aval, tile-major u) with ndiag <= ND diagonals.  U
// tiles at a time: every load of the group (U x ndiag diagonal values and
// neighbour entries) is issued before the first multiply-add, so a warp keeps
// U x ndiag x 256 bytes in flight instead of waiting once per row tile.
template <int U, int ND, typename T, typename S, typename C>
__device__ __forceinline__ void product_tiles(const SysDesc<T, S, C>& sd, const OpDesc& op,
                                              const S* __restrict__ uj, typename RealOf<C>::type sj,
                                              int r0, int r1) {
    typedef BasisIx<1> BI;
    const C* __restrict__ av = sd.aval;
    C* __restrict__ w = sd.w;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tend = (r1 + 31) >> 5;
    for (int tb = (r0 >> 5) + warp; tb < tend; tb += U * SYLV_NWARP) {
        C a[U][ND];
        S x[U][ND];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int i = (tb + q * SYLV_NWARP) * 32 + lane;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const int k = i + op.offs[d];
                const bool ok = d < op.ndiag && i < r1 && k >= 0 && k < op.n;
                a[q][d] = ok ? av[(size_t)d * op.n + i] : zero<C>();
                x[q][d] = ok ? uj[BI::row(sd, k)] : cvt<S>(zero<C>());
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int i = (tb + q * SYLV_NWARP) * 32 + lane;
            C y = zero<C>();
#pragma unroll
            for (int d = 0; d < ND; ++d)
                if (d < op.ndiag) y += a[q][d] * cvt<C>(x[q][d]);
            if (i < r1) w[i] = sj * y;
        }
    }
}

// Rows [r0, r1) of sweep a with NV >= j accumulators per kind.
template <int NV, typename T, typename S, typename C>
__device__ __forceinline__ void dcgs_a_rows(const SysDesc<T, S, C>& sd, const OpDesc& op, const SysState<T>* st,
                                            int j, bool product, typename RealOf<C>::type sj, int r0, int r1,
                                            T* out, T (*red)[PSTRIDE]) {
    typedef BasisIx<1> BI;
    const S* __restrict__ V = sd.V;
    C* __restrict__ w = sd.w;
    const S* __restrict__ uj = V + BI::vec(sd, j);
    // acc[0..NV): X_l^* U, acc[NV..2NV): X_l^* Y, acc[2NV] = U^* U, acc[2NV+1] = U^* Y
    C acc[2 * NV + 2];
#pragma unroll
    for (int l = 0; l < 2 * NV + 2; ++l) acc[l] = zero<C>();
    auto body = [&](const C uv, const C wv, auto vl) {
#pragma unroll
        for (int l = 0; l < NV; ++l) {
            if (l < j) {
                const C xl = cvt<C>(vl(l));
                acc[l] += cmul(xl, uv);
                acc[NV + l] += cmul(xl, wv);
            }
        }
        acc[2 * NV] += cmul(uv, uv);
        acc[2 * NV + 1] += cmul(uv, wv);
    };
    if constexpr (Staged<S, C>::value) {
        if (product) {
            if (sd.aval && op.ndiag <= 5) {
                product_tiles<4, 5>(sd, op, uj, sj, r0, r1);      // 2D five-point stencils
            } else if (sd.aval && op.ndiag <= 7) {
                product_tiles<4, 7>(sd, op, uj, sj, r0, r1);      // 3D seven-point stencils
            } else if (sd.aval) {
                product_tiles<2, SYLV_MAXDIAG>(sd, op, uj, sj, r0, r1);
            } else {
                const int lane = threadIdx.x & 31;
#pragma unroll 2
                for (int t = (r0 >> 5) + (int)(threadIdx.x >> 5); t < ((r1 + 31) >> 5); t += SYLV_NWARP) {
                    const int i = t * 32 + lane;
                    if (i < r1) w[i] = spmv_row<1>(sd, op, st, uj, sj, i);
                }
            }
            __syncwarp();
        }
        stream_tiles<NV + 1, S, C>(V, sd.tstride, w, r0 >> 5, (r1 + 31) >> 5, r1, j + 1,
                                   [&](int, const S* sv, C wv) {
                                       const C uv = cvt<C>(sv[32 * j]);
                                       body(uv, product ? wv : zero<C>(), [&](int l) { return sv[32 * l]; });
                                   });
    } else {
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            C wv = zero<C>();
            if (product) {
                wv = spmv_row<1>(sd, op, st, uj, sj, i);
                w[i] = wv;
            }
            const S* __restrict__ vr = V + BI::row(sd, i);
            body(cvt<C>(vr[BI::vec(sd, j)]), wv, [&](int l) { return vr[BI::vec(sd, l)]; });
        }
    }
    // compact the used sums: s (j), z (j), alpha, gamma at 0..2j+1; warps
    // are combined in C and each sum is converted to T once
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C (*rc)[PSTRIDE] = reinterpret_cast<C (*)[PSTRIDE]>(red);
#pragma unroll
    for (int q = 0; q < 2 * NV + 2; ++q) {
        const int l = q < NV ? q : (q < 2 * NV ? q - NV : q - 2 * NV);
        const int dst = q < NV ? l : (q < 2 * NV ? j + l : 2 * j + l);
        const bool used = q < 2 * NV ? (l < j) : true;
        if (used) {
            const C v = warp_sum(acc[q]);
            if (lane == 0) rc[warp][dst] = v;
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < 2 * j + 2; l += blockDim.x) {
        C sum = rc[0][l];
#pragma unroll
        for (int q = 1; q < SYLV_NWARP; ++q) sum += rc[q][l];
        out[l] = cvt<T>(sum);
    }
}


// ---------------------------------------------------------------------------
// The sequential part of a delayed-CGS2 step is split in two.  What the next
// sweep needs - beta, the coefficients of sweep b, the first pass of column
// j - is formed by the last block of each system in k_dcgs_a (dcgs_step_tail);
// the Givens update of the completed column, the stop test and, at the end
// of a cycle, the least-squares solution run in one extra block per system
// of k_dcgs_b (dcgs_givens), beside that kernel's sweep.  On this GPU a
// float64 instruction costs a whole warp slot of a small pipe even with one
// active lane, so these scalar recurrences take microseconds; outside the
// critical path they overlap the sweep.  A cycle that the Givens update ends
// has its sweep b done for nothing (its vectors are not used).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                 :: "r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem) : "memory");
}

// Byte ranges [lo, hi) (multiples of 8) of *st copied to the same offsets of *ss.
template <typename T>
__device__ __forceinline__ void state_copy_async(const SysState<T>* st, SysState<T>* ss, size_t lo, size_t hi) {
    const char* g = reinterpret_cast<const char*>(st);
    char* d = reinterpret_cast<char*>(ss);
    for (size_t q = lo / 8 + threadIdx.x; q < hi / 8; q += blockDim.x) cp_async8(d + 8 * q, g + 8 * q);
}

// Dynamic shared memory of k_dcgs_a: the sweep stages, then (in the tail) the
// copy of the system state.
template <typename T, typename S, typename C> constexpr int dcgs_a_smem_bytes() {
    return sweep_smem_bytes<S, C>() > (int)sizeof(SysState<T>) ? sweep_smem_bytes<S, C>() : (int)sizeof(SysState<T>);
}

// Shared scratch of the Givens block of k_dcgs_b (in its dynamic shared memory).
template <typename T> struct GivensScratch {
    T R[SYLV_MR * SYLV_MAXV];
    T H[SYLV_MR * SYLV_MAXV];
    T col[SYLV_MAXV + 1];
    T g[SYLV_MAXV];
    T sn[SYLV_MR];
    T fs[SYLV_MAXV];
    double cs[SYLV_MR];
    double scale[SYLV_MAXV];
};
template <typename T, typename S, typename C> constexpr int dcgs_b_smem_bytes() {
    return sweep_smem_bytes<S, C>() > (int)sizeof(GivensScratch<T>) ? sweep_smem_bytes<S, C>()
                                                                    : (int)sizeof(GivensScratch<T>);
}

// Last block of system st in k_dcgs_a: beta, Hessenberg column j - 1 (first
// pass + s, subdiagonal beta; its Givens update is left to k_dcgs_b), and
// when the cycle can go on the coefficients of sweep b (the first pass of
// column j is also left to k_dcgs_b).  The fields it reads are copied to
// shared memory in one burst of asynchronous copies, issued together with the
// loads of the chunk reduction.
template <typename T, typename S, typename C>
__device__ void dcgs_step_tail(const SysDesc<T, S, C>& sd, SysState<T>* st, int j, double sj) {
    extern __shared__ __align__(16) unsigned char sweep_dsm[];
    SysState<T>& ss = *reinterpret_cast<SysState<T>*>(sweep_dsm);
    __shared__ T tot[PSTRIDE];
    __shared__ T s_s[SYLV_MAXV], s_z[SYLV_MAXV];
    __shared__ double s_beta, s_ib;
    __shared__ T s_vy;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // scalars, scale and h1
    state_copy_async(st, &ss, 0, offsetof(SysState<T>, h2));
    cp_async_commit();
    reduce_chunks(sd.part, sd.nchunks, PSTRIDE, 2 * j + 2, tot);
    cp_async_wait<0>();
    __syncthreads();
    // s = V^* u_j (scaled), z = V^* y, beta = ||u_j - V s||: one warp, lane l < j
    if (warp == 0) {
        T sl = zero<T>(), zl = zero<T>();
        if (lane < j) {
            sl = (ss.scale[lane] * sj) * tot[lane];
            zl = ss.scale[lane] * tot[j + lane];
            s_s[lane] = sl;
            s_z[lane] = zl;
        }
        const double nss = warp_sum(abs2(sl));
        const T sz = warp_sum(conjg(sl) * zl);
        if (lane == 0) {
            // beta and 1 / beta from one reciprocal square root (the float64
            // square root and divisions are long dependent sequences here)
            const double alpha = sj * sj * re(tot[2 * j]);
            const double x = fmax(alpha - nss, 0.0);
            const double rs = x > 0.0 ? rsqrt(x) : 0.0;
            s_beta = x * rs;
            s_ib = rs;
            s_vy = ((double)sj * tot[2 * j + 1] - sz) * rs;
            st->counter = 0;
        }
    }
    __syncthreads();
    const double beta = s_beta;
    if (j >= 1) {
        // Hessenberg column j - 1 as formed, for the Givens block and for the
        // first pass of the next columns
        for (int i = threadIdx.x; i <= j; i += blockDim.x)
            st->Hr[(j - 1) * SYLV_MAXV + i] = i < j ? ss.h1[i] + s_s[i] : make_scalar<T>(beta, 0.0);
        if (threadIdx.x == 0) st->gpend = j;
    }
    // the cycle goes on unless the restart length is reached or beta is zero
    // or not finite; the Givens block then ends it (j >= 1), else it ends here
    const bool go = j < sd.restart && beta > 0.0 && isfinite(beta);
    if (!go) {
        if (threadIdx.x == 0) {
            if (j == 0) {
                if (!isfinite(beta)) st->status = ST_NONFINITE;
                st->nvec = 0;
                st->phase = PH_UPDATE;
            }
            st->upd = 0;
        }
        return;
    }
    // the coefficients of sweep b, and the inputs of the first pass of column j
    const double ib = s_ib;
    const T vy = s_vy;
    for (int l = threadIdx.x; l < j; l += blockDim.x) {
        st->h2[l] = ss.scale[l] * s_s[l];      // v_j   = sj U - sum h2_l X_l
        st->cz[l] = ss.scale[l] * s_z[l];      // u_j+1 = Y - sum cz_l X_l - cv X_j
        st->fs[l] = s_s[l];
        st->fz[l] = s_z[l];
    }
    if (threadIdx.x == 0) {
        st->cv = ib * vy;
        st->sjb = sj;
        st->jb = j;
        st->upd = 1;
        st->scale[j] = ib;
        st->scale[j + 1] = ib;
        st->j = j + 1;
        st->fib = ib;
        st->fvy = vy;
        st->h1pend = j + 1;
    }
}

// Givens block of system st in k_dcgs_b.  Warp 0: the pending Hessenberg
// column c = gpend - 1 (formed in k_dcgs_a) gets the previous rotations and a
// new one; g and the residual estimate are updated and the Arnoldi step is
// counted; the cycle ends when the estimate meets the tolerance, the column
// is the last of the restart length, the step cap is reached, the
// subdiagonal is zero or a value is not finite.  At the end of a cycle the
// least-squares solution y is formed (back substitution, one warp) and the
// system moves to the update phase.  Warps 1..7 meanwhile form the first
// pass of the new column jn = h1pend - 1, h1 = (z - H s) / beta over the
// formed columns 0..jn-1 (four lanes per row), which the next k_dcgs_a
// completes.
template <typename T, typename S, typename C>
__device__ void dcgs_givens(const SysDesc<T, S, C>& sd, SysState<T>* st) {
    extern __shared__ __align__(16) unsigned char sweep_dsm[];
    GivensScratch<T>& gs = *reinterpret_cast<GivensScratch<T>*>(sweep_dsm);
    __shared__ int s_end, s_c, s_jn;
    if (threadIdx.x == 0) {
        s_c = st->gpend - 1;
        s_jn = st->h1pend - 1;
    }
    __syncthreads();
    const int c = s_c, jn = s_jn;
    // column c of H and the rotation state (c >= 0); formed columns 0..jn-1 (jn >= 1)
    if (c >= 0) {
        for (int i = threadIdx.x; i <= c + 1; i += blockDim.x) gs.col[i] = st->Hr[c * SYLV_MAXV + i];
        for (int i = threadIdx.x; i <= c; i += blockDim.x) {
            gs.g[i] = st->g[i];
            gs.scale[i] = st->scale[i];
            if (i < c) { gs.cs[i] = st->cs[i]; gs.sn[i] = st->sn[i]; }
        }
        for (int q = threadIdx.x; q < c * SYLV_MAXV; q += blockDim.x) gs.R[q] = st->R[q];
    }
    for (int q = threadIdx.x; q < (jn > 0 ? jn : 0) * SYLV_MAXV; q += blockDim.x) gs.H[q] = st->Hr[q];
    for (int q = threadIdx.x; q < jn; q += blockDim.x) gs.fs[q] = st->fs[q];
    __syncthreads();
    if (threadIdx.x == 0 && c >= 0) {
        // previous rotations applied to the column, carried down its rows
        T carry = gs.col[0];
        for (int i = 0; i < c; ++i) {
            const double cc_ = gs.cs[i];
            const T sn_ = gs.sn[i];
            const T nx = gs.col[i + 1];
            const T t0 = cc_ * carry + sn_ * nx;
            carry = cc_ * nx - conjg(sn_) * carry;
            gs.R[c * SYLV_MAXV + i] = t0;
            st->R[c * SYLV_MAXV + i] = t0;
        }
        const T hn = gs.col[c + 1];
        const double hnr = re(hn);
        double cr;
        T sr;
        givens(carry, hn, cr, sr);
        st->cs[c] = cr;
        st->sn[c] = sr;
        const T rcc = cr * carry + sr * hn;
        gs.R[c * SYLV_MAXV + c] = rcc;
        st->R[c * SYLV_MAXV + c] = rcc;
        const T gc = gs.g[c];
        const T gc1 = -(conjg(sr) * gc);
        st->g[c + 1] = gc1;
        st->g[c] = cr * gc;
        gs.g[c] = cr * gc;
        const double est = absv(gc1);
        const int iters = st->iters + 1;
        st->est = est;
        st->iters = iters;
        if (sd.hist && iters - 1 < sd.hist_cap) sd.hist[iters - 1] = est;
        int e;
        if (!isfinite(est) || !isfinite(hnr)) {
            st->status = ST_NONFINITE;
            st->nvec = 0;
            st->phase = PH_UPDATE;
            e = 2;
        } else if (est <= st->tol || c + 1 >= sd.restart || iters >= st->max_iters || hnr == 0.0) {
            st->nvec = c + 1;
            e = 1;
        } else {
            e = 0;
        }
        if (e != 0) st->upd = 0;
        st->gpend = 0;
        s_end = e;
    } else if (threadIdx.x == 0) {
        s_end = 0;
    }
    if (jn >= 0 && threadIdx.x >= 32) {
        // first pass of column jn: row i = (t - 32) / 4, columns c' = part, part + 4, ...
        const int t = threadIdx.x - 32, i = t >> 2, part = t & 3;
        T hs = zero<T>();
        if (i <= jn)
            for (int q = (i > 0 ? i - 1 : 0) + part; q < jn; q += 4) hs += gs.H[q * SYLV_MAXV + i] * gs.fs[q];
        hs += shfl_xor(hs, 1);
        hs += shfl_xor(hs, 2);
        if (part == 0 && i <= jn) {
            const T zi = i < jn ? st->fz[i] : st->fvy;
            st->h1[i] = st->fib * (zi - hs);
        }
        if (t == 0) st->h1pend = 0;
    }
    __syncthreads();
    if (s_end != 1 || threadIdx.x >= 32) return;
    // end of the cycle: back substitution R y = g, lane l owns g[l]; the
    // reciprocals of the diagonal are formed first, in parallel
    const int lane = threadIdx.x;
    const int k = c + 1;
    T gl = lane < k ? gs.g[lane] : zero<T>();
    const T rll = lane < k ? gs.R[lane * SYLV_MAXV + lane] : zero<T>();
    const T rinv = absv(rll) != 0.0 ? sdiv(make_scalar<T>(1.0, 0.0), rll) : zero<T>();
    T yl = zero<T>();
    for (int i = k - 1; i >= 0; --i) {
        const T yi = shfl_idx(gl, i) * shfl_idx(rinv, i);
        if (lane == i) yl = yi;
        if (lane < i) gl -= gs.R[i * SYLV_MAXV + lane] * yi;
    }
    if (lane < k) st->y[lane] = gs.scale[lane] * yl;
    __syncwarp();
    if (lane == 0) st->phase = PH_UPDATE;
}

template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK, (SweepOcc<C>::value > 1 && sizeof(C) == 4) ? 2 : 1)
k_dcgs_a(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts, const OpDesc* __restrict__ ops,
         const Item* __restrict__ items, BatchCtl* ctl) {
    typedef typename RealOf<C>::type CR;
    __shared__ T red[SYLV_NWARP][PSTRIDE];
    pdl_wait();
    count_launch(ctl, K_SPMV);
    if (ctl->graph && blockIdx.x == 0 && threadIdx.x == 0) {
        cudaGraphSetConditional(ctl->h_loop, 0u);
        if (ctl->bouter) cudaGraphSetConditional(ctl->h_bouter, 0u);
    }
    const Item it = items[blockIdx.x];
    SysState<T>* st = sts + it.sys;
    if (st->phase != PH_ARNOLDI) return;
    const SysDesc<T, S, C> sd = sysd[it.sys];
    const OpDesc op = ops[sd.op];
    const int j = st->j;
    const bool product = j < sd.restart;
    const double sj = st->scale[j];
    const int r0 = it.chunk * sd.rows_per_chunk;
    const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
    count_work(ctl, K_SPMV, it.chunk,
               (product ? (double)op.nnz * sizeof(C) + (double)sd.n * (sizeof(S) + sizeof(C)) : 0.0) +
                   (double)(j + 1) * sd.n * sizeof(S),
               FmaFlops<C>::v * ((product ? (double)op.nnz : 0.0) + (2.0 * j + 2.0) * sd.n));
    T* out = sd.part + (size_t)it.chunk * PSTRIDE;
#define SYLV_DCGSA_CALL(NV) dcgs_a_rows<NV, T, S, C>(sd, op, st, j, product, (CR)sj, r0, r1, out, red)
    if (j == 0) {
        SYLV_DCGSA_CALL(4);
    } else {
        SYLV_BUCKET_SWITCH(j - 1, SYLV_DCGSA_CALL)
    }
#undef SYLV_DCGSA_CALL
    pdl_trigger();
    if (!last_block(&st->counter, sd.nchunks)) return;
    dcgs_step_tail<T, S, C>(sd, st, j, sj);
}

// Rows [r0, r1) of sweep b: X_j <- sj U - sum_l a_l X_l, slot j+1 <- Y - sum_l c_l X_l - cv X_j.
template <int NV, typename T, typename S, typename C>
__device__ __forceinline__ void dcgs_b_rows(const SysDesc<T, S, C>& sd, int jb, C su, const C* ca, const C* cz, C cv,
                                            int r0, int r1) {
    typedef BasisIx<1> BI;
    S* __restrict__ V = sd.V;
    const C* __restrict__ w = sd.w;
    auto body = [&](int i, const C uv, const C wv, auto vl) {
        C xn = su * uv;
        C un = wv;
#pragma unroll
        for (int l = 0; l < NV; ++l) {
            if (l < jb) {
                const C xl = cvt<C>(vl(l));
                xn -= ca[l] * xl;
                un -= cz[l] * xl;
            }
        }
        const S xs = cvt<S>(xn);
        un -= cv * cvt<C>(xs);
        const size_t ri = BI::row(sd, i);
        V[ri + BI::vec(sd, jb)] = xs;
        V[ri + BI::vec(sd, jb + 1)] = cvt<S>(un);
    };
    if constexpr (Staged<S, C>::value) {
        stream_tiles<NV + 1, S, C>(V, sd.tstride, w, r0 >> 5, (r1 + 31) >> 5, r1, jb + 1,
                                   [&](int i, const S* sv, C wv) {
                                       body(i, cvt<C>(sv[32 * jb]), wv, [&](int l) { return sv[32 * l]; });
                                   });
    } else {
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const S* __restrict__ vr = V + BI::row(sd, i);
            body(i, cvt<C>(vr[BI::vec(sd, jb)]), w[i], [&](int l) { return vr[BI::vec(sd, l)]; });
        }
    }
}

// Grid: nsys Givens blocks (block q < nsys serves system q), then one block
// per work item for the sweep.
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK, SweepOcc<C>::value)
k_dcgs_b(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts, const Item* __restrict__ items,
         BatchCtl* ctl, int nsys) {
    pdl_wait();
    count_launch(ctl, K_CGS3);
    if ((int)blockIdx.x < nsys) {
        SysState<T>* sg = sts + blockIdx.x;
        if (sg->gpend > 0 || sg->h1pend > 0) dcgs_givens<T, S, C>(sysd[blockIdx.x], sg);
        if (ctl->graph) graph_tail<T>(ctl, sts, K_CGS3);
        return;
    }
    const Item it = items[blockIdx.x - nsys];
    SysState<T>* st = sts + it.sys;
    if (st->phase == PH_ARNOLDI && st->upd) {
        const SysDesc<T, S, C> sd = sysd[it.sys];
        const int jb = st->jb;
        __shared__ C ca[SYLV_MAXV], cz[SYLV_MAXV];
        for (int l = threadIdx.x; l < jb; l += blockDim.x) {
            ca[l] = cvt<C>(st->h2[l]);
            cz[l] = cvt<C>(st->cz[l]);
        }
        const C su = cvt<C>(make_scalar<T>(st->sjb, 0.0));
        const C cv = cvt<C>(st->cv);
        count_work(ctl, K_CGS3, it.chunk, (double)(jb + 1) * sd.n * sizeof(S) + (double)sd.n * (sizeof(C) + 2 * sizeof(S)),
                   FmaFlops<C>::v * (2.0 * jb + 2.0) * sd.n);
        __syncthreads();
        const int r0 = it.chunk * sd.rows_per_chunk;
        const int r1 = min(sd.n, r0 + sd.rows_per_chunk);
#define SYLV_DCGSB_CALL(NV) dcgs_b_rows<NV, T, S, C>(sd, jb, su, ca, cz, cv, r0, r1)
        if (jb == 0) {
            SYLV_DCGSB_CALL(4);
        } else {
            SYLV_BUCKET_SWITCH(jb - 1, SYLV_DCGSB_CALL)
        }
#undef SYLV_DCGSB_CALL
    }
    if (ctl->graph) graph_tail<T>(ctl, sts, K_CGS3);
}

// ---------------------------------------------------------------------------
// Restart, part 1: x += P^{-1} sum_l y_l V_l  (y already carries the scales).
// The combination is formed in the sweep precision C, the update in float64.
// ---------------------------------------------------------------------------
// The restart kernels run every device iteration but have work only when a
// cycle ends: a grid of a few blocks per SM strides over the work items, so
// an idle launch is cheap.
template <typename T, typename S, typename C>
__device__ __forceinline__ void restart_update_item(const SysDesc<T, S, C>* __restrict__ sysd,
                                                    SysState<T>* __restrict__ sts, const Item it, BatchCtl* ctl) {
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

template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_restart_update(const SysDesc<T, S, C>* __restrict__ sysd, SysState<T>* __restrict__ sts,
                 const Item* __restrict__ items, BatchCtl* ctl) {
    pdl_wait();
    count_launch(ctl, K_RUPD);
    const int ni = ctl->nitems;
    for (int q = blockIdx.x; q < ni; q += gridDim.x) {
        restart_update_item<T, S, C>(sysd, sts, items[q], ctl);
        __syncthreads();          // shared coefficients are rewritten by the next item
    }
}

// ---------------------------------------------------------------------------
// Restart, part 2: r = b - (Op + sigma I) x (float64), V_0 = r, ||r||, then
// the decision: converged / iteration cap / non-finite -> done, else a new
// cycle with v_0 = r / ||r||.
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
__device__ __forceinline__ void restart_residual_item(const SysDesc<T, S, C>* __restrict__ sysd,
                                                      SysState<T>* __restrict__ sts,
                                                      const OpDesc* __restrict__ ops, const Item it, BatchCtl* ctl) {
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
            st->upd = 0;
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
    pdl_wait();
    count_launch(ctl, K_RRES);
    const int ni = ctl->nitems;
    for (int q = blockIdx.x; q < ni; q += gridDim.x) {
        restart_residual_item<T, S, C>(sysd, sts, ops, items[q], ctl);
        __syncthreads();          // shared reduction buffers are reused by the next item
    }
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
        if (pinv) pinv[i] = sdiv(make_scalar<T>(1.0, 0.0), shifted_diag(op, i, sigma));
        if (!aval) continue;
        for (int d = 0; d < op.ndiag; ++d) {
            const int k = i + op.offs[d];
            T a = zero<T>();
            if (k >= 0 && k < op.n) {
                a = make_scalar<T>(op.dval[(size_t)d * op.n + i], 0.0);
                if (op.mval) a = a + sigma * op.mval[(size_t)d * op.n + i];
                else if (op.offs[d] == 0) a = a + sigma;
                if (pinv) a = a * sdiv(make_scalar<T>(1.0, 0.0), shifted_diag(op, k, sigma));
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
