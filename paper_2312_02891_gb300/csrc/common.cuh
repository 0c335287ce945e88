// common.cuh - scalar types, conversions, descriptors and reduction helpers
// shared by the device code of the inexact LR-ADI solver.
//
// Three scalar roles appear in the templates:
//   T  the float64 type of the outer iteration, the true residuals, the
//      solutions and the Hessenberg least squares (double or cplx);
//   S  the storage type of the Krylov basis (double, float or bf16, and their
//      complex pairs);
//   C  the arithmetic type of the basis sweeps and the preconditioned
//      operator product (double or float, and complex pairs).
// The float64 path is T = S = C; the mixed path keeps T in float64 and runs
// the sweeps in float32 (the inner solves may be inexact, Sec. 3).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <math.h>

#ifndef SYLV_MR
#define SYLV_MR 30                 // maximum GMRES restart length
#endif
#define SYLV_MAXV (SYLV_MR + 1)    // basis vectors per cycle
#define SYLV_MAXDIAG 9             // diagonals of a stencil-stored operator (2D Q1 mass: 9)
#define SYLV_BLOCK 256             // threads per block of the vector kernels
#define SYLV_NWARP (SYLV_BLOCK / 32)

namespace sylv {

// ---------------------------------------------------------------------------
// Scalars.  Complex types are interleaved (re, im) pairs.
// ---------------------------------------------------------------------------
struct __align__(16) cplx { double x, y; };
struct __align__(8) cflt { float x, y; };
struct __align__(4) cbf16 { __nv_bfloat16 x, y; };
typedef __nv_bfloat16 bf16;

#define HD __host__ __device__ __forceinline__

HD double re(double a) { return a; }
HD double re(cplx a) { return a.x; }
HD float re(float a) { return a; }
HD float re(cflt a) { return a.x; }
HD double im(double) { return 0.0; }
HD double im(cplx a) { return a.y; }
HD double conjg(double a) { return a; }
HD cplx conjg(cplx a) { return {a.x, -a.y}; }
HD float conjg(float a) { return a; }
HD cflt conjg(cflt a) { return {a.x, -a.y}; }
HD double abs2(double a) { return a * a; }
HD double abs2(cplx a) { return a.x * a.x + a.y * a.y; }
HD float abs2(float a) { return a * a; }
HD float abs2(cflt a) { return a.x * a.x + a.y * a.y; }

HD cplx operator+(cplx a, cplx b) { return {a.x + b.x, a.y + b.y}; }
HD cplx operator-(cplx a, cplx b) { return {a.x - b.x, a.y - b.y}; }
HD cplx operator-(cplx a) { return {-a.x, -a.y}; }
HD cplx operator+(double a, cplx b) { return {a + b.x, b.y}; }
HD cplx operator+(cplx a, double b) { return {a.x + b, a.y}; }
HD cplx operator*(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
HD cplx operator*(double s, cplx a) { return {s * a.x, s * a.y}; }
HD cplx operator*(cplx a, double s) { return {s * a.x, s * a.y}; }
HD cplx& operator+=(cplx& a, cplx b) { a.x += b.x; a.y += b.y; return a; }
HD cplx& operator-=(cplx& a, cplx b) { a.x -= b.x; a.y -= b.y; return a; }

HD cflt operator+(cflt a, cflt b) { return {a.x + b.x, a.y + b.y}; }
HD cflt operator-(cflt a, cflt b) { return {a.x - b.x, a.y - b.y}; }
HD cflt operator-(cflt a) { return {-a.x, -a.y}; }
HD cflt operator*(cflt a, cflt b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
HD cflt operator*(float s, cflt a) { return {s * a.x, s * a.y}; }
HD cflt operator*(cflt a, float s) { return {s * a.x, s * a.y}; }
HD cflt& operator+=(cflt& a, cflt b) { a.x += b.x; a.y += b.y; return a; }
HD cflt& operator-=(cflt& a, cflt b) { a.x -= b.x; a.y -= b.y; return a; }

HD cplx to_cplx(double a) { return {a, 0.0}; }
HD cplx to_cplx(cplx a) { return a; }

HD cplx cdiv(cplx a, cplx b) {
    // a / b by Smith's method (R. L. Smith, CACM 1962) to avoid overflow.
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return {(a.x + a.y * r) / d, (a.y - a.x * r) / d};
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return {(a.x * r + a.y) / d, (a.y * r - a.x) / d};
    }
}
HD double sdiv(double a, double b) { return a / b; }
HD cplx sdiv(cplx a, cplx b) { return cdiv(a, b); }

template <typename T> HD T make_scalar(double r, double i);
template <> HD double make_scalar<double>(double r, double) { return r; }
template <> HD cplx make_scalar<cplx>(double r, double i) { return {r, i}; }
template <> HD float make_scalar<float>(double r, double) { return (float)r; }
template <> HD cflt make_scalar<cflt>(double r, double i) { return {(float)r, (float)i}; }
template <typename T> HD T zero() { return make_scalar<T>(0.0, 0.0); }

// conj(a) * b
HD double cmul(double a, double b) { return a * b; }
HD cplx cmul(cplx a, cplx b) { return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }
HD float cmul(float a, float b) { return a * b; }
HD cflt cmul(cflt a, cflt b) { return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }

// real part type of a scalar (the type of scale factors in its arithmetic)
template <typename X> struct RealOf { typedef X type; };
template <> struct RealOf<cplx> { typedef double type; };
template <> struct RealOf<cflt> { typedef float type; };

// Resident blocks per SM the basis sweeps are compiled for.  The 32-bit
// sweeps are latency-bound (they need many loads in flight per SM, so more
// resident warps); the float64 sweeps are bound by the float64 pipe and keep
// their registers.
template <typename C> struct SweepOcc { static constexpr int value = 1; };
template <> struct SweepOcc<float> { static constexpr int value = 3; };
template <> struct SweepOcc<cflt> { static constexpr int value = 2; };

// ---------------------------------------------------------------------------
// Conversions between the roles (storage <-> arithmetic <-> float64).
// ---------------------------------------------------------------------------
template <typename To, typename From> struct Cvt;
template <typename X> struct Cvt<X, X> { static HD X f(X a) { return a; } };
template <> struct Cvt<float, double> { static HD float f(double a) { return (float)a; } };
template <> struct Cvt<double, float> { static HD double f(float a) { return (double)a; } };
template <> struct Cvt<cflt, cplx> { static HD cflt f(cplx a) { return {(float)a.x, (float)a.y}; } };
template <> struct Cvt<cplx, cflt> { static HD cplx f(cflt a) { return {(double)a.x, (double)a.y}; } };
template <> struct Cvt<float, bf16> { static __device__ __forceinline__ float f(bf16 a) { return __bfloat162float(a); } };
template <> struct Cvt<bf16, float> { static __device__ __forceinline__ bf16 f(float a) { return __float2bfloat16_rn(a); } };
template <> struct Cvt<double, bf16> { static __device__ __forceinline__ double f(bf16 a) { return (double)__bfloat162float(a); } };
template <> struct Cvt<bf16, double> { static __device__ __forceinline__ bf16 f(double a) { return __double2bfloat16(a); } };
template <> struct Cvt<cflt, cbf16> {
    static __device__ __forceinline__ cflt f(cbf16 a) { return {__bfloat162float(a.x), __bfloat162float(a.y)}; }
};
template <> struct Cvt<cbf16, cflt> {
    static __device__ __forceinline__ cbf16 f(cflt a) { return {__float2bfloat16_rn(a.x), __float2bfloat16_rn(a.y)}; }
};
template <> struct Cvt<cplx, cbf16> {
    static __device__ __forceinline__ cplx f(cbf16 a) {
        return {(double)__bfloat162float(a.x), (double)__bfloat162float(a.y)};
    }
};
template <> struct Cvt<cbf16, cplx> {
    static __device__ __forceinline__ cbf16 f(cplx a) { return {__double2bfloat16(a.x), __double2bfloat16(a.y)}; }
};
template <typename To, typename From> __device__ __forceinline__ To cvt(From a) { return Cvt<To, From>::f(a); }

// ---------------------------------------------------------------------------
// Warp reductions and cache-bypassing loads.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ cplx shfl_xor(cplx v, int m) {
    return {__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}
__device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ cflt shfl_xor(cflt v, int m) {
    return {__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}
__device__ __forceinline__ double shfl_idx(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ cplx shfl_idx(cplx v, int src) {
    return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}
template <typename X> __device__ __forceinline__ X warp_sum(X v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += shfl_xor(v, m);
    return v;
}
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ cplx ldcg(const cplx* p) {
    double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}
// Loads through the read-only (non-coherent) path: for data that no thread of
// the kernel writes, or that only the loading thread overwrites afterwards.
// They let the compiler move the next row's loads ahead of this row's stores.
__device__ __forceinline__ float ldro(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ldro(const double* p) { return __ldg(p); }
__device__ __forceinline__ cflt ldro(const cflt* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cplx ldro(const cplx* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}

// ---------------------------------------------------------------------------
// Sparse operator: stored by diagonals (finite-difference stencils) or CSR.
// ---------------------------------------------------------------------------
struct OpDesc {
    int n;
    int fmt;                        // 1 = by diagonals, 0 = CSR
    int ndiag;
    int offs[SYLV_MAXDIAG];         // column offset of each stored diagonal
    const double* dval;             // ndiag x n: dval[d*n + i] = Op[i][i + offs[d]]
    const int* rowptr;              // CSR
    const int* colind;
    const double* val;
    const double* diag;             // main diagonal (Jacobi)
    long long nnz;                  // nonzeros of the matrix (algorithmic byte counts)
    // mass matrix of the generalized equation (eq. (gsylv)): the shifted
    // operator is Op + sigma Mass; all null for Mass = I
    const double* mval;             // by diagonals, on the offsets of the operator (fmt 1)
    const int* mrowptr;             // CSR (fmt 0)
    const int* mcolind;
    const double* mvalc;
    const double* mdiag;            // main diagonal of Mass (Jacobi)
    long long mnnz;
};

// y_i = sum_j Op[i][j] * X(j) + sigma * (Mass X)(i), X(k) supplied by the
// caller (Mass = I unless the operator carries a mass matrix).
template <typename T, typename XF>
__device__ __forceinline__ T op_row(const OpDesc& op, int i, T sigma, XF X) {
    T acc = zero<T>();
    if (op.fmt == 1) {
        if (op.mval) {
            T macc = zero<T>();
#pragma unroll
            for (int d = 0; d < SYLV_MAXDIAG; ++d) {
                if (d < op.ndiag) {
                    int k = i + op.offs[d];
                    if (k >= 0 && k < op.n) {
                        const T x = X(k);
                        acc += op.dval[(size_t)d * op.n + i] * x;
                        macc += op.mval[(size_t)d * op.n + i] * x;
                    }
                }
            }
            return acc + sigma * macc;
        }
#pragma unroll
        for (int d = 0; d < SYLV_MAXDIAG; ++d) {
            if (d < op.ndiag) {
                int k = i + op.offs[d];
                if (k >= 0 && k < op.n) acc += op.dval[(size_t)d * op.n + i] * X(k);
            }
        }
    } else {
        int p0 = op.rowptr[i], p1 = op.rowptr[i + 1];
        for (int p = p0; p < p1; ++p) acc += op.val[p] * X(op.colind[p]);
        if (op.mvalc) {
            T macc = zero<T>();
            for (int p = op.mrowptr[i]; p < op.mrowptr[i + 1]; ++p) macc += op.mvalc[p] * X(op.mcolind[p]);
            return acc + sigma * macc;
        }
    }
    return acc + sigma * X(i);
}

// (Mass X)(i) (X(i) when the operator carries no mass matrix).
template <typename T, typename XF>
__device__ __forceinline__ T mass_row(const OpDesc& op, int i, XF X) {
    if (op.fmt == 1 && op.mval) {
        T acc = zero<T>();
#pragma unroll
        for (int d = 0; d < SYLV_MAXDIAG; ++d) {
            if (d < op.ndiag) {
                int k = i + op.offs[d];
                if (k >= 0 && k < op.n) acc += op.mval[(size_t)d * op.n + i] * X(k);
            }
        }
        return acc;
    }
    if (op.fmt == 0 && op.mvalc) {
        T acc = zero<T>();
        for (int p = op.mrowptr[i]; p < op.mrowptr[i + 1]; ++p) acc += op.mvalc[p] * X(op.mcolind[p]);
        return acc;
    }
    return X(i);
}

// diag(Op) + sigma diag(Mass) at row i: the Jacobi preconditioner.
template <typename T>
__device__ __forceinline__ T shifted_diag(const OpDesc& op, int i, T sigma) {
    return op.diag[i] + sigma * (op.mdiag ? op.mdiag[i] : 1.0);
}

// ---------------------------------------------------------------------------
// One shifted system solved by restarted GMRES: descriptor (fixed for a
// batch) and state (changed by the kernels).
// ---------------------------------------------------------------------------
enum Phase : int { PH_DONE = 0, PH_ARNOLDI = 1, PH_UPDATE = 2, PH_RESID = 3 };
enum SysStatus : int { ST_OK = 0, ST_STALL = 1, ST_NONFINITE = 2 };

template <typename T, typename S, typename C>
struct SysDesc {
    int n;
    int op;                 // index into the batch's operator table
    int nchunks;            // work units of this system
    int rows_per_chunk;
    size_t ldv;             // column-major basis: stride between basis vectors
    size_t tstride;         // tile-major basis: elements per 32-row tile (32 x vectors)
    S* V;                   // (restart + 1) basis vectors, stored unnormalised
    C* w;                   // Arnoldi work vector (operator output)
    T* part;                // nchunks x PSTRIDE partial sums
    const T* pinv;          // Jacobi: 1 / (diag + sigma), or null
    const C* aval;          // stencil operators: (Op + sigma I) P^{-1} by diagonals, C precision
    double* hist;           // optional: Givens estimate (GMRES) or recurrence residual (BiCGstab) per step
    int hist_cap;
    int restart;
    C* bv;                  // BiCGstab: the system's vectors (BVec order), ldv apart; null for GMRES
    const C* rres;          // BiCGstab: the last true residual (column-major); null: slot 0 of V
};

// Basis addressing.  Tile-major (LAY 1, the solver's own basis): rows are
// grouped in tiles of 32, and a tile stores its 32 rows of every basis vector
// contiguously, so the loads of one warp for all vectors of a row tile fall
// in one small contiguous range (one page, not one page per vector) and the
// per-vector offsets are compile-time constants off a single base pointer.
// Column-major (LAY 0): vectors ldv apart, for callers' own buffers.
template <int LAY> struct BasisIx;
template <> struct BasisIx<0> {
    template <class D> __device__ __forceinline__ static size_t row(const D& sd, int i) { return (size_t)i; }
    template <class D> __device__ __forceinline__ static size_t vec(const D& sd, int l) { return (size_t)l * sd.ldv; }
};
template <> struct BasisIx<1> {
    template <class D> __device__ __forceinline__ static size_t row(const D& sd, int i) {
        return (size_t)(i >> 5) * sd.tstride + (size_t)(i & 31);
    }
    template <class D> __device__ __forceinline__ static size_t vec(const D&, int l) { return (size_t)l * 32; }
};

template <typename T>
struct SysState {
    int phase;
    int j;                  // index of the newest basis vector in the cycle
    int iters;              // Arnoldi steps so far
    int cycles;
    int max_iters;
    int status;
    int nvec;               // basis vectors combined at the cycle's end
    unsigned counter;       // blocks finished in the current launch
    double tol;
    double resnorm;         // true residual norm after the last cycle
    double est;             // Givens residual estimate
    double nrm2;            // reduced squared norm (scratch of the last block)
    T sigma;
    T* x;                   // solution
    const T* b;             // right-hand side
    double scale[SYLV_MAXV];     // v_l = scale[l] * V_l
    T h1[SYLV_MAXV];
    T h2[SYLV_MAXV];
    T R[SYLV_MR * SYLV_MAXV];    // rotated Hessenberg columns, R[j*MAXV + i]
    double cs[SYLV_MR];
    T sn[SYLV_MR];
    T g[SYLV_MAXV];
    T y[SYLV_MR];                // scale-folded least-squares solution
    // delayed CGS2 (DCGS2): Hessenberg columns as formed (unrotated),
    // coefficients of the pending update sweep and its step
    T Hr[SYLV_MR * SYLV_MAXV];
    T cz[SYLV_MAXV];
    T cv;
    double sjb;
    int jb;
    int upd;
    int gpend;              // delayed CGS2: Hessenberg column gpend - 1 awaits its Givens update (0: none)
    int h1pend;             // delayed CGS2: first pass of column h1pend - 1 still to form (0: none)
    double fib;             // delayed CGS2, inputs of that first pass: 1 / beta,
    T fvy;                  //   v_j^* y,
    T fs[SYLV_MAXV];        //   s = V^* u_j (scaled),
    T fz[SYLV_MAXV];        //   z = V^* y (scaled)
    // BiCGstab: rho = rhat^* r of the current residual, the step's alpha and
    // omega, beta of the next search direction; bfin: the step ended early
    // (||s|| met the tolerance, omega = 0)
    T brho, balpha, bomega, bbeta;
    int bfin;
    double bnorm0;          // BiCGstab: residual norm at the start of the cycle
};

// Work item of a launch: (system, chunk).
struct Item { int sys; int chunk; };

// Kernel ids of the per-kernel statistics.
enum KernelId : int { K_SPMV = 0, K_CGS2 = 1, K_CGS3 = 2, K_RUPD = 3, K_RRES = 4, K_CTRL = 5,
                      K_STEP = 6, K_GRAM = 7, K_COUNT = 8 };

struct BatchCtl {
    int n_active;           // systems not yet done
    int ticks;              // device iterations of the current inner loop
    int* h_flag;            // mapped host word set to 0 when n_active reaches 0
    double bytes[K_COUNT];  // algorithmic bytes moved, per kernel, summed over launches
    double flops[K_COUNT];  // algorithmic floating-point operations, same
    // device-driven CUDA graph: the kernels set the conditional nodes
    int graph;              // 1 while a graph launch drives the iteration
    int nsys;               // systems scanned by the grid-level decisions
    int max_ticks;          // cap of device iterations per inner loop
    int capped;             // inner loops stopped by the cap
    unsigned gdone[K_COUNT];               // blocks finished, per kernel (grid-level last block)
    cudaGraphConditionalHandle h_loop;     // WHILE: device iterations of the inner solves
    cudaGraphConditionalHandle h_restart;  // IF: restart kernels in this iteration
    cudaGraphConditionalHandle h_outer;    // WHILE: outer steps of Algorithm 1
    unsigned long long launch_count[K_COUNT];  // launches, counted by block 0 of each kernel
    int n_inst_open;        // batched solves: instances not finished (0 for a single solve)
    int* h_open;            // batched solves, host-driven: mapped host word cleared when n_inst_open reaches 0
    int nitems;             // work items of the batch (grid-stride kernels)
    // batched graph: IF node around the outer-step kernels, set when a column
    // system finishes (an instance may then take its outer step), cleared by
    // the first inner kernel of every device iteration
    int bouter;             // 1 when h_bouter belongs to the running graph
    cudaGraphConditionalHandle h_bouter;
    int stage_fault;        // a shared-memory staging wait gave up (the affected columns end non-finite)
    // BiCGstab work list of the device iteration (items of groups with an
    // active column) and, in a graph whose step kernels are device-updatable,
    // their node handles (the list kernel sets their grids to its length)
    int nlist;
    int dyn_grid;
    cudaGraphDeviceNode_t dn_step[3];
};

__device__ __forceinline__ void count_launch(BatchCtl* ctl, int kid) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && ctl) atomicAdd(&ctl->launch_count[kid], 1ull);
}

// Real flops of one multiply-add in the arithmetic type X (complex: 8).
template <typename X> struct FmaFlops { static constexpr double v = 2.0; };
template <> struct FmaFlops<cplx> { static constexpr double v = 8.0; };
template <> struct FmaFlops<cflt> { static constexpr double v = 8.0; };

// Chunk 0 of each system adds the system's algorithmic bytes and
// multiply-adds (converted to flops by the caller's type) for this launch.
// Algorithmic bytes and flops of a launch, added once per system (chunk 0,
// thread 0).  A macro, so that the float64 expressions are evaluated only by
// that thread: in the 32-bit kernels every thread evaluating them kept this
// GPU's small float64 pipe busy at the start of every block.
#define count_work(ctl, kid, chunk, BYTES, FLOPS)                  \
    do {                                                           \
        if ((chunk) == 0 && threadIdx.x == 0 && (ctl)) {           \
            atomicAdd(&(ctl)->bytes[kid], (double)(BYTES));        \
            atomicAdd(&(ctl)->flops[kid], (double)(FLOPS));        \
        }                                                          \
    } while (0)

}  // namespace sylv
