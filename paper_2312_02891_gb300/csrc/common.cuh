// common.cuh - scalar types, descriptors and reduction helpers shared by the
// device code of the inexact LR-ADI solver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#ifndef SYLV_MR
#define SYLV_MR 30                 // maximum GMRES restart length
#endif
#define SYLV_MAXV (SYLV_MR + 1)    // basis vectors per cycle
#define SYLV_MAXDIAG 8             // diagonals of a stencil-stored operator
#define SYLV_BLOCK 256             // threads per block of the vector kernels
#define SYLV_NWARP (SYLV_BLOCK / 32)

namespace sylv {

// ---------------------------------------------------------------------------
// Scalars: double (real shifts) and cplx (complex shifts).  cplx is laid out
// as two doubles, 16-byte aligned, so complex vectors are interleaved pairs.
// ---------------------------------------------------------------------------
struct __align__(16) cplx { double x, y; };

__host__ __device__ __forceinline__ double re(double a) { return a; }
__host__ __device__ __forceinline__ double re(cplx a) { return a.x; }
__host__ __device__ __forceinline__ double im(double) { return 0.0; }
__host__ __device__ __forceinline__ double im(cplx a) { return a.y; }
__host__ __device__ __forceinline__ double conjg(double a) { return a; }
__host__ __device__ __forceinline__ cplx conjg(cplx a) { return {a.x, -a.y}; }
__host__ __device__ __forceinline__ double abs2(double a) { return a * a; }
__host__ __device__ __forceinline__ double abs2(cplx a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ cplx operator+(cplx a, cplx b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a, cplx b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a) { return {-a.x, -a.y}; }
__host__ __device__ __forceinline__ cplx operator+(double a, cplx b) { return {a + b.x, b.y}; }
__host__ __device__ __forceinline__ cplx operator+(cplx a, double b) { return {a.x + b, a.y}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, cplx b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ __forceinline__ cplx operator*(double s, cplx a) { return {s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, double s) { return {s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ cplx& operator+=(cplx& a, cplx b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ __forceinline__ cplx& operator-=(cplx& a, cplx b) { a.x -= b.x; a.y -= b.y; return a; }
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    // a / b by Smith's method (R. L. Smith, CACM 1962) to avoid overflow.
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return {(a.x + a.y * r) / d, (a.y - a.x * r) / d};
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return {(a.x * r + a.y) / d, (a.y * r - a.x) / d};
    }
}
__host__ __device__ __forceinline__ double sdiv(double a, double b) { return a / b; }
__host__ __device__ __forceinline__ cplx sdiv(cplx a, cplx b) { return cdiv(a, b); }

template <typename T> __host__ __device__ __forceinline__ T make_scalar(double r, double i);
template <> __host__ __device__ __forceinline__ double make_scalar<double>(double r, double) { return r; }
template <> __host__ __device__ __forceinline__ cplx make_scalar<cplx>(double r, double i) { return {r, i}; }
template <typename T> __host__ __device__ __forceinline__ T zero() { return make_scalar<T>(0.0, 0.0); }

// conj(a) * b
__host__ __device__ __forceinline__ double cmul(double a, double b) { return a * b; }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}

__device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ cplx shfl_xor(cplx v, int m) {
    return {__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += shfl_xor(v, m);
    return v;
}
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ cplx ldcg(const cplx* p) {
    double2 v = __ldcg(reinterpret_cast<const double2*>(p));
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
};

// y_i = sum_j Op[i][j] * X(j) + sigma * X(i), X(k) supplied by the caller.
template <typename T, typename XF>
__device__ __forceinline__ T op_row(const OpDesc& op, int i, T sigma, XF X) {
    T acc = zero<T>();
    if (op.fmt == 1) {
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
    }
    return acc + sigma * X(i);
}

// ---------------------------------------------------------------------------
// One shifted system solved by restarted GMRES: descriptor (fixed for a
// batch) and state (changed by the kernels).
// ---------------------------------------------------------------------------
enum Phase : int { PH_DONE = 0, PH_ARNOLDI = 1, PH_UPDATE = 2, PH_RESID = 3 };
enum SysStatus : int { ST_OK = 0, ST_STALL = 1, ST_NONFINITE = 2 };

template <typename T>
struct SysDesc {
    int n;
    int op;                 // index into the batch's operator table
    int nchunks;            // work units of this system
    int rows_per_chunk;
    size_t ldv;             // stride between basis vectors
    T* V;                   // (restart + 1) basis vectors, stored unnormalised
    T* w;                   // Arnoldi work vector (operator output)
    T* part;                // nchunks x SYLV_MAXV+1 partial sums
    const T* pinv;          // Jacobi: 1 / (diag + sigma), or null
    double* hist;           // optional: Givens estimate per Arnoldi step
    int hist_cap;
    int restart;
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
};

// Work item of a launch: (system, chunk).
struct Item { int sys; int chunk; };

// Per-batch device control block.
struct BatchCtl {
    int n_active;           // systems not yet done
    int ticks;
    int* h_flag;            // mapped host word set to 0 when n_active reaches 0
};

}  // namespace sylv
