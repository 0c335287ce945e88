// inst.cuh - explicit instantiation of the solver for one combination of the
// float64 scalar T, the Krylov basis storage S and the sweep arithmetic C.
// Each inst_*.cu includes this header after defining SYLV_SUFFIX, SYLV_T,
// SYLV_S and SYLV_C, so the combinations compile in parallel.
#pragma once
#include "batch.cuh"

namespace sylv {

template <typename T> T shift_to(sylv_shift s);
template <> inline double shift_to<double>(sylv_shift s) { return s.re; }
template <> inline cplx shift_to<cplx>(sylv_shift s) { return cplx{s.re, s.im}; }

}  // namespace sylv

#define SYLV_CAT2(a, b) a##b
#define SYLV_CAT(a, b) SYLV_CAT2(a, b)

namespace sylv {

int SYLV_CAT(make_adi_, SYLV_SUFFIX)(const AdiArgs& a, AdiBase** out) {
    return make_adi_t<SYLV_T, SYLV_S, SYLV_C>(a, out);
}

int SYLV_CAT(make_batch_, SYLV_SUFFIX)(const std::vector<BatchProb>& ps, const sylv_opts& o, cudaStream_t s,
                                       BatchBase** out) {
    return make_batch_t<SYLV_T, SYLV_S, SYLV_C>(ps, o, s, out);
}

int SYLV_CAT(gmres_, SYLV_SUFFIX)(const DevOp& op, sylv_shift sigma, int jacobi, const void* B, void* X,
                                  int ncols, double tol, int restart, int max_iters, int* iters,
                                  double* res, double* hist, cudaStream_t s) {
    return gmres_t<SYLV_T, SYLV_S, SYLV_C>(op, shift_to<SYLV_T>(sigma), jacobi, B, X, ncols, tol, restart,
                                           max_iters, iters, res, hist, s);
}

int SYLV_CAT(arnoldi_, SYLV_SUFFIX)(const DevOp& op, sylv_shift sigma, int jacobi, const void* v0, int k, int ortho,
                                    void* V_out, void* H_out, cudaStream_t s) {
    return arnoldi_t<SYLV_T, SYLV_S, SYLV_C>(op, shift_to<SYLV_T>(sigma), jacobi, v0, k, ortho, V_out, H_out, s);
}

int SYLV_CAT(bicgstab_, SYLV_SUFFIX)(const DevOp& op, sylv_shift sigma, int jacobi, const void* B, void* X,
                                     int ncols, double tol, int max_iters, int* iters, double* res,
                                     double* hist, cudaStream_t s) {
    return bicgstab_t<SYLV_T, SYLV_S, SYLV_C>(op, shift_to<SYLV_T>(sigma), jacobi, B, X, ncols, tol, max_iters,
                                              iters, res, hist, s);
}

}  // namespace sylv
