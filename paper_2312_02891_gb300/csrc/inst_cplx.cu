// inst_cplx.cu - the solver for complex shift pairs (complex128 vectors,
// real matrices), the complex formulation the paper keeps (Sec. 3.3,
// "Complex Shift Parameters").
#include "engine.cuh"

namespace sylv {

int make_adi_cplx(const AdiArgs& a, AdiBase** out) { return make_adi_t<cplx>(a, out); }

int gmres_cplx(const DevOp& op, sylv_shift sigma, int jacobi, const void* B, void* X, int ncols,
               double tol, int restart, int max_iters, int* iters, double* res, double* hist,
               cudaStream_t s) {
    return gmres_t<cplx>(op, cplx{sigma.re, sigma.im}, jacobi, B, X, ncols, tol, restart, max_iters,
                         iters, res, hist, s);
}

int cgs2_cplx(const void* V, int n, int k, void* w, void* h, cudaStream_t s) {
    return cgs2_t<cplx>(V, n, k, w, h, s);
}

int op_apply_cplx(const DevOp& op, sylv_shift sigma, int jacobi, const void* X, void* Y, int ncols,
                  cudaStream_t s) {
    return op_apply_t<cplx>(op, cplx{sigma.re, sigma.im}, jacobi, X, Y, ncols, s);
}

}  // namespace sylv
