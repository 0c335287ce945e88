// inst_c128.cu - complex shifts, complex128 throughout (the complex
// formulation the paper keeps, Sec. 3.3 "Complex Shift Parameters"); also the
// standalone CGS2 and shifted product for complex data.
#define SYLV_SUFFIX c128
#define SYLV_T cplx
#define SYLV_S cplx
#define SYLV_C cplx
#include "inst.cuh"

namespace sylv {

int cgs2_cplx(const void* V, int n, int k, void* w, void* h, cudaStream_t s) {
    return cgs2_t<cplx>(V, n, k, w, h, s);
}

int op_apply_cplx(const DevOp& op, sylv_shift sigma, int jacobi, const void* X, void* Y, int ncols,
                  cudaStream_t s) {
    return op_apply_t<cplx>(op, cplx{sigma.re, sigma.im}, jacobi, X, Y, ncols, s);
}

}  // namespace sylv
