// inst_r64.cu - real shifts, float64 throughout; also the standalone CGS2,
// shifted product and controller entry points for real data.
#define SYLV_SUFFIX r64
#define SYLV_T double
#define SYLV_S double
#define SYLV_C double
#include "inst.cuh"

namespace sylv {

// Evaluate the controller for a list of inputs (parity tests of step a1).
__global__ void k_controller_eval(int count, int strategy, int bl_clamp, double dminA, double dmaxA,
                                  double dminB, double dmaxB, const double* in, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double* p = in + (size_t)i * 11;
    controller_eval(strategy, bl_clamp, p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7],
                    dminA, dmaxA, dminB, dmaxB, p[8], out + 3 * i, out + 3 * i + 1, out + 3 * i + 2);
}

int cgs2_real(const void* V, int n, int k, void* w, void* h, cudaStream_t s) {
    return cgs2_t<double>(V, n, k, w, h, s);
}

int op_apply_real(const DevOp& op, double sigma, int jacobi, const void* X, void* Y, int ncols,
                  cudaStream_t s) {
    return op_apply_t<double>(op, sigma, jacobi, X, Y, ncols, s);
}

int controller_eval_dev(const sylv_opts* o, int count, const double* in, double* out) {
    if (!o || !in || !out || count < 0) { set_error("controller_eval: invalid arguments"); return SYLV_ERR_INVALID; }
    if (count == 0) return SYLV_OK;
    Dev<double> din, dout;
    SYLV_TRY(din.alloc((size_t)count * 11));
    SYLV_TRY(dout.alloc((size_t)count * 3));
    SYLV_CK(cudaMemcpy(din.p, in, (size_t)count * 11 * sizeof(double), cudaMemcpyHostToDevice));
    k_controller_eval<<<(count + 127) / 128, 128>>>(count, o->strategy, o->bl_clamp, o->dmin_A, o->dmax_A,
                                                     o->dmin_B, o->dmax_B, din.p, dout.p);
    SYLV_CK(cudaGetLastError());
    SYLV_CK(cudaMemcpy(out, dout.p, (size_t)count * 3 * sizeof(double), cudaMemcpyDeviceToHost));
    return SYLV_OK;
}

}  // namespace sylv
