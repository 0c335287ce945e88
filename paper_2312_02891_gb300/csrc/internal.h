// internal.h - host-side declarations shared by the translation units of the
// solver library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>
#include "../../include/sylv_adi.h"
#include "common.cuh"

namespace sylv {

void set_error(const char* fmt, ...);

#define SYLV_CK(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::sylv::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                              __FILE__, __LINE__);                                      \
            return SYLV_ERR_CUDA;                                                       \
        }                                                                               \
    } while (0)

#define SYLV_TRY(expr)            \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != SYLV_OK) return rc_; \
    } while (0)

// Host copy of a validated CSR matrix.
struct HostCsr {
    int n = 0;
    std::vector<int> rp, ci;
    std::vector<double> v;
};

int load_csr(const sylv_csr* c, HostCsr& out);
void transpose_csr(const HostCsr& a, HostCsr& t);

// Device operator owned by a sylv_op.
struct DevOp {
    OpDesc desc{};
    int is_stencil = 0;
    int has_mass = 0;
    double* d_dval = nullptr;
    int* d_rp = nullptr;
    int* d_ci = nullptr;
    double* d_v = nullptr;
    double* d_diag = nullptr;
    double* d_mval = nullptr;       // mass by diagonals
    int* d_mrp = nullptr;           // mass in CSR
    int* d_mci = nullptr;
    double* d_mv = nullptr;
    double* d_mdiag = nullptr;
    // the operator, and optionally the mass matrix of Op + sigma Mass (same size)
    int upload(const HostCsr& h, const HostCsr* mass = nullptr);
    void release();
};

int num_sms();

// Type-erased entry points implemented for double (real shifts) and cplx.
struct AdiBase {
    virtual ~AdiBase() {}
    virtual int solve() = 0;
    virtual int set_rhs(const double* f, const double* g, int on_device) = 0;
    virtual int info(sylv_info* out) const = 0;
    virtual int history(double* buf, int cap, int* rows) const = 0;
    virtual int factors(void* Z, void* Y, void* gamma, int on_device, int* kr) const = 0;
    virtual int profile(int on) = 0;
    virtual int kernel_stats(double* ms, double* bytes, double* flops, long long* launches) const = 0;
    virtual int core(double* G, int ld, int* kr) const = 0;
    virtual int is_real() const = 0;     // factors are real (real shifts or real double steps)
    virtual int tuning(int* chosen, int* cand, double* ms, int cap, int* count) const = 0;
};

struct AdiArgs {
    const DevOp* A;
    const DevOp* Bt;
    int n, m, r;
    const double* f;
    const double* g;
    const sylv_shift* alpha;
    const sylv_shift* beta;
    int nshift;
    double tau;
    sylv_opts o;
    cudaStream_t stream;
};

// One instance of a batched solve; the operators are owned by the batch
// handle.  dminA/dminB/fixed_tol are the options resolved for this instance's
// tolerance.
struct BatchProb {
    const DevOp* A;
    const DevOp* Bt;
    int n, m, r;
    const double* f;
    const double* g;
    const sylv_shift* alpha;
    const sylv_shift* beta;
    int nshift;
    double tau;
    double dminA, dminB, fixed_tol;
};

struct BatchBase {
    virtual ~BatchBase() {}
    virtual int solve() = 0;
    virtual int info(int i, sylv_info* out) const = 0;
    virtual int history(int i, double* buf, int cap, int* rows) const = 0;
    virtual int factors(int i, void* Z, void* Y, void* gamma, int on_device, int* kr) const = 0;
    virtual int stats(long long* launches, double* bytes, double* flops, long long* ticks) const = 0;
    virtual int profile(int on) = 0;
    virtual int kernel_stats(double* ms, double* bytes, double* flops, long long* launches) const = 0;
    virtual int set_rhs(int i, const double* f, const double* g) = 0;
    virtual int tuning(int* chosen, int* cand, double* ms, int cap, int* count) const = 0;
};

// One instantiation per (shift type, precision): r = real shifts, c = complex
// shifts; 64/128 = float64 throughout, 32/64 = float32 basis and sweeps,
// bf = bfloat16 basis with float32 sweeps.
#define SYLV_DECL_INST(SUFFIX)                                                                      \
    int make_adi_##SUFFIX(const AdiArgs& a, AdiBase** out);                                         \
    int gmres_##SUFFIX(const DevOp& op, sylv_shift sigma, int jacobi, const void* B, void* X,       \
                       int ncols, double tol, int restart, int max_iters, int* iters, double* res, \
                       double* hist, cudaStream_t s);                                                \
    int arnoldi_##SUFFIX(const DevOp& op, sylv_shift sigma, int jacobi, const void* v0, int k, int ortho, \
                         void* V_out, void* H_out, cudaStream_t s);                                \
    int bicgstab_##SUFFIX(const DevOp& op, sylv_shift sigma, int jacobi, const void* B, void* X,    \
                          int ncols, double tol, int max_iters, int* iters, double* res, double* hist, \
                          cudaStream_t s);                                                          \
    int make_batch_##SUFFIX(const std::vector<BatchProb>& ps, const sylv_opts& o, cudaStream_t s,      \
                            BatchBase** out);
SYLV_DECL_INST(r64)
SYLV_DECL_INST(r32)
SYLV_DECL_INST(rbf)
SYLV_DECL_INST(c128)
SYLV_DECL_INST(c64)
SYLV_DECL_INST(cbf)
#undef SYLV_DECL_INST
int cgs2_real(const void* V, int n, int k, void* w, void* h, cudaStream_t s);
int cgs2_cplx(const void* V, int n, int k, void* w, void* h, cudaStream_t s);
int op_apply_real(const DevOp& op, double sigma, int jacobi, const void* X, void* Y, int ncols, cudaStream_t s);
int op_apply_cplx(const DevOp& op, sylv_shift sigma, int jacobi, const void* X, void* Y, int ncols, cudaStream_t s);
int controller_eval_dev(const sylv_opts* o, int count, const double* in, double* out);

}  // namespace sylv

struct sylv_op {
    sylv::DevOp op;
};

struct sylv_batch {
    sylv::BatchBase* impl = nullptr;
    std::vector<sylv::DevOp> ops;     // A_i, B_i^T for instance i at 2i, 2i + 1
    int count = 0;
    int is_complex = 0;
    cudaStream_t stream = nullptr;
};

struct sylv_handle {
    sylv::AdiBase* impl = nullptr;
    sylv::DevOp A, Bt;
    int is_complex = 0;
    int solved = 0;
    int last_status = SYLV_ERR_NOT_SOLVED;
    cudaStream_t stream = nullptr;
};
