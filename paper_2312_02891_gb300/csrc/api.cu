// api.cu - the extern "C" boundary declared in include/sylv_adi.h.  Argument
// checking and dispatch only; every step of the solve runs in the kernels.
#include <cmath>
#include <cstring>
#include <new>
#include "internal.h"

namespace sylv {
const char* last_error_cstr();
}

using namespace sylv;

static bool shift_is_complex(sylv_shift s) { return s.im != 0.0; }

// Arguments of one problem (shared by the single and the batched create):
// sizes, tolerance, finite shifts, conjugate pairs adjacent.
static int check_problem(const double* f, const double* g, int32_t r, const sylv_shift* alpha,
                         const sylv_shift* beta, int32_t n_shifts, double tol, bool* cplx_out) {
    if (!f || !g || !alpha || !beta || n_shifts <= 0) {
        set_error("null f/g/shifts or n_shifts <= 0");
        return SYLV_ERR_INVALID;
    }
    if (r < 1 || r > SYLV_MAX_RANK) {
        set_error("rank r=%d outside 1..%d", r, SYLV_MAX_RANK);
        return r < 1 ? SYLV_ERR_INVALID : SYLV_ERR_UNSUPPORTED;
    }
    if (!(tol > 0.0 && tol < 1.0)) { set_error("tol must lie in (0, 1)"); return SYLV_ERR_INVALID; }
    bool cplx = false;
    for (int i = 0; i < n_shifts; ++i) {
        if (!std::isfinite(alpha[i].re) || !std::isfinite(alpha[i].im) || !std::isfinite(beta[i].re) ||
            !std::isfinite(beta[i].im)) {
            set_error("non-finite shift %d", i);
            return SYLV_ERR_INVALID;
        }
        cplx |= shift_is_complex(alpha[i]) || shift_is_complex(beta[i]);
    }
    if (cplx) {
        // conjugate pairs must be adjacent: a complex pair at i is followed by its conjugate
        for (int i = 0; i < n_shifts; ++i) {
            if (!(shift_is_complex(alpha[i]) || shift_is_complex(beta[i]))) continue;
            if (i + 1 >= n_shifts || alpha[i + 1].re != alpha[i].re || alpha[i + 1].im != -alpha[i].im ||
                beta[i + 1].re != beta[i].re || beta[i + 1].im != -beta[i].im) {
                set_error("complex shift pair %d is not followed by its conjugate pair", i);
                return SYLV_ERR_INVALID;
            }
            ++i;
        }
    }
    *cplx_out = cplx;
    return SYLV_OK;
}

// Options with the tolerance-dependent defaults filled in, validated.
static int resolve_opts(const sylv_opts* opts, double tol, sylv_opts* o) {
    if (opts) *o = *opts; else sylv_opts_default(o);
    if (o->dmin_A <= 0) o->dmin_A = tol / 20;
    if (o->dmin_B <= 0) o->dmin_B = tol / 20;
    if (o->fixed_tol <= 0) o->fixed_tol = tol / 20;
    if (o->restart < 1 || o->restart > SYLV_MAX_RESTART) {
        set_error("restart %d outside 1..%d", o->restart, SYLV_MAX_RESTART);
        return SYLV_ERR_UNSUPPORTED;
    }
    if (o->kmax < 1 || o->max_inner < 1 || o->strategy < 0 || o->strategy > SYLV_STRAT_BL_B ||
        !(o->xi > 0.0 && o->xi <= 1.0) || !(o->dmax_A > 0) || !(o->dmax_B > 0)) {
        set_error("invalid options (kmax, max_inner, strategy, xi or dmax)");
        return SYLV_ERR_INVALID;
    }
    if (o->restart_every < 0) {
        set_error("restart_every %d < 0", o->restart_every);
        return SYLV_ERR_INVALID;
    }
    if (o->ortho != SYLV_ORTHO_CGS2 && o->ortho != SYLV_ORTHO_DCGS2) {
        set_error("unknown orthogonalisation %d", o->ortho);
        return SYLV_ERR_INVALID;
    }
    if (o->precision < SYLV_PREC_FP64 || o->precision > SYLV_PREC_BF16) {
        set_error("precision %d not built", o->precision);
        return SYLV_ERR_UNSUPPORTED;
    }
    if (o->inner != SYLV_INNER_GMRES && o->inner != SYLV_INNER_BICGSTAB) {
        set_error("unknown inner solver %d", o->inner);
        return SYLV_ERR_INVALID;
    }
    if (o->real_pairs != 0 && o->real_pairs != 1) {
        set_error("real_pairs must be 0 or 1");
        return SYLV_ERR_INVALID;
    }
    if (o->inner == SYLV_INNER_BICGSTAB && o->precision == SYLV_PREC_BF16) {
        set_error("BiCGstab keeps no Krylov basis: use SYLV_PREC_FP32 (float32 vectors) or SYLV_PREC_FP64");
        return SYLV_ERR_UNSUPPORTED;
    }
    return SYLV_OK;
}

extern "C" {

const char* sylv_last_error(void) { return last_error_cstr(); }

int sylv_opts_default(sylv_opts* o) {
    if (!o) { set_error("sylv_opts_default: null"); return SYLV_ERR_INVALID; }
    std::memset(o, 0, sizeof(*o));
    o->xi = 1.0;
    o->dmin_A = o->dmin_B = 0.0;        // tau / 20 at create
    o->dmax_A = o->dmax_B = 0.1;
    o->kmax = 50;
    o->strategy = SYLV_STRAT_BL_MID;
    o->fixed_tol = 0.0;                 // tau / 20 at create
    o->restart = 30;
    o->max_inner = 20000;
    o->precision = SYLV_PREC_FP64;
    o->jacobi = 1;
    o->bl_clamp = 0;
    o->rows_per_chunk = 0;
    o->driver = 1;
    o->ortho = SYLV_ORTHO_CGS2;
    o->restart_every = 4;
    o->inner = SYLV_INNER_GMRES;
    o->real_pairs = 0;
    o->autotune = 0;
    return SYLV_OK;
}

int sylv_op_create_g(const sylv_csr* csr, const sylv_csr* mass, int32_t transpose, sylv_op** out) {
    if (!out) { set_error("sylv_op_create: null out"); return SYLV_ERR_INVALID; }
    *out = nullptr;
    HostCsr h, ht, hm, hmt;
    SYLV_TRY(load_csr(csr, h));
    if (mass) SYLV_TRY(load_csr(mass, hm));
    sylv_op* op = new (std::nothrow) sylv_op();
    if (!op) { set_error("host allocation failed"); return SYLV_ERR_NOMEM; }
    int rc;
    if (transpose) {
        transpose_csr(h, ht);
        if (mass) transpose_csr(hm, hmt);
        rc = op->op.upload(ht, mass ? &hmt : nullptr);
    } else {
        rc = op->op.upload(h, mass ? &hm : nullptr);
    }
    if (rc != SYLV_OK) { op->op.release(); delete op; return rc; }
    *out = op;
    return SYLV_OK;
}

int sylv_op_create(const sylv_csr* csr, int32_t transpose, sylv_op** out) {
    return sylv_op_create_g(csr, nullptr, transpose, out);
}

int sylv_op_format(const sylv_op* op, int32_t* is_stencil, int32_t* ndiag, int32_t* n) {
    if (!op) { set_error("sylv_op_format: null op"); return SYLV_ERR_INVALID; }
    if (is_stencil) *is_stencil = op->op.is_stencil;
    if (ndiag) *ndiag = op->op.desc.ndiag;
    if (n) *n = op->op.desc.n;
    return SYLV_OK;
}

int sylv_op_apply(const sylv_op* op, sylv_shift sigma, int32_t jacobi, int32_t is_complex,
                  const void* X, void* Y, int32_t ncols, void* stream) {
    if (!op) { set_error("sylv_op_apply: null op"); return SYLV_ERR_INVALID; }
    cudaStream_t s = (cudaStream_t)stream;
    if (is_complex) return op_apply_cplx(op->op, sigma, jacobi, X, Y, ncols, s);
    if (shift_is_complex(sigma)) { set_error("complex shift with real vectors"); return SYLV_ERR_INVALID; }
    return op_apply_real(op->op, sigma.re, jacobi, X, Y, ncols, s);
}

int sylv_op_destroy(sylv_op* op) {
    if (!op) return SYLV_OK;
    op->op.release();
    delete op;
    return SYLV_OK;
}

int sylv_cgs2(const void* V, int32_t n, int32_t k, void* w, void* h_out, int32_t is_complex, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    return is_complex ? cgs2_cplx(V, n, k, w, h_out, s) : cgs2_real(V, n, k, w, h_out, s);
}

int sylv_gmres(const sylv_op* op, sylv_shift sigma, int32_t jacobi, int32_t is_complex,
               const void* B, void* X, int32_t ncols, double tol, int32_t restart,
               int32_t max_iters, int32_t precision, int32_t* iters_out, double* resnorm_out,
               double* hist_out, void* stream) {
    if (!op) { set_error("sylv_gmres: null op"); return SYLV_ERR_INVALID; }
    if (!(tol >= 0.0)) { set_error("sylv_gmres: tol must be >= 0"); return SYLV_ERR_INVALID; }
    if (!is_complex && shift_is_complex(sigma)) { set_error("complex shift with real vectors"); return SYLV_ERR_INVALID; }
    cudaStream_t s = (cudaStream_t)stream;
    auto fn = is_complex ? (precision == SYLV_PREC_FP32 ? gmres_c64 : precision == SYLV_PREC_BF16 ? gmres_cbf : gmres_c128)
                         : (precision == SYLV_PREC_FP32 ? gmres_r32 : precision == SYLV_PREC_BF16 ? gmres_rbf : gmres_r64);
    if (precision < SYLV_PREC_FP64 || precision > SYLV_PREC_BF16) { set_error("unknown precision %d", precision); return SYLV_ERR_INVALID; }
    return fn(op->op, sigma, jacobi, B, X, ncols, tol, restart, max_iters, iters_out, resnorm_out, hist_out, s);
}

int sylv_arnoldi(const sylv_op* op, sylv_shift sigma, int32_t jacobi, int32_t is_complex, const void* v0,
                 int32_t k, int32_t precision, int32_t ortho, void* V_out, void* H_out, void* stream) {
    if (!op) { set_error("sylv_arnoldi: null op"); return SYLV_ERR_INVALID; }
    if (!is_complex && shift_is_complex(sigma)) { set_error("complex shift with real vectors"); return SYLV_ERR_INVALID; }
    if (precision < SYLV_PREC_FP64 || precision > SYLV_PREC_BF16) { set_error("unknown precision %d", precision); return SYLV_ERR_INVALID; }
    cudaStream_t s = (cudaStream_t)stream;
    auto fn = is_complex ? (precision == SYLV_PREC_FP32 ? arnoldi_c64 : precision == SYLV_PREC_BF16 ? arnoldi_cbf : arnoldi_c128)
                         : (precision == SYLV_PREC_FP32 ? arnoldi_r32 : precision == SYLV_PREC_BF16 ? arnoldi_rbf : arnoldi_r64);
    return fn(op->op, sigma, jacobi, v0, k, ortho, V_out, H_out, s);
}

int sylv_bicgstab(const sylv_op* op, sylv_shift sigma, int32_t jacobi, int32_t is_complex,
                  const void* B, void* X, int32_t ncols, double tol, int32_t max_iters,
                  int32_t precision, int32_t* iters_out, double* resnorm_out, double* hist_out,
                  void* stream) {
    if (!op) { set_error("sylv_bicgstab: null op"); return SYLV_ERR_INVALID; }
    if (!(tol >= 0.0)) { set_error("sylv_bicgstab: tol must be >= 0"); return SYLV_ERR_INVALID; }
    if (!is_complex && shift_is_complex(sigma)) { set_error("complex shift with real vectors"); return SYLV_ERR_INVALID; }
    if (precision != SYLV_PREC_FP64 && precision != SYLV_PREC_FP32) {
        set_error("sylv_bicgstab: precision %d not built (FP64 or FP32)", precision);
        return precision == SYLV_PREC_BF16 ? SYLV_ERR_UNSUPPORTED : SYLV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto fn = is_complex ? (precision == SYLV_PREC_FP32 ? bicgstab_c64 : bicgstab_c128)
                         : (precision == SYLV_PREC_FP32 ? bicgstab_r32 : bicgstab_r64);
    return fn(op->op, sigma, jacobi, B, X, ncols, tol, max_iters, iters_out, resnorm_out, hist_out, s);
}

int sylv_controller_eval(const sylv_opts* o, int32_t count, const double* in, double* out) {
    return controller_eval_dev(o, count, in, out);
}

int sylv_adi_create_g(const sylv_csr* A, const sylv_csr* B, const sylv_csr* M, const sylv_csr* Cm,
                      const double* f, const double* g, int32_t r, const sylv_shift* alpha,
                      const sylv_shift* beta, int32_t n_shifts, double tol, const sylv_opts* opts,
                      void* stream, sylv_handle** out) {
    if (!out) { set_error("sylv_adi_create: null out"); return SYLV_ERR_INVALID; }
    *out = nullptr;
    sylv_opts o;
    bool cplx = false;
    int vrc = check_problem(f, g, r, alpha, beta, n_shifts, tol, &cplx);
    if (vrc == SYLV_OK) vrc = resolve_opts(opts, tol, &o);
    if (vrc != SYLV_OK) return vrc;
    if ((M || Cm) && cplx && o.real_pairs) {
        set_error("the real double step is not built for the generalized equation (real_pairs = 0)");
        return SYLV_ERR_UNSUPPORTED;
    }
    sylv_handle* h = new (std::nothrow) sylv_handle();
    if (!h) { set_error("host allocation failed"); return SYLV_ERR_NOMEM; }
    h->stream = (cudaStream_t)stream;
    h->is_complex = (cplx && !o.real_pairs) ? 1 : 0;      // real double steps give real factors
    HostCsr ha, hb, hbt, hm, hc, hct;
    int rc = load_csr(A, ha);
    if (rc == SYLV_OK) rc = load_csr(B, hb);
    if (rc == SYLV_OK && M) rc = load_csr(M, hm);
    if (rc == SYLV_OK && Cm) rc = load_csr(Cm, hc);
    if (rc == SYLV_OK && ((M && hm.n != ha.n) || (Cm && hc.n != hb.n))) {
        set_error("M must match A and C must match B in size");
        rc = SYLV_ERR_INVALID;
    }
    // the B-side systems use (B + alpha C)^* = B^T + conj(alpha) C^T (real B, C)
    if (rc == SYLV_OK) { transpose_csr(hb, hbt); rc = h->A.upload(ha, M ? &hm : nullptr); }
    if (rc == SYLV_OK) {
        if (Cm) transpose_csr(hc, hct);
        rc = h->Bt.upload(hbt, Cm ? &hct : nullptr);
    }
    if (rc == SYLV_OK) {
        AdiArgs a{&h->A, &h->Bt, ha.n, hb.n, r, f, g, alpha, beta, n_shifts, tol, o, h->stream};
        auto mk = cplx ? (o.precision == SYLV_PREC_FP32 ? make_adi_c64 : o.precision == SYLV_PREC_BF16 ? make_adi_cbf : make_adi_c128)
                       : (o.precision == SYLV_PREC_FP32 ? make_adi_r32 : o.precision == SYLV_PREC_BF16 ? make_adi_rbf : make_adi_r64);
        rc = mk(a, &h->impl);
    }
    if (rc != SYLV_OK) {
        h->A.release();
        h->Bt.release();
        delete h;
        return rc;
    }
    *out = h;
    return SYLV_OK;
}

int sylv_adi_create(const sylv_csr* A, const sylv_csr* B, const double* f, const double* g,
                    int32_t r, const sylv_shift* alpha, const sylv_shift* beta, int32_t n_shifts,
                    double tol, const sylv_opts* opts, void* stream, sylv_handle** out) {
    return sylv_adi_create_g(A, B, nullptr, nullptr, f, g, r, alpha, beta, n_shifts, tol, opts, stream, out);
}

int sylv_adi_set_rhs(sylv_handle* h, const double* f, const double* g) {
    if (!h) { set_error("null handle"); return SYLV_ERR_INVALID; }
    return h->impl->set_rhs(f, g, 0);
}

int sylv_adi_set_rhs_device(sylv_handle* h, const double* f, const double* g) {
    if (!h) { set_error("null handle"); return SYLV_ERR_INVALID; }
    return h->impl->set_rhs(f, g, 1);
}

int sylv_adi_solve(sylv_handle* h) {
    if (!h) { set_error("null handle"); return SYLV_ERR_INVALID; }
    h->last_status = h->impl->solve();
    h->solved = 1;
    return h->last_status;
}

int sylv_adi_info(const sylv_handle* h, sylv_info* info) {
    if (!h || !info) { set_error("null handle or info"); return SYLV_ERR_INVALID; }
    return h->impl->info(info);
}

int sylv_adi_history(const sylv_handle* h, double* buf, int32_t cap, int32_t* rows) {
    if (!h || (!buf && cap > 0)) { set_error("null handle or buffer"); return SYLV_ERR_INVALID; }
    if (!h->solved) { set_error("no solve yet"); return SYLV_ERR_NOT_SOLVED; }
    return h->impl->history(buf, cap, rows);
}

int sylv_adi_factors(const sylv_handle* h, void* Z, void* Y, void* gamma, int32_t on_device,
                     int32_t* kr_out, int32_t* is_complex) {
    if (!h) { set_error("null handle"); return SYLV_ERR_INVALID; }
    if (!h->solved) { set_error("no solve yet"); return SYLV_ERR_NOT_SOLVED; }
    if (is_complex) *is_complex = h->is_complex;
    return h->impl->factors(Z, Y, gamma, on_device, kr_out);
}

int sylv_adi_core(const sylv_handle* h, double* G, int32_t ld, int32_t* kr_out) {
    if (!h) { set_error("null handle"); return SYLV_ERR_INVALID; }
    if (!h->solved) { set_error("no solve yet"); return SYLV_ERR_NOT_SOLVED; }
    int kr = 0;
    const int rc = h->impl->core(G, ld, &kr);
    if (kr_out) *kr_out = kr;
    return rc;
}

int sylv_adi_tuning(const sylv_handle* h, int32_t* rows_per_chunk, int32_t* cand, double* ms, int32_t cap,
                    int32_t* count) {
    if (!h) { set_error("null handle"); return SYLV_ERR_INVALID; }
    if (cap > 0 && (!cand || !ms)) { set_error("null candidate buffers"); return SYLV_ERR_INVALID; }
    return h->impl->tuning(rows_per_chunk, cand, ms, cap, count);
}

int sylv_adi_batch_tuning(const sylv_batch* b, int32_t* rows_per_chunk, int32_t* cand, double* ms, int32_t cap,
                          int32_t* count) {
    if (!b) { set_error("null batch"); return SYLV_ERR_INVALID; }
    if (cap > 0 && (!cand || !ms)) { set_error("null candidate buffers"); return SYLV_ERR_INVALID; }
    return b->impl->tuning(rows_per_chunk, cand, ms, cap, count);
}

int sylv_adi_profile(sylv_handle* h, int32_t enable) {
    if (!h) { set_error("null handle"); return SYLV_ERR_INVALID; }
    return h->impl->profile(enable ? 1 : 0);
}

int sylv_adi_kernel_stats(const sylv_handle* h, double* ms, double* bytes, double* flops, int64_t* launches) {
    if (!h) { set_error("null handle"); return SYLV_ERR_INVALID; }
    return h->impl->kernel_stats(ms, bytes, flops, (long long*)launches);
}

int sylv_adi_destroy(sylv_handle* h) {
    if (!h) return SYLV_OK;
    delete h->impl;
    h->A.release();
    h->Bt.release();
    delete h;
    return SYLV_OK;
}

// ---- batched solves ----

static void release_batch(sylv_batch* b) {
    if (!b) return;
    delete b->impl;
    for (auto& op : b->ops) op.release();
    delete b;
}

int sylv_adi_batch_create(int32_t count, const sylv_problem* probs, const sylv_opts* opts, void* stream,
                          sylv_batch** out) {
    if (!out) { set_error("sylv_adi_batch_create: null out"); return SYLV_ERR_INVALID; }
    *out = nullptr;
    if (count < 1 || !probs) { set_error("batch: count %d < 1 or null problems", count); return SYLV_ERR_INVALID; }
    sylv_opts o;
    bool cplx = false;
    std::vector<sylv_opts> per(count);
    for (int i = 0; i < count; ++i) {
        const sylv_problem& p = probs[i];
        bool ci = false;
        int rc = check_problem(p.f, p.g, p.r, p.alpha, p.beta, p.n_shifts, p.tol, &ci);
        if (rc == SYLV_OK) rc = resolve_opts(opts, p.tol, &per[i]);
        if (rc != SYLV_OK) {
            const std::string msg = last_error_cstr();
            set_error("batch instance %d: %s", i, msg.c_str());
            return rc;
        }
        cplx |= ci;
    }
    o = per[0];
    if (cplx && o.real_pairs) {
        set_error("batch: the real double step of conjugate pairs is not built for batches (real_pairs = 0)");
        return SYLV_ERR_UNSUPPORTED;
    }
    sylv_batch* b = new (std::nothrow) sylv_batch();
    if (!b) { set_error("host allocation failed"); return SYLV_ERR_NOMEM; }
    b->count = count;
    b->is_complex = cplx ? 1 : 0;
    b->stream = (cudaStream_t)stream;
    b->ops.resize(2 * (size_t)count);
    std::vector<BatchProb> ps(count);
    int rc = SYLV_OK;
    for (int i = 0; i < count && rc == SYLV_OK; ++i) {
        HostCsr ha, hb, hbt;
        rc = load_csr(probs[i].A, ha);
        if (rc == SYLV_OK) rc = load_csr(probs[i].B, hb);
        if (rc == SYLV_OK) { transpose_csr(hb, hbt); rc = b->ops[2 * i].upload(ha); }
        if (rc == SYLV_OK) rc = b->ops[2 * i + 1].upload(hbt);
        if (rc != SYLV_OK) {
            const std::string msg = last_error_cstr();
            set_error("batch instance %d: %s", i, msg.c_str());
            break;
        }
        const sylv_problem& p = probs[i];
        ps[i] = BatchProb{&b->ops[2 * i], &b->ops[2 * i + 1], ha.n, hb.n, p.r, p.f, p.g, p.alpha, p.beta,
                          p.n_shifts, p.tol, per[i].dmin_A, per[i].dmin_B, per[i].fixed_tol};
    }
    if (rc == SYLV_OK) {
        auto mk = cplx ? (o.precision == SYLV_PREC_FP32 ? make_batch_c64 : o.precision == SYLV_PREC_BF16 ? make_batch_cbf : make_batch_c128)
                       : (o.precision == SYLV_PREC_FP32 ? make_batch_r32 : o.precision == SYLV_PREC_BF16 ? make_batch_rbf : make_batch_r64);
        rc = mk(ps, o, b->stream, &b->impl);
    }
    if (rc != SYLV_OK) {
        release_batch(b);
        return rc;
    }
    *out = b;
    return SYLV_OK;
}

int sylv_adi_batch_solve(sylv_batch* b) {
    if (!b) { set_error("null batch"); return SYLV_ERR_INVALID; }
    return b->impl->solve();
}

static int batch_index(const sylv_batch* b, int32_t i) {
    if (!b) { set_error("null batch"); return SYLV_ERR_INVALID; }
    if (i < 0 || i >= b->count) { set_error("instance %d outside 0..%d", i, b->count - 1); return SYLV_ERR_INVALID; }
    return SYLV_OK;
}

int sylv_adi_batch_info(const sylv_batch* b, int32_t i, sylv_info* info) {
    SYLV_TRY(batch_index(b, i));
    if (!info) { set_error("null info"); return SYLV_ERR_INVALID; }
    return b->impl->info(i, info);
}

int sylv_adi_batch_history(const sylv_batch* b, int32_t i, double* buf, int32_t cap, int32_t* rows) {
    SYLV_TRY(batch_index(b, i));
    if (!buf && cap > 0) { set_error("null buffer"); return SYLV_ERR_INVALID; }
    return b->impl->history(i, buf, cap, rows);
}

int sylv_adi_batch_factors(const sylv_batch* b, int32_t i, void* Z, void* Y, void* gamma, int32_t on_device,
                           int32_t* kr_out, int32_t* is_complex) {
    SYLV_TRY(batch_index(b, i));
    if (is_complex) *is_complex = b->is_complex;
    return b->impl->factors(i, Z, Y, gamma, on_device, kr_out);
}

int sylv_adi_batch_stats(const sylv_batch* b, int64_t* launches, double* bytes, double* flops, int64_t* ticks) {
    if (!b) { set_error("null batch"); return SYLV_ERR_INVALID; }
    return b->impl->stats((long long*)launches, bytes, flops, (long long*)ticks);
}

int sylv_adi_batch_set_rhs(sylv_batch* b, int32_t i, const double* f, const double* g) {
    SYLV_TRY(batch_index(b, i));
    return b->impl->set_rhs(i, f, g);
}

int sylv_adi_batch_profile(sylv_batch* b, int32_t enable) {
    if (!b) { set_error("null batch"); return SYLV_ERR_INVALID; }
    return b->impl->profile(enable ? 1 : 0);
}

int sylv_adi_batch_kernel_stats(const sylv_batch* b, double* ms, double* bytes, double* flops, int64_t* launches) {
    if (!b) { set_error("null batch"); return SYLV_ERR_INVALID; }
    return b->impl->kernel_stats(ms, bytes, flops, (long long*)launches);
}

int sylv_adi_batch_destroy(sylv_batch* b) {
    release_batch(b);
    return SYLV_OK;
}

}  // extern "C"
