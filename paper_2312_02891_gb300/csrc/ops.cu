// ops.cu - host handling of the sparse operators: CSR validation, the
// transpose needed for (B + alpha I)^* = B^T + conj(alpha) I (real B), the
// diagonal extraction for the Jacobi preconditioner, and the choice of
// storage: by diagonals when the nonzeros lie on at most SYLV_MAXDIAG fixed
// offsets (the finite-difference stencils of the paper's convection-diffusion
// examples), CSR otherwise.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include "internal.h"

namespace sylv {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

const char* last_error_cstr() { return g_err.c_str(); }

int num_sms() {
    static int cached = 0;
    if (cached) return cached;
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
        cached = v;
    else
        return 152;
    return cached;
}

int load_csr(const sylv_csr* c, HostCsr& h) {
    if (!c) { set_error("null CSR descriptor"); return SYLV_ERR_INVALID; }
    if (c->n_rows <= 0 || c->n_rows != c->n_cols) {
        set_error("CSR must be square with n > 0 (got %d x %d)", c->n_rows, c->n_cols);
        return SYLV_ERR_INVALID;
    }
    if (c->nnz < 0 || c->nnz > 0x7fffffffLL) { set_error("CSR nnz out of range"); return SYLV_ERR_INVALID; }
    if (!c->rowptr || (c->nnz > 0 && (!c->colind || !c->val))) {
        set_error("CSR has null arrays");
        return SYLV_ERR_INVALID;
    }
    const int n = c->n_rows;
    const size_t nnz = (size_t)c->nnz;
    h.n = n;
    h.rp.resize(n + 1);
    h.ci.resize(nnz);
    h.v.resize(nnz);
    if (c->on_device) {
        SYLV_CK(cudaMemcpy(h.rp.data(), c->rowptr, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
        if (nnz) {
            SYLV_CK(cudaMemcpy(h.ci.data(), c->colind, nnz * sizeof(int), cudaMemcpyDeviceToHost));
            SYLV_CK(cudaMemcpy(h.v.data(), c->val, nnz * sizeof(double), cudaMemcpyDeviceToHost));
        }
    } else {
        std::memcpy(h.rp.data(), c->rowptr, (n + 1) * sizeof(int));
        if (nnz) {
            std::memcpy(h.ci.data(), c->colind, nnz * sizeof(int));
            std::memcpy(h.v.data(), c->val, nnz * sizeof(double));
        }
    }
    if (h.rp[0] != 0 || (size_t)h.rp[n] != nnz) {
        set_error("CSR rowptr must start at 0 and end at nnz");
        return SYLV_ERR_INVALID;
    }
    for (int i = 0; i < n; ++i) {
        if (h.rp[i + 1] < h.rp[i]) { set_error("CSR rowptr decreases at row %d", i); return SYLV_ERR_INVALID; }
        for (int p = h.rp[i]; p < h.rp[i + 1]; ++p)
            if (h.ci[p] < 0 || h.ci[p] >= n) {
                set_error("CSR column index %d out of range in row %d", h.ci[p], i);
                return SYLV_ERR_INVALID;
            }
    }
    return SYLV_OK;
}

void transpose_csr(const HostCsr& a, HostCsr& t) {
    const int n = a.n;
    t.n = n;
    t.rp.assign(n + 1, 0);
    t.ci.resize(a.ci.size());
    t.v.resize(a.v.size());
    for (size_t p = 0; p < a.ci.size(); ++p) t.rp[a.ci[p] + 1]++;
    for (int i = 0; i < n; ++i) t.rp[i + 1] += t.rp[i];
    std::vector<int> pos(t.rp.begin(), t.rp.end() - 1);
    for (int i = 0; i < n; ++i)
        for (int p = a.rp[i]; p < a.rp[i + 1]; ++p) {
            const int q = pos[a.ci[p]]++;
            t.ci[q] = i;
            t.v[q] = a.v[p];
        }
}

void DevOp::release() {
    for (double** q : {&d_dval, &d_v, &d_diag, &d_mval, &d_mv, &d_mdiag})
        if (*q) { cudaFree(*q); *q = nullptr; }
    for (int** q : {&d_rp, &d_ci, &d_mrp, &d_mci})
        if (*q) { cudaFree(*q); *q = nullptr; }
}

template <typename X>
static int to_device(X** dst, const std::vector<X>& src) {
    if (src.empty()) { *dst = nullptr; return SYLV_OK; }
    SYLV_CK(cudaMalloc((void**)dst, src.size() * sizeof(X)));
    SYLV_CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(X), cudaMemcpyHostToDevice));
    return SYLV_OK;
}

int DevOp::upload(const HostCsr& h, const HostCsr* mass) {
    release();
    const int n = h.n;
    if (mass && mass->n != n) { set_error("mass matrix of size %d for an operator of size %d", mass->n, n); return SYLV_ERR_INVALID; }
    std::vector<double> diag(n, 0.0), mdiag(mass ? n : 0, 0.0);
    // offsets of the nonzeros of the operator and of the mass matrix together
    std::map<int, int> offs;
    bool stencil = true;
    auto scan = [&](const HostCsr& c, std::vector<double>& dg) {
        for (int i = 0; i < n; ++i)
            for (int p = c.rp[i]; p < c.rp[i + 1]; ++p) {
                const int o = c.ci[p] - i;
                if (o == 0) dg[i] += c.v[p];
                if (stencil && !offs.count(o)) {
                    if ((int)offs.size() >= SYLV_MAXDIAG) stencil = false;
                    else offs[o] = 0;
                }
            }
    };
    scan(h, diag);
    if (mass) scan(*mass, mdiag);
    desc = OpDesc{};
    desc.n = n;
    desc.nnz = (long long)h.ci.size();
    desc.mnnz = mass ? (long long)mass->ci.size() : 0;
    has_mass = mass ? 1 : 0;
    if (stencil) {
        int d = 0;
        for (auto& kv : offs) { kv.second = d; desc.offs[d] = kv.first; ++d; }
        desc.ndiag = d;
        desc.fmt = 1;
        auto by_diag = [&](const HostCsr& c) {
            std::vector<double> dv((size_t)d * n, 0.0);
            for (int i = 0; i < n; ++i)
                for (int p = c.rp[i]; p < c.rp[i + 1]; ++p) dv[(size_t)offs[c.ci[p] - i] * n + i] += c.v[p];
            return dv;
        };
        SYLV_TRY(to_device(&d_dval, by_diag(h)));
        desc.dval = d_dval;
        if (mass) {
            SYLV_TRY(to_device(&d_mval, by_diag(*mass)));
            desc.mval = d_mval;
        }
    } else {
        desc.fmt = 0;
        SYLV_TRY(to_device(&d_rp, h.rp));
        SYLV_TRY(to_device(&d_ci, h.ci));
        SYLV_TRY(to_device(&d_v, h.v));
        desc.rowptr = d_rp;
        desc.colind = d_ci;
        desc.val = d_v;
        if (mass) {
            SYLV_TRY(to_device(&d_mrp, mass->rp));
            SYLV_TRY(to_device(&d_mci, mass->ci));
            SYLV_TRY(to_device(&d_mv, mass->v));
            desc.mrowptr = d_mrp;
            desc.mcolind = d_mci;
            desc.mvalc = d_mv;
        }
    }
    is_stencil = stencil ? 1 : 0;
    SYLV_TRY(to_device(&d_diag, diag));
    desc.diag = d_diag;
    if (mass) {
        SYLV_TRY(to_device(&d_mdiag, mdiag));
        desc.mdiag = d_mdiag;
    }
    return SYLV_OK;
}

}  // namespace sylv
