// noalloc.cu - a CGS2 orthogonalisation step that allocates nothing.
//
// sylv_cgs2 builds a small solver batch for each call (device buffers for the
// basis copy, partial sums and the step's state).  Some callers cannot let a
// library allocate GPU memory at call time: code running inside a memory pool
// or arena that owns the whole device budget, applications that must not
// allocate after start-up (latency-critical or certified loops), and callers
// that are themselves inside an allocator or a custom memory manager.  For
// them sylv_cgs2_noalloc runs the same three sweep kernels with all scratch in
// one file-scope __device__ array of SYLV_NOALLOC_SCRATCH_BYTES bytes, which
// every GPU that loads this library holds until the process exits.
#include <cstddef>
#include "engine.cuh"

namespace sylv {

constexpr size_t kScratchBytes = SYLV_NOALLOC_SCRATCH_BYTES;
constexpr int kRowsPerChunk = 4096;

// The scratch.  Host code must not pass this name to a kernel: on the host it
// is only a stand-in for the device array.  Its device address comes from
// cudaGetSymbolAddress, looked up with the device current on each call.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

typedef SysDesc<double, double, double> Desc64;
typedef SysState<double> State64;

// Layout of the scratch (each part 256-byte aligned).
struct ScratchLayout {
    size_t ctl, desc, state, op, items, part, total;
    explicit ScratchLayout(int nchunks) {
        auto up = [](size_t v) { return (v + 255) / 256 * 256; };
        ctl = 0;
        desc = up(ctl + sizeof(BatchCtl));
        state = up(desc + sizeof(Desc64));
        op = up(state + sizeof(State64));
        items = up(op + sizeof(OpDesc));
        part = up(items + sizeof(Item) * (size_t)nchunks);
        total = part + sizeof(double) * PSTRIDE * (size_t)nchunks;
    }
};

// Device address of g_scratch on the current device.  It is looked up on
// every call (a cheap query): an address cached across calls would go stale
// if the primary context were torn down and recreated, which reloads the
// module and may place the array elsewhere.
static int scratch_address(unsigned char** out) {
    void* p = nullptr;
    SYLV_CK(cudaGetSymbolAddress(&p, g_scratch));
    *out = static_cast<unsigned char*>(p);
    return SYLV_OK;
}

// Chunk table of the single system: items[c] = (0, c).
__global__ void k_noalloc_items(Item* items, int nchunks) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x)
        items[c] = Item{0, c};
}

// v *= scale[k] of the step's state (normalises the new basis vector in place).
__global__ void k_noalloc_scale(double* __restrict__ v, const State64* __restrict__ st, int k, int n) {
    const double s = st->scale[k];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] *= s;
}

}  // namespace sylv

using namespace sylv;

// Largest chunk count whose layout fits the scratch (the layout grows
// with the chunk count, so a binary search finds it).
static int max_chunks() {
    int lo = 0, hi = (int)(kScratchBytes / sizeof(Item)) + 1;     // layout(lo) fits, layout(hi) does not
    while (hi - lo > 1) {
        const int mid = lo + (hi - lo) / 2;
        if (ScratchLayout(mid).total <= kScratchBytes) lo = mid; else hi = mid;
    }
    return lo;
}

extern "C" int sylv_cgs2_noalloc_max_rows(void) {
    const long long rows = (long long)max_chunks() * kRowsPerChunk;
    return rows > 0x7fffffff ? 0x7fffffff : (int)rows;
}

extern "C" int sylv_cgs2_noalloc(double* V, int32_t n, int32_t k, const double* w, double* h_out, void* stream) {
    if (!V || !w || !h_out || n <= 0 || k < 1 || k > SYLV_MR) {
        set_error("sylv_cgs2_noalloc: invalid arguments (n=%d k=%d, 1 <= k <= %d)", n, k, SYLV_MR);
        return SYLV_ERR_INVALID;
    }
    const int nchunks = (n + kRowsPerChunk - 1) / kRowsPerChunk;
    const ScratchLayout L(nchunks);
    if (L.total > kScratchBytes) {
        set_error("sylv_cgs2_noalloc: n=%d exceeds the %d rows its %zu-byte static scratch holds",
                  n, sylv_cgs2_noalloc_max_rows(), (size_t)kScratchBytes);
        return SYLV_ERR_INVALID;
    }
    unsigned char* base = nullptr;
    SYLV_TRY(scratch_address(&base));
    cudaStream_t s = (cudaStream_t)stream;
    // Every call rewrites the parts it reads: the control block, the
    // descriptor, the state (whose completion counter must start at zero) and
    // the chunk table.  Partial sums are written before they are read.
    BatchCtl ctl{};
    ctl.n_active = 1;
    Desc64 d{};
    d.n = n;
    d.op = 0;
    d.nchunks = nchunks;
    d.rows_per_chunk = kRowsPerChunk;
    d.ldv = (size_t)n;
    d.V = V;                                  // caller's n x (k+1) block, column k receives the result
    d.w = const_cast<double*>(w);             // read only in this mode
    d.part = reinterpret_cast<double*>(base + L.part);
    d.restart = k;
    State64 st;
    std::memset(&st, 0, sizeof(st));
    st.phase = PH_ARNOLDI;
    st.j = k - 1;
    for (int l = 0; l < k; ++l) st.scale[l] = 1.0;
    OpDesc op{};
    op.n = n;
    SYLV_CK(cudaMemcpyAsync(base + L.ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
    SYLV_CK(cudaMemcpyAsync(base + L.desc, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    SYLV_CK(cudaMemcpyAsync(base + L.state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    SYLV_CK(cudaMemcpyAsync(base + L.op, &op, sizeof(op), cudaMemcpyHostToDevice, s));
    auto* dc = reinterpret_cast<BatchCtl*>(base + L.ctl);
    auto* dd = reinterpret_cast<const Desc64*>(base + L.desc);
    auto* ds = reinterpret_cast<State64*>(base + L.state);
    auto* dop = reinterpret_cast<const OpDesc*>(base + L.op);
    auto* di = reinterpret_cast<Item*>(base + L.items);
    k_noalloc_items<<<std::max(1, std::min(num_sms(), (nchunks + 255) / 256)), 256, 0, s>>>(di, nchunks);
    k_arnoldi_spmv<double, double, double, 0><<<nchunks, SYLV_BLOCK, 0, s>>>(dd, ds, dop, di, dc, 1);
    k_cgs_pass2<double, double, double, 0><<<nchunks, SYLV_BLOCK, 0, s>>>(dd, ds, di, dc);
    k_cgs_pass3<double, double, double, 0><<<nchunks, SYLV_BLOCK, 0, s>>>(dd, ds, di, dc, 1);
    const int grid = std::max(1, std::min(num_sms() * 4, (n + 255) / 256));
    k_noalloc_scale<<<grid, 256, 0, s>>>(V + (size_t)k * n, ds, k, n);
    SYLV_CK(cudaGetLastError());
    // h + h2 and the norm: column k-1 of the state's R (k + 1 entries)
    const unsigned char* rcol = base + L.state + offsetof(State64, R) + sizeof(double) * (size_t)(k - 1) * SYLV_MAXV;
    SYLV_CK(cudaMemcpyAsync(h_out, rcol, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s));
    SYLV_CK(cudaStreamSynchronize(s));
    return SYLV_OK;
}
