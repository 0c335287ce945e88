// engine.cuh - host orchestration of the batched GMRES solves and of the
// inexact LR-ADI outer loop (Algorithm 1).  Instantiated for double (real
// shifts) in inst_real.cu and for cplx (complex shifts) in inst_cplx.cu.
#pragma once
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "internal.h"
#include "pair_kernels.cuh"

namespace sylv {

template <typename T> struct Dev;   // RAII device buffer
template <typename T> struct Dev {
    T* p = nullptr;
    size_t count = 0;
    int alloc(size_t n) {
        release();
        if (n == 0) return SYLV_OK;
        cudaError_t e = cudaMalloc((void**)&p, n * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
            return SYLV_ERR_NOMEM;
        }
        count = n;
        return SYLV_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        count = 0;
    }
    ~Dev() { release(); }
};

inline size_t round_ld(size_t n) { return (n + 31) / 32 * 32; }

// The staged sweeps take more than the default 48 KB of dynamic shared
// memory: allow it once per instantiation (the attribute is per device, so
// it is set again on the device current at each call; it is cheap).
template <typename T, typename S, typename C>
int sweep_kernel_setup() {
    const int b = sweep_smem_bytes<S, C>();
    if constexpr (sweep_smem_bytes<S, C>() > 48 * 1024) {
        SYLV_CK(cudaFuncSetAttribute(k_arnoldi_spmv<T, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        SYLV_CK(cudaFuncSetAttribute(k_cgs_pass2<T, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        SYLV_CK(cudaFuncSetAttribute(k_cgs_pass3<T, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    }
    if constexpr (dcgs_b_smem_bytes<T, S, C>() > 48 * 1024)
        SYLV_CK(cudaFuncSetAttribute(k_dcgs_b<T, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dcgs_b_smem_bytes<T, S, C>()));
    if constexpr (dcgs_a_smem_bytes<T, S, C>() > 48 * 1024)
        SYLV_CK(cudaFuncSetAttribute(k_dcgs_a<T, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dcgs_a_smem_bytes<T, S, C>()));
    (void)b;
    return SYLV_OK;
}

// Rows per work item of the basis sweeps, in whole 32-row tiles, at least
// 256 rows: one wave of resident blocks over all rows of the batch for the
// 32-bit sweeps (several resident blocks per SM hide each other's fixed
// costs; measured best on the 2D benchmark workload), two waves for the
// float64 sweeps (one resident block per SM).  sys_rows holds the rows of
// every system: each system rounds its chunk count up, so the chunk is
// widened (by at most a quarter) until all chunks fit the wave - a block
// left over for a second wave delays its system's reduction by a whole
// block's work.
template <typename T, typename S, typename C>
int sweep_rows_per_chunk(const std::vector<long long>& sys_rows, int ortho) {
    long long total_rows = 0;
    for (long long q : sys_rows) total_rows += q;
    // the wave is set by the sweep kernel with the fewest resident blocks
    // (the delayed-CGS2 dot kernel holds twice the accumulators)
    int per_sm = 0;
    const void* fn = ortho == 1 ? (const void*)k_dcgs_a<T, S, C> : (const void*)k_cgs_pass2<T, S, C>;
    const int smem = ortho == 1 ? dcgs_a_smem_bytes<T, S, C>() : sweep_smem_bytes<S, C>();
    if (sweep_kernel_setup<T, S, C>() != SYLV_OK ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SYLV_BLOCK, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long waves = SweepOcc<C>::value > 1 ? 1 : 2;
    const long long items = waves * num_sms() * per_sm;
    long long rpc = (total_rows + items - 1) / items;
    rpc = std::max<long long>(256, std::min<long long>((rpc + 31) / 32 * 32, 1 << 16));
    auto chunks = [&](long long c) {
        long long k = 0;
        for (long long q : sys_rows) k += (q + c - 1) / c;
        return k;
    };
    long long fit = rpc;
    while (chunks(fit) > items && fit + 32 <= std::min<long long>(rpc + rpc / 4, 1 << 16)) fit += 32;
    return (int)(chunks(fit) <= items ? fit : rpc);
}

// Rows per work item of the BiCGstab kernels (one item = a row chunk of a
// group of column systems, one block each): at most 768 rows, so that three
// staged four-column items of a 2D stencil with N <= 256 fit an SM's shared
// memory, and fewer when the groups' rows would give under eight items per
// SM (256 at the least).
template <typename T, typename S, typename C>
int bicg_rows_per_chunk(const std::vector<long long>& group_rows) {
    long long total_rows = 0;
    for (long long q : group_rows) total_rows += q;
    const long long items = (long long)num_sms() * 8;
    const long long rpc = (total_rows + items - 1) / items;
    return (int)std::max<long long>(256, std::min<long long>(768, (rpc + 31) / 32 * 32));
}

// Rows of the BiCGstab groups formed from consecutive column systems with the
// same rows, operator, Jacobi inverse and stencil values (at most BG_MAXCOL
// columns each): the partition Engine::setup uses.
template <typename P1, typename P2>
std::vector<std::pair<int, int>> bicg_groups(const std::vector<int>& sys_n, const std::vector<int>& sys_op,
                                             const std::vector<P1>& pinv, const std::vector<P2>& aval) {
    std::vector<std::pair<int, int>> g;    // (first system, columns)
    for (int q = 0; q < (int)sys_n.size(); ++q) {
        const P2 aq = aval.empty() ? P2() : aval[q];
        if (!g.empty()) {
            const int f = g.back().first;
            const P2 af = aval.empty() ? P2() : aval[f];
            if (g.back().second < BG_MAXCOL && sys_n[f] == sys_n[q] && sys_op[f] == sys_op[q] && pinv[f] == pinv[q] &&
                af == aq) {
                g.back().second++;
                continue;
            }
        }
        g.push_back({q, 1});
    }
    return g;
}

// Elements of one system's tile-major basis: whole 32-row tiles.
template <class D>
inline size_t basis_elems(const D& d) { return (size_t)((d.n + 31) / 32) * d.tstride; }

// A batch of shifted systems solved together by restarted GMRES.
template <typename T, typename S, typename C>
struct Engine {
    cudaStream_t stream = nullptr;
    int nsys = 0, nitems = 0, restart = 30;
    std::vector<SysDesc<T, S, C>> h_sd;
    Dev<SysDesc<T, S, C>> d_sd;
    Dev<SysState<T>> d_st;
    Dev<Item> d_items;
    Dev<OpDesc> d_ops;
    Dev<BatchCtl> d_ctl;
    Dev<S> d_V;
    Dev<C> d_w;
    Dev<T> d_part;
    int* h_flag = nullptr;        // mapped pinned word
    int* d_hflag = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    long long ticks = 0;
    // statistics: launches per kernel; with profiling, event-timed milliseconds
    int profile = 0;
    cudaEvent_t pev[4][6] = {};
    int pending[4] = {0, 0, 0, 0};
    int pkid[4][5] = {};                // kernel id of each timed interval
    int ortho = 0;                      // 0: CGS2 (three sweeps), 1: delayed CGS2 (two sweeps)
    int inner = 0;                      // 0: restarted GMRES, 1: BiCGstab
    // BiCGstab: groups of column systems, their work items and vectors
    int ngroups = 0, ngitems = 0;
    std::vector<BGroup<T, C>> h_groups;
    Dev<BGroup<T, C>> d_groups;
    Dev<Item> d_gitems;
    Dev<Item> d_glist;                  // work list of the device iteration (k_bicg_list)
    Dev<C> d_bv;
    Dev<T> d_gpart;
    Dev<unsigned> d_gcount;
    // BiCGstab step kernels a and b: dynamic shared memory of a staged work
    // item (the largest one that fits; 0: every item reads global memory
    // directly)
    int bicg_smem[2] = {0, 0};
    int restart_every = 1;              // host driver: restart kernels every k-th device iteration
    double kernel_ms[K_COUNT] = {};     // event-timed milliseconds of the sampled launches
    long long samples[K_COUNT] = {};    // sampled launches
    long long launches[K_COUNT] = {};   // all launches
    long long tick_no = 0;
    int prof_every = 4;
    // host driver: programmatic dependent launches (off if unsupported or if
    // the environment sets SYLV_NO_PDL)
    int pdl = std::getenv("SYLV_NO_PDL") ? 0 : 1;

    ~Engine() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        for (auto& row : pev)
            for (auto& e : row)
                if (e) cudaEventDestroy(e);
        if (h_flag) cudaFreeHost(h_flag);
    }

    // sys_n[q], sys_op[q]: rows and operator of system q; pinv[q]: Jacobi
    // buffer or null; aval[q]: pre-scaled stencil buffer or null (empty: all
    // null); hist[q]: per-step estimate buffer or null.
    int setup(const std::vector<int>& sys_n, const std::vector<int>& sys_op,
              const std::vector<OpDesc>& ops, const std::vector<T*>& pinv,
              const std::vector<C*>& aval, const std::vector<double*>& hist, int hist_cap,
              int restart_, int rpc, cudaStream_t s) {
        stream = s;
        restart = restart_;
        nsys = (int)sys_n.size();
        SYLV_TRY((sweep_kernel_setup<T, S, C>()));
        if (rpc <= 0) {
            if (inner == 1) {
                std::vector<long long> grows;
                for (const auto& g : bicg_groups(sys_n, sys_op, pinv, aval)) grows.push_back(sys_n[g.first]);
                rpc = bicg_rows_per_chunk<T, S, C>(grows);
            } else {
                rpc = sweep_rows_per_chunk<T, S, C>(std::vector<long long>(sys_n.begin(), sys_n.end()), ortho);
            }
        }
        rpc = (rpc + 31) / 32 * 32;       // chunks hold whole 32-row basis tiles
        size_t vtot = 0, wtot = 0, ptot = 0, btot = 0;
        std::vector<Item> items;
        h_sd.resize(nsys);
        for (int q = 0; q < nsys; ++q) {
            SysDesc<T, S, C>& d = h_sd[q];
            d = SysDesc<T, S, C>{};
            d.aval = aval.empty() ? nullptr : aval[q];
            d.n = sys_n[q];
            d.op = sys_op[q];
            d.rows_per_chunk = rpc;
            d.nchunks = (sys_n[q] + rpc - 1) / rpc;
            d.ldv = round_ld(sys_n[q]);
            d.tstride = (size_t)(restart + 1) * 32;
            d.restart = restart;
            d.hist = hist.empty() ? nullptr : hist[q];
            d.hist_cap = hist_cap;
            d.pinv = pinv[q];
            if (inner == 1) {
                btot += (size_t)BV_COUNT * d.ldv;       // no Krylov basis, no work vector
            } else {
                vtot += basis_elems(d);
                wtot += d.ldv;
            }
            ptot += (size_t)d.nchunks * PSTRIDE;
            for (int c = 0; c < d.nchunks; ++c) items.push_back({q, c});
        }
        nitems = (int)items.size();
        SYLV_TRY(d_V.alloc(vtot));
        SYLV_TRY(d_w.alloc(wtot));
        SYLV_TRY(d_part.alloc(ptot));
        SYLV_TRY(d_bv.alloc(btot));
        if (btot) SYLV_CK(cudaMemset(d_bv.p, 0, btot * sizeof(C)));
        size_t vo = 0, wo = 0, po = 0, bo = 0;
        for (int q = 0; q < nsys; ++q) {
            SysDesc<T, S, C>& d = h_sd[q];
            if (inner == 1) {
                d.bv = d_bv.p + bo;
                d.rres = d.bv + (size_t)BV_R * d.ldv;
                bo += (size_t)BV_COUNT * d.ldv;
            } else {
                d.V = d_V.p + vo;
                d.w = d_w.p + wo;
                vo += basis_elems(d);
                wo += d.ldv;
            }
            d.part = d_part.p + po;
            po += (size_t)d.nchunks * PSTRIDE;
        }
        if (inner == 1) {
            // groups of consecutive systems sharing rows, operator and shift data;
            // their vectors are consecutive in d_bv (BV_COUNT * ldv apart)
            const auto gs = bicg_groups(sys_n, sys_op, pinv, aval);
            ngroups = (int)gs.size();
            size_t gp = 0;
            for (const auto& g : gs) gp += (size_t)h_sd[g.first].nchunks * BG_PSTRIDE;
            SYLV_TRY(d_gpart.alloc(gp));
            SYLV_TRY(d_gcount.alloc(ngroups));
            SYLV_CK(cudaMemset(d_gcount.p, 0, ngroups * sizeof(unsigned)));
            std::vector<Item> gitems;
            h_groups.resize(ngroups);
            gp = 0;
            for (int g = 0; g < ngroups; ++g) {
                BGroup<T, C>& bg = h_groups[g];
                const SysDesc<T, S, C>& d0 = h_sd[gs[g].first];
                const OpDesc& od = ops[d0.op];
                bg = BGroup<T, C>{};
                bg.sys0 = gs[g].first;
                bg.ncol = gs[g].second;
                bg.nchunks = d0.nchunks;
                bg.part = d_gpart.p + gp;
                bg.counter = d_gcount.p + g;
                bg.n = d0.n;
                bg.rpc = d0.rows_per_chunk;
                bg.ldv = d0.ldv;
                bg.bv = d0.bv;
                bg.aval = d0.aval;
                bg.pinv = d0.pinv;
                bg.ndiag = od.fmt == 1 ? od.ndiag : 0;
                for (int d = 0; d < bg.ndiag; ++d) bg.offs[d] = od.offs[d];
                bg.halo = op_halo_of(bg.offs, bg.ndiag);
                bg.nnz = (double)od.nnz;
                gp += (size_t)bg.nchunks * BG_PSTRIDE;
                for (int c = 0; c < bg.nchunks; ++c) gitems.push_back({g, c});
            }
            ngitems = (int)gitems.size();
            SYLV_TRY(d_groups.alloc(ngroups));
            SYLV_TRY(d_gitems.alloc(gitems.size()));
            SYLV_TRY(d_glist.alloc(gitems.size()));
            SYLV_CK(cudaMemcpy(d_groups.p, h_groups.data(), ngroups * sizeof(BGroup<T, C>), cudaMemcpyHostToDevice));
            SYLV_CK(cudaMemcpy(d_gitems.p, gitems.data(), gitems.size() * sizeof(Item), cudaMemcpyHostToDevice));
            SYLV_TRY(bicg_launch_setup());
        }
        SYLV_TRY(d_sd.alloc(nsys));
        SYLV_TRY(d_st.alloc(nsys));
        SYLV_TRY(d_items.alloc(items.size()));
        SYLV_TRY(d_ops.alloc(ops.size()));
        SYLV_TRY(d_ctl.alloc(1));
        SYLV_CK(cudaMemcpy(d_sd.p, h_sd.data(), nsys * sizeof(SysDesc<T, S, C>), cudaMemcpyHostToDevice));
        SYLV_CK(cudaMemcpy(d_items.p, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice));
        SYLV_CK(cudaMemcpy(d_ops.p, ops.data(), ops.size() * sizeof(OpDesc), cudaMemcpyHostToDevice));
        SYLV_CK(cudaMemset(d_st.p, 0, nsys * sizeof(SysState<T>)));
        if (vtot) SYLV_CK(cudaMemset(d_V.p, 0, vtot * sizeof(S)));
        SYLV_CK(cudaHostAlloc((void**)&h_flag, sizeof(int), cudaHostAllocMapped));
        *h_flag = 0;
        SYLV_CK(cudaHostGetDevicePointer((void**)&d_hflag, h_flag, 0));
        BatchCtl c{};
        c.h_flag = d_hflag;
        c.nitems = nitems;
        SYLV_CK(cudaMemcpy(d_ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice));
        for (auto& e : ev) SYLV_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return SYLV_OK;
    }

    // Dynamic shared memory of the staged step kernels a and b: the largest
    // work item of a stencil group (all columns active) that fits the cap
    // (larger items read global memory directly).
    int bicg_launch_setup() {
        const void* kern[2] = {(const void*)k_bicg_a<T, S, C>, (const void*)k_bicg_b<T, S, C>};
        for (int k = 0; k < 2; ++k) {
            size_t cap = 0;
            for (const auto& bg : h_groups) {
                if (!bg.aval) continue;
                const size_t b = k == 0 ? stage_bytes_a<C>(bg.rpc, bg.halo, bg.ndiag, bg.ncol)
                                        : stage_bytes_b<C>(bg.rpc, bg.halo, bg.ndiag, bg.ncol);
                if (b <= SYLV_BICG_SMEM_CAP) cap = std::max(cap, b);
            }
            bicg_smem[k] = (int)cap;
            SYLV_CK(cudaFuncSetAttribute(kern[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
        }
        return SYLV_OK;
    }

    // BiCGstab nodes of a graph body: k_bicg_list -> k_bicg_a -> k_bicg_b ->
    // k_bicg_c after dep (null: none), *last = the node of k_bicg_c.  With
    // try_dyn the step-kernel nodes are made device-updatable, so that the
    // list kernel sets their grids to the list's length (dyn_grid = 1 and
    // their handles in dn on success); otherwise they keep the full grid and
    // their blocks beyond the list return at once.
    int dyn_grid = 0;
    cudaGraphDeviceNode_t dn[3] = {};
    int add_bicg_nodes(cudaGraph_t body, cudaGraphNode_t* dep, cudaGraphNode_t* last, bool try_dyn) {
        auto add = [&](cudaGraphNode_t* node, cudaGraphNode_t* d, void* func, int grid, void** args, int smem) {
            cudaKernelNodeParams kp = {};
            kp.func = func;
            kp.gridDim = dim3(grid);
            kp.blockDim = dim3(SYLV_BLOCK);
            kp.sharedMemBytes = smem;
            kp.kernelParams = args;
            kp.extra = nullptr;
            return cudaGraphAddKernelNode(node, body, d, d ? 1 : 0, &kp);
        };
        auto* sdp = d_sd.p;
        auto* stp = d_st.p;
        auto* opp = d_ops.p;
        auto* grp = d_groups.p;
        auto* glp = d_glist.p;
        auto* ctp = d_ctl.p;
        int ng = ngroups, sma = bicg_smem[0], smb = bicg_smem[1];
        void* al[] = {&grp, &ng, &stp, &glp, &ctp};
        void* aa[] = {&sdp, &stp, &opp, &grp, &glp, &sma, &ctp};
        void* ab[] = {&sdp, &stp, &opp, &grp, &glp, &smb, &ctp};
        void* ac[] = {&sdp, &stp, &grp, &glp, &ctp};
        cudaGraphNode_t nl, n[3];
        SYLV_CK(add(&nl, dep, (void*)k_bicg_list<T, C>, 1, al, 0));
        SYLV_CK(add(&n[0], &nl, (void*)k_bicg_a<T, S, C>, ngitems, aa, sma));
        SYLV_CK(add(&n[1], &n[0], (void*)k_bicg_b<T, S, C>, ngitems, ab, smb));
        SYLV_CK(add(&n[2], &n[1], (void*)k_bicg_c<T, S, C>, ngitems, ac, 0));
        *last = n[2];
        dyn_grid = 0;
        if (!try_dyn) return SYLV_OK;
        for (int k = 0; k < 3; ++k) {
            cudaKernelNodeAttrValue v = {};
            v.deviceUpdatableKernelNode.deviceUpdatable = 1;
            cudaKernelNodeAttrValue o = {};
            if (cudaGraphKernelNodeSetAttribute(n[k], cudaKernelNodeAttributeDeviceUpdatableKernelNode, &v) !=
                    cudaSuccess ||
                cudaGraphKernelNodeGetAttribute(n[k], cudaKernelNodeAttributeDeviceUpdatableKernelNode, &o) !=
                    cudaSuccess ||
                !o.deviceUpdatableKernelNode.devNode) {
                (void)cudaGetLastError();
                return SYLV_OK;
            }
            dn[k] = o.deviceUpdatableKernelNode.devNode;
        }
        dyn_grid = 1;
        return SYLV_OK;
    }

    // The control block's work-list fields of a graph built with
    // add_bicg_nodes (device handles, whether the grids follow the list).
    void set_dyn_fields(BatchCtl& c) const {
        c.dyn_grid = dyn_grid;
        for (int k = 0; k < 3; ++k) c.dn_step[k] = dyn_grid ? dn[k] : cudaGraphDeviceNode_t{};
    }

    // Reports (and clears) a shared-memory staging wait of the BiCGstab
    // kernels that gave up during the last solve; the columns it touched
    // then hold non-finite values.
    int take_stage_fault() {
        int f = 0;
        SYLV_CK(cudaMemcpy(&f, &d_ctl.p->stage_fault, sizeof(int), cudaMemcpyDeviceToHost));
        if (!f) return SYLV_OK;
        const int z = 0;
        SYLV_CK(cudaMemcpy(&d_ctl.p->stage_fault, &z, sizeof(int), cudaMemcpyHostToDevice));
        set_error("a shared-memory staging wait of the BiCGstab kernels gave up; the affected columns are not finite");
        return SYLV_ERR_CUDA;
    }

    // Blocks of the restart kernels (grid-stride over the work items).
    int restart_grid() const { return std::max(1, std::min(inner == 1 ? ngitems : nitems, 2 * num_sms())); }

    // A kernel of the device iteration, launched with programmatic stream
    // serialization (the kernel waits for its predecessor in pdl_enter());
    // if the launch with the attribute is refused, later launches go without.
    template <typename... P, typename... A>
    int launch(void (*kern)(P...), dim3 grid, size_t smem, A... args) {
        const dim3 block(SYLV_BLOCK);
        if (pdl) {
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = grid;
            cfg.blockDim = block;
            cfg.dynamicSmemBytes = smem;
            cfg.stream = stream;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            if (cudaLaunchKernelEx(&cfg, kern, args...) == cudaSuccess) return SYLV_OK;
            (void)cudaGetLastError();
            pdl = 0;
        }
        kern<<<grid, block, smem, stream>>>(args...);
        SYLV_CK(cudaGetLastError());
        return SYLV_OK;
    }

    // One device iteration: every active system advances one Arnoldi step
    // and restarts if its cycle ended.
    // With profiling on, every prof_every-th tick is bracketed by events.
    int launch_tick(int cgs_mode = 0, int slot = 0, bool with_restart = true) {
        const dim3 grid(nitems), block(SYLV_BLOCK);
        cudaEvent_t* pe = (profile && (tick_no++ % prof_every) == 0) ? pev[slot] : nullptr;
        if (pe) SYLV_CK(cudaEventRecord(pe[0], stream));
        const int sm = sweep_smem_bytes<S, C>();
        int nk = 0;
        auto mark = [&](int kid) -> int {
            if (pe) {
                pkid[slot][nk] = kid;
                SYLV_CK(cudaEventRecord(pe[++nk], stream));
            }
            launches[kid]++;
            return SYLV_OK;
        };
        if (inner == 1) {
            const dim3 g(ngitems);
            SYLV_TRY(launch(k_bicg_list<T, C>, dim3(1), 0, d_groups.p, ngroups, d_st.p, d_glist.p, d_ctl.p));
            SYLV_TRY(mark(K_RUPD));
            SYLV_TRY(launch(k_bicg_a<T, S, C>, g, bicg_smem[0], d_sd.p, d_st.p, d_ops.p, d_groups.p, d_glist.p,
                            bicg_smem[0], d_ctl.p));
            SYLV_TRY(mark(K_SPMV));
            SYLV_TRY(launch(k_bicg_b<T, S, C>, g, bicg_smem[1], d_sd.p, d_st.p, d_ops.p, d_groups.p, d_glist.p,
                            bicg_smem[1], d_ctl.p));
            SYLV_TRY(mark(K_CGS2));
            SYLV_TRY(launch(k_bicg_c<T, S, C>, g, 0, d_sd.p, d_st.p, d_groups.p, d_glist.p, d_ctl.p));
            SYLV_TRY(mark(K_CGS3));
            if (with_restart) {
                SYLV_TRY(launch(k_bicg_resid<T, S, C>, dim3(restart_grid()), 0, d_sd.p, d_st.p, d_ops.p, d_groups.p,
                                d_gitems.p, ngitems, d_ctl.p));
                SYLV_TRY(mark(K_RRES));
            }
            if (pe) pending[slot] = nk;
            SYLV_CK(cudaGetLastError());
            return SYLV_OK;
        }
        if (ortho == 1 && cgs_mode == 0) {
            SYLV_TRY(launch(k_dcgs_a<T, S, C>, grid, dcgs_a_smem_bytes<T, S, C>(), d_sd.p, d_st.p, d_ops.p,
                            d_items.p, d_ctl.p));
            SYLV_TRY(mark(K_SPMV));
            SYLV_TRY(launch(k_dcgs_b<T, S, C>, dim3(nitems + nsys), dcgs_b_smem_bytes<T, S, C>(), d_sd.p, d_st.p,
                            d_items.p, d_ctl.p, nsys));
            SYLV_TRY(mark(K_CGS3));
        } else {
            k_arnoldi_spmv<T, S, C><<<grid, block, sm, stream>>>(d_sd.p, d_st.p, d_ops.p, d_items.p, d_ctl.p, cgs_mode);
            SYLV_TRY(mark(K_SPMV));
            k_cgs_pass2<T, S, C><<<grid, block, sm, stream>>>(d_sd.p, d_st.p, d_items.p, d_ctl.p);
            SYLV_TRY(mark(K_CGS2));
            k_cgs_pass3<T, S, C><<<grid, block, sm, stream>>>(d_sd.p, d_st.p, d_items.p, d_ctl.p, cgs_mode);
            SYLV_TRY(mark(K_CGS3));
        }
        if (cgs_mode == 0 && with_restart) {
            const dim3 rgrid(restart_grid());
            SYLV_TRY(launch(k_restart_update<T, S, C>, rgrid, 0, d_sd.p, d_st.p, d_items.p, d_ctl.p));
            SYLV_TRY(mark(K_RUPD));
            SYLV_TRY(launch(k_restart_residual<T, S, C>, rgrid, 0, d_sd.p, d_st.p, d_ops.p, d_items.p, d_ctl.p));
            SYLV_TRY(mark(K_RRES));
        }
        if (pe) pending[slot] = nk;
        SYLV_CK(cudaGetLastError());
        return SYLV_OK;
    }

    // Add the event-timed durations of a finished tick to the totals.
    int harvest(int slot) {
        if (pending[slot]) SYLV_CK(cudaEventSynchronize(pev[slot][pending[slot]]));
        for (int q = 0; q < pending[slot]; ++q) {
            float ms = 0.f;
            SYLV_CK(cudaEventElapsedTime(&ms, pev[slot][q], pev[slot][q + 1]));
            kernel_ms[pkid[slot][q]] += ms;
            samples[pkid[slot][q]] += 1;
        }
        pending[slot] = 0;
        return SYLV_OK;
    }

    int set_profile(int on) {
        profile = on;
        tick_no = 0;
        for (int q = 0; q < K_COUNT; ++q) { kernel_ms[q] = 0.0; launches[q] = 0; samples[q] = 0; }
        for (int sl = 0; sl < 4; ++sl) pending[sl] = 0;
        if (on && !pev[0][0])
            for (int sl = 0; sl < 4; ++sl)
                for (int q = 0; q < 6; ++q) SYLV_CK(cudaEventCreate(&pev[sl][q]));
        BatchCtl c{};
        SYLV_CK(cudaMemcpy(&c, d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost));
        for (int q = 0; q < K_COUNT; ++q) { c.bytes[q] = 0.0; c.flops[q] = 0.0; }
        SYLV_CK(cudaMemcpy(d_ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice));
        return SYLV_OK;
    }

    int read_work(double* bytes, double* flops) const {
        BatchCtl c{};
        SYLV_CK(cudaMemcpy(&c, d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost));
        for (int q = 0; q < K_COUNT; ++q) { bytes[q] = c.bytes[q]; flops[q] = c.flops[q]; }
        return SYLV_OK;
    }

    // Launch ticks until every system is done (the device clears *h_flag),
    // keeping at most four ticks in flight.  The caller sets *h_flag = 1
    // before the work that activates the systems.  The restart kernels run
    // in the first tick and then every restart_every-th one: a system whose
    // cycle ended waits (its sweeps skip it) until the next restart tick, and
    // its arithmetic does not change.
    int run(long long max_ticks) {
        const int D = 4;
        // flow control: one event per G ticks (an event recorded between two
        // kernels ends their programmatic overlap), at most D events (2 with
        // programmatic launches, so about 8 ticks) in flight
        const int G = pdl ? 4 : 1, DE = pdl ? 2 : D;
        long long t = 0, grp = 0;
        while (*(volatile int*)h_flag != 0) {
            if (t >= max_ticks) {
                set_error("inner solves did not finish within %lld device iterations", max_ticks);
                return SYLV_ERR_INNER_STALL;
            }
            const int slot = (int)(t % D);
            if (pending[slot]) SYLV_TRY(harvest(slot));
            SYLV_TRY(launch_tick(0, slot, restart_every <= 1 || t % restart_every == 0));
            ++t;
            if (t % G == 0) {
                SYLV_CK(cudaEventRecord(ev[grp % DE], stream));
                ++grp;
                if (grp >= DE) SYLV_CK(cudaEventSynchronize(ev[grp % DE]));
            }
        }
        ticks += t;
        if (profile) {
            SYLV_CK(cudaStreamSynchronize(stream));
            for (int sl = 0; sl < D; ++sl)
                if (pending[sl]) SYLV_TRY(harvest(sl));
        }
        return SYLV_OK;
    }
};

// ---------------------------------------------------------------------------
// Autotuner of the work-chunk size (rows per work item) of the inner-solver
// kernels.  Each candidate builds the engine of the actual systems, fills the
// vectors with a fixed pseudo-random pattern and the operators' stencil
// values with a diagonally dominant stencil of the same diagonals (so the
// iteration neither breaks down nor converges during the probe), and times
// device iterations with CUDA events: BiCGstab 2 + 12 steps, GMRES one cycle.
// The fastest candidate wins; every candidate and its time are kept.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_pattern(double& x, double u, double) { x = u; }
__device__ __forceinline__ void set_pattern(float& x, double u, double) { x = (float)u; }
__device__ __forceinline__ void set_pattern(bf16& x, double u, double) { x = __double2bfloat16(u); }
__device__ __forceinline__ void set_pattern(cplx& x, double u, double v) { x = {u, v}; }
__device__ __forceinline__ void set_pattern(cflt& x, double u, double v) { x = {(float)u, (float)v}; }
__device__ __forceinline__ void set_pattern(cbf16& x, double u, double v) { x = {__double2bfloat16(u), __double2bfloat16(v)}; }

template <typename X>
__global__ void k_fill_pattern(X* v, size_t n, unsigned seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned h = (unsigned)(i * 2654435761u) ^ seed;
        h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
        const double u = (double)(h & 0xffffff) / 16777216.0 - 0.5;
        set_pattern(v[i], u, 0.25 - u);
    }
}

template <typename C>
__global__ void k_fill_stencil(C* aval, OpDesc op) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < op.n; i += gridDim.x * blockDim.x)
        for (int d = 0; d < op.ndiag; ++d)
            aval[(size_t)d * op.n + i] = make_scalar<C>(op.offs[d] == 0 ? 1.0 : -0.1, 0.0);
}

struct TuneResult {
    int chosen = 0;
    std::vector<int> cand;
    std::vector<double> ms;      // per device iteration
};

template <typename T, typename S, typename C>
int autotune_rpc(const std::vector<int>& sys_n, const std::vector<int>& sys_op, const std::vector<OpDesc>& ops,
                 const std::vector<T*>& pinv, const std::vector<C*>& aval, int restart, int ortho, int inner,
                 cudaStream_t s, TuneResult* out) {
    // candidates: the one-wave rule and fixed sizes up to the largest system
    std::vector<long long> rows(sys_n.begin(), sys_n.end());
    int auto_rpc;
    if (inner == 1) {
        std::vector<long long> grows;
        for (const auto& g : bicg_groups(sys_n, sys_op, pinv, aval)) grows.push_back(sys_n[g.first]);
        auto_rpc = bicg_rows_per_chunk<T, S, C>(grows);
    } else {
        auto_rpc = sweep_rows_per_chunk<T, S, C>(rows, ortho);
    }
    const int nmax = *std::max_element(sys_n.begin(), sys_n.end());
    std::vector<int> cand{(auto_rpc + 31) / 32 * 32};
    for (int c : {512, 768, 1024, 1536, 2048, 4096, 8192})
        if (c <= std::max(nmax, 256) && std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
    // synthetic stencil values for every operator that has pre-scaled diagonals
    std::vector<Dev<C>> tav(aval.size());
    std::vector<C*> av(aval.size(), nullptr);
    for (size_t q = 0; q < aval.size(); ++q) {
        if (!aval[q]) continue;
        size_t f = q;
        for (size_t p = 0; p < q; ++p)
            if (aval[p] == aval[q]) { f = p; break; }
        if (f != q) { av[q] = av[f]; continue; }
        const OpDesc& od = ops[sys_op[q]];
        SYLV_TRY(tav[q].alloc((size_t)od.ndiag * od.n));
        k_fill_stencil<C><<<num_sms() * 2, 256, 0, s>>>(tav[q].p, od);
        av[q] = tav[q].p;
    }
    // one solution vector per system (a shared one would make the update
    // kernel's stores of all systems collide on the same addresses)
    Dev<T> xs;
    size_t xtot = 0;
    for (int q : sys_n) xtot += (size_t)q;
    SYLV_TRY(xs.alloc(xtot));
    SYLV_CK(cudaMemsetAsync(xs.p, 0, xtot * sizeof(T), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SYLV_CK(cudaEventCreate(&e0));
    SYLV_CK(cudaEventCreate(&e1));
    out->cand.clear();
    out->ms.clear();
    double best = 1e300;
    int rc = SYLV_OK;
    for (int c : cand) {
        Engine<T, S, C> eng;
        eng.ortho = ortho;
        eng.inner = inner;
        eng.pdl = 1;
        rc = eng.setup(sys_n, sys_op, ops, pinv, av, {}, 0, restart, c, s);
        if (rc != SYLV_OK) break;
        const int nsys = eng.nsys;
        if (inner == 1) {
            k_fill_pattern<C><<<num_sms() * 4, 256, 0, s>>>(eng.d_bv.p, eng.d_bv.count, 12345u);
        } else {
            k_fill_pattern<S><<<num_sms() * 4, 256, 0, s>>>(eng.d_V.p, eng.d_V.count, 12345u);
        }
        std::vector<SysState<T>> st(nsys);
        size_t xo = 0;
        for (int q = 0; q < nsys; ++q) {
            std::memset(&st[q], 0, sizeof(SysState<T>));
            st[q].phase = PH_ARNOLDI;
            st[q].max_iters = 1 << 30;
            st[q].tol = 0.0;
            st[q].x = xs.p + xo;
            xo += (size_t)sys_n[q];
            st[q].scale[0] = 1.0;
            st[q].g[0] = make_scalar<T>(1.0, 0.0);
            st[q].brho = make_scalar<T>(1.0, 0.0);
            st[q].balpha = make_scalar<T>(1.0, 0.0);
            st[q].bomega = make_scalar<T>(1.0, 0.0);
            st[q].bbeta = make_scalar<T>(0.5, 0.0);
            st[q].bnorm0 = NAN;                 // no drift restart during the probe
        }
        SYLV_CK(cudaMemcpyAsync(eng.d_st.p, st.data(), nsys * sizeof(SysState<T>), cudaMemcpyHostToDevice, s));
        BatchCtl cc{};
        cc.n_active = nsys;
        cc.nitems = eng.nitems;
        SYLV_CK(cudaMemcpyAsync(eng.d_ctl.p, &cc, sizeof(cc), cudaMemcpyHostToDevice, s));
        const int warm = inner == 1 ? 2 : 0, timed = inner == 1 ? 12 : std::max(1, restart - 1);
        for (int t = 0; t < warm; ++t) SYLV_TRY(eng.launch_tick(0, 0, false));
        SYLV_CK(cudaEventRecord(e0, s));
        for (int t = 0; t < timed; ++t) SYLV_TRY(eng.launch_tick(0, 0, false));
        SYLV_CK(cudaEventRecord(e1, s));
        SYLV_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        SYLV_CK(cudaEventElapsedTime(&ms, e0, e1));
        const double per = ms / timed;
        out->cand.push_back(c);
        out->ms.push_back(per);
        if (per < best) { best = per; out->chosen = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SYLV_CK(cudaStreamSynchronize(s));
    return rc;
}

// ---------------------------------------------------------------------------
// Standalone entry points for one operator: batched GMRES, CGS2, product.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_op_apply(OpDesc op, T sigma, int jacobi, const T* __restrict__ X, T* __restrict__ Y,
                           int ncols) {
    const long long total = (long long)op.n * ncols;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(idx / op.n), i = (int)(idx % op.n);
        const T* x = X + (size_t)c * op.n;
        T y;
        if (jacobi)
            y = op_row<T>(op, i, sigma, [&](int k) {
                return sdiv(make_scalar<T>(1.0, 0.0), shifted_diag(op, k, sigma)) * x[k];
            });
        else
            y = op_row<T>(op, i, sigma, [&](int k) { return x[k]; });
        Y[(size_t)c * op.n + i] = y;
    }
}

template <typename T>
int op_apply_t(const DevOp& op, T sigma, int jacobi, const void* X, void* Y, int ncols, cudaStream_t s) {
    if (!X || !Y || ncols < 0) { set_error("op_apply: null buffer or negative ncols"); return SYLV_ERR_INVALID; }
    if (ncols == 0 || op.desc.n == 0) return SYLV_OK;
    long long total = (long long)op.desc.n * ncols;
    int grid = (int)std::min<long long>((total + 255) / 256, (long long)num_sms() * 16);
    k_op_apply<T><<<grid, 256, 0, s>>>(op.desc, sigma, jacobi, (const T*)X, (T*)Y, ncols);
    SYLV_CK(cudaGetLastError());
    return SYLV_OK;
}

// dst = scale * (column col of a tile-major basis with tile stride tstride).
template <typename T>
__global__ void k_copy_scaled(const T* __restrict__ V, size_t tstride, int col, double scale, T* __restrict__ dst,
                              int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = scale * V[(size_t)(i >> 5) * tstride + (size_t)col * 32 + (i & 31)];
}

// Columns 0..k-1 of a column-major n x k block (leading dimension n) into a
// tile-major basis.
template <typename T>
__global__ void k_to_tiles(const T* __restrict__ src, int n, int k, T* __restrict__ V, size_t tstride) {
    const long long tot = (long long)n * k;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(q / n), i = (int)(q - (long long)l * n);
        V[(size_t)(i >> 5) * tstride + (size_t)l * 32 + (i & 31)] = src[q];
    }
}

// Stencil operators whose main diagonal is stored get the pre-scaled diagonals.
inline bool scaled_op_possible(const OpDesc& d) {
    if (d.fmt != 1) return false;
    for (int q = 0; q < d.ndiag; ++q)
        if (d.offs[q] == 0) return true;
    return false;
}

// Jacobi inverse and pre-scaled diagonals for one operator and shift.
template <typename T, typename C>
int shifted_op_setup(const OpDesc& op, T sigma, T* pinv, C* aval, cudaStream_t s) {
    if (!pinv && !aval) return SYLV_OK;
    const int grid = std::max(1, std::min(num_sms() * 4, (op.n + SYLV_BLOCK - 1) / SYLV_BLOCK));
    k_shifted_op<T, C><<<grid, SYLV_BLOCK, 0, s>>>(op, sigma, pinv, aval);
    SYLV_CK(cudaGetLastError());
    return SYLV_OK;
}

// Batched shifted solves of one operator: restarted GMRES (inner = 0) or
// BiCGstab (inner = 1, restart unused).
template <typename T, typename S, typename C>
int krylov_t(const DevOp& op, T sigma, int jacobi, const void* B, void* X, int ncols, double tol,
             int restart, int max_iters, int* iters, double* res, double* hist, cudaStream_t s, int inner) {
    const char* name = inner == 1 ? "bicgstab" : "gmres";
    if (inner == 1) restart = 1;
    if (!B || !X || ncols <= 0 || restart < 1 || restart > SYLV_MR || max_iters < 1) {
        set_error("%s: invalid arguments (ncols=%d restart=%d max_iters=%d)", name, ncols, restart, max_iters);
        return SYLV_ERR_INVALID;
    }
    const int n = op.desc.n;
    Engine<T, S, C> eng;
    eng.inner = inner;
    Dev<T> pinv;
    Dev<C> aval;
    Dev<double> d_hist;
    if (jacobi) SYLV_TRY(pinv.alloc(n));
    if (scaled_op_possible(op.desc)) SYLV_TRY(aval.alloc((size_t)op.desc.ndiag * n));
    if (hist) SYLV_TRY(d_hist.alloc((size_t)ncols * max_iters));
    std::vector<int> sn(ncols, n), so(ncols, 0);
    std::vector<T*> pv(ncols, jacobi ? pinv.p : nullptr);
    std::vector<C*> av(ncols, aval.p);
    std::vector<double*> hv;
    if (hist)
        for (int c = 0; c < ncols; ++c) hv.push_back(d_hist.p + (size_t)c * max_iters);
    std::vector<OpDesc> ops{op.desc};
    SYLV_TRY(eng.setup(sn, so, ops, pv, av, hv, max_iters, restart, 0, s));
    std::vector<SysState<T>> st(ncols);
    for (int c = 0; c < ncols; ++c) {
        std::memset(&st[c], 0, sizeof(SysState<T>));
        st[c].phase = PH_RESID;
        st[c].max_iters = max_iters;
        st[c].tol = tol;
        st[c].sigma = sigma;
        st[c].x = (T*)X + (size_t)c * n;
        st[c].b = (const T*)B + (size_t)c * n;
    }
    SYLV_CK(cudaMemcpyAsync(eng.d_st.p, st.data(), ncols * sizeof(SysState<T>), cudaMemcpyHostToDevice, s));
    BatchCtl c{};
    c.n_active = ncols;
    c.h_flag = eng.d_hflag;
    c.nitems = eng.nitems;
    SYLV_CK(cudaMemcpyAsync(eng.d_ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice, s));
    SYLV_TRY((shifted_op_setup<T, C>(op.desc, sigma, pinv.p, aval.p, s)));
    k_zero_x<T, S, C><<<eng.nitems, SYLV_BLOCK, 0, s>>>(eng.d_sd.p, eng.d_st.p, eng.d_items.p);
    SYLV_CK(cudaGetLastError());
    SYLV_CK(cudaStreamSynchronize(s));
    *eng.h_flag = 1;
    SYLV_TRY(eng.run((long long)max_iters + 8));
    SYLV_CK(cudaStreamSynchronize(s));
    SYLV_TRY(eng.take_stage_fault());
    SYLV_CK(cudaMemcpy(st.data(), eng.d_st.p, ncols * sizeof(SysState<T>), cudaMemcpyDeviceToHost));
    int stalled = 0;
    for (int c = 0; c < ncols; ++c) {
        if (iters) iters[c] = st[c].iters;
        if (res) res[c] = st[c].resnorm;
        stalled |= (st[c].status != ST_OK);
    }
    if (hist) {
        std::vector<double> hh((size_t)ncols * max_iters);
        SYLV_CK(cudaMemcpy(hh.data(), d_hist.p, hh.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (int c = 0; c < ncols; ++c)
            for (int i = 0; i < max_iters; ++i)
                hist[(size_t)c * max_iters + i] = i < st[c].iters ? hh[(size_t)c * max_iters + i] : 0.0;
    }
    for (int c = 0; c < ncols; ++c)
        if (st[c].status == ST_NONFINITE) { set_error("%s: non-finite value in column %d", name, c); return SYLV_ERR_NONFINITE; }
    if (stalled) { set_error("%s: a column reached max_iters", name); return SYLV_ERR_INNER_STALL; }
    return SYLV_OK;
}

template <typename T, typename S, typename C>
int gmres_t(const DevOp& op, T sigma, int jacobi, const void* B, void* X, int ncols, double tol,
            int restart, int max_iters, int* iters, double* res, double* hist, cudaStream_t s) {
    return krylov_t<T, S, C>(op, sigma, jacobi, B, X, ncols, tol, restart, max_iters, iters, res, hist, s, 0);
}

template <typename T, typename S, typename C>
int bicgstab_t(const DevOp& op, T sigma, int jacobi, const void* B, void* X, int ncols, double tol,
               int max_iters, int* iters, double* res, double* hist, cudaStream_t s) {
    return krylov_t<T, S, C>(op, sigma, jacobi, B, X, ncols, tol, 1, max_iters, iters, res, hist, s, 1);
}

// Column col of a tile-major basis (storage S) times scale, as T.
template <typename T, typename S>
__global__ void k_basis_column(const S* __restrict__ V, size_t tstride, int col, double scale, T* __restrict__ dst,
                               int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = scale * cvt<T>(V[(size_t)(i >> 5) * tstride + (size_t)col * 32 + (i & 31)]);
}

// v (T, length n) into slot 0 of a tile-major basis of storage S.
template <typename T, typename S>
__global__ void k_basis_set0(const T* __restrict__ v, int n, S* __restrict__ V, size_t tstride) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        V[(size_t)(i >> 5) * tstride + (i & 31)] = cvt<S>(v[i]);
}

// One Arnoldi cycle of k steps of the inner GMRES, as the solver runs it
// (precision S/C, CGS2 or delayed CGS2, right Jacobi): v0 (device, T) is the
// start vector; V_out (device, n x (k + 1), T) receives the basis vectors
// v_0 .. v_k as scale x stored vector (with DCGS2 v_k is not completed by
// the cycle and is left zero), H_out (host, (k + 1) x k, T, column-major) the
// Hessenberg matrix as formed.
template <typename T, typename S, typename C>
int arnoldi_t(const DevOp& op, T sigma, int jacobi, const void* v0, int k, int ortho, void* V_out, void* H_out,
              cudaStream_t s) {
    if (!v0 || !V_out || !H_out || k < 1 || k > SYLV_MR || (ortho != 0 && ortho != 1)) {
        set_error("arnoldi: invalid arguments (k=%d, 1 <= k <= %d, ortho=%d)", k, SYLV_MR, ortho);
        return SYLV_ERR_INVALID;
    }
    const int n = op.desc.n;
    Engine<T, S, C> eng;
    eng.ortho = ortho;
    Dev<T> pinv;
    Dev<C> aval;
    if (jacobi) SYLV_TRY(pinv.alloc(n));
    if (scaled_op_possible(op.desc)) SYLV_TRY(aval.alloc((size_t)op.desc.ndiag * n));
    const std::vector<int> sn{n}, so{0};
    const std::vector<T*> pv{jacobi ? pinv.p : nullptr};
    const std::vector<C*> av{aval.p};
    std::vector<OpDesc> ops{op.desc};
    SYLV_TRY(eng.setup(sn, so, ops, pv, av, {}, 0, k, 0, s));
    SYLV_TRY((shifted_op_setup<T, C>(op.desc, sigma, pinv.p, aval.p, s)));
    const SysDesc<T, S, C>& d = eng.h_sd[0];
    k_basis_set0<T, S><<<num_sms() * 4, 256, 0, s>>>((const T*)v0, n, d.V, d.tstride);
    SYLV_CK(cudaGetLastError());
    SysState<T> st;
    std::memset(&st, 0, sizeof(st));
    st.phase = PH_ARNOLDI;
    st.j = 0;
    st.scale[0] = 1.0;
    st.g[0] = make_scalar<T>(1.0, 0.0);
    st.tol = 0.0;                         // the cycle runs to its restart length
    st.max_iters = k;
    st.sigma = sigma;
    SYLV_CK(cudaMemcpyAsync(eng.d_st.p, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    BatchCtl c{};
    c.n_active = 1;
    c.h_flag = eng.d_hflag;
    c.nitems = eng.nitems;
    SYLV_CK(cudaMemcpyAsync(eng.d_ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice, s));
    // k steps (CGS2), k + 1 device iterations with the delayed second pass;
    // iterations after the cycle's end find the system in the update phase
    for (int t = 0; t < k + 1; ++t) SYLV_TRY(eng.launch_tick(0, 0, false));
    SYLV_CK(cudaStreamSynchronize(s));
    SYLV_CK(cudaMemcpy(&st, eng.d_st.p, sizeof(st), cudaMemcpyDeviceToHost));
    if (st.phase != PH_UPDATE || st.nvec != k) {
        set_error("arnoldi: the cycle ended after %d of %d steps (breakdown or non-finite value)", st.nvec, k);
        return SYLV_ERR_NONFINITE;
    }
    T* Vo = (T*)V_out;
    SYLV_CK(cudaMemsetAsync(Vo, 0, (size_t)n * (k + 1) * sizeof(T), s));
    const int last = ortho == 1 ? k - 1 : k;
    for (int l = 0; l <= last; ++l) {
        k_basis_column<T, S><<<num_sms() * 4, 256, 0, s>>>(d.V, d.tstride, l, st.scale[l], Vo + (size_t)l * n, n);
        SYLV_CK(cudaGetLastError());
    }
    SYLV_CK(cudaStreamSynchronize(s));
    T* ho = (T*)H_out;
    for (int j = 0; j < k; ++j)
        for (int i = 0; i <= k; ++i) ho[(size_t)j * (k + 1) + i] = i <= j + 1 ? st.Hr[j * SYLV_MAXV + i] : zero<T>();
    return SYLV_OK;
}

template <typename T>
int cgs2_t(const void* V, int n, int k, void* w, void* h, cudaStream_t s) {
    if (!V || !w || !h || n <= 0 || k < 1 || k > SYLV_MR) {
        set_error("cgs2: invalid arguments (n=%d k=%d, 1 <= k <= %d)", n, k, SYLV_MR);
        return SYLV_ERR_INVALID;
    }
    Engine<T, T, T> eng;
    DevOp dummy;
    dummy.desc.n = n;
    std::vector<OpDesc> ops{dummy.desc};
    const std::vector<int> sn{n}, so{0};
    const std::vector<T*> pv{nullptr};
    SYLV_TRY(eng.setup(sn, so, ops, pv, std::vector<T*>(), std::vector<double*>(), 0, k, 0, s));
    const SysDesc<T, T, T>& d = eng.h_sd[0];
    k_to_tiles<T><<<num_sms() * 4, 256, 0, s>>>((const T*)V, n, k, d.V, d.tstride);
    SYLV_CK(cudaGetLastError());
    SYLV_CK(cudaMemcpyAsync(d.w, w, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SysState<T> st;
    std::memset(&st, 0, sizeof(st));
    st.phase = PH_ARNOLDI;
    st.j = k - 1;
    for (int l = 0; l < k; ++l) st.scale[l] = 1.0;
    SYLV_CK(cudaMemcpyAsync(eng.d_st.p, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    BatchCtl c{};
    c.n_active = 1;
    c.h_flag = eng.d_hflag;
    c.nitems = eng.nitems;
    SYLV_CK(cudaMemcpyAsync(eng.d_ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice, s));
    SYLV_TRY(eng.launch_tick(1));
    SYLV_CK(cudaStreamSynchronize(s));
    SYLV_CK(cudaMemcpy(&st, eng.d_st.p, sizeof(st), cudaMemcpyDeviceToHost));
    k_copy_scaled<T><<<num_sms() * 4, 256, 0, s>>>(d.V, d.tstride, k, st.scale[k], (T*)w, n);
    SYLV_CK(cudaGetLastError());
    SYLV_CK(cudaStreamSynchronize(s));
    T* ho = (T*)h;
    for (int l = 0; l <= k; ++l) ho[l] = st.R[(k - 1) * SYLV_MAXV + l];
    return SYLV_OK;
}

// ---------------------------------------------------------------------------
// The inexact LR-ADI solver (Algorithm 1) on one GPU.
// ---------------------------------------------------------------------------
template <typename T, typename S, typename C>
struct Adi : AdiBase {
    AdiDev<T, S, C> d{};
    Engine<T, S, C> eng;
    cudaStream_t stream = nullptr;
    int n = 0, m = 0, r = 0, kmax = 0, max_inner = 0;
    Dev<double> f, g, hist;
    Dev<T> w, t, Z, Y, gam, alpha, beta, pinvA, pinvB, gpart;
    Dev<C> avalA, avalB;
    Dev<AdiState<T>> st;
    TuneResult tune;                // chunk-size autotuner (opts.autotune)
    // real double steps of conjugate pairs (complex shifts, opts.real_pairs)
    int real_pairs = 0;
    Dev<T> XA, XB, XA2, XB2;
    Dev<double> Zr, Yr, core_rec, RsA, RsB, pgpart;
    int* h_done = nullptr;
    int* d_hdone = nullptr;
    int solved = 0;
    int last_status = SYLV_ERR_NOT_SOLVED;
    long long ticks = 0;
    long long launches_last = 0;

    ~Adi() override {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (h_done) cudaFreeHost(h_done);
        for (auto& e : aev)
            if (e) cudaEventDestroy(e);
    }

    int profile(int on) override { return eng.set_profile(on); }

    int kernel_stats(double* ms, double* bytes, double* flops, long long* launches) const override {
        double b[K_COUNT], f[K_COUNT];
        SYLV_TRY(eng.read_work(b, f));
        for (int q = 0; q < K_COUNT; ++q) {
            // sampled mean duration times all launches
            if (ms) ms[q] = eng.samples[q] > 0 ? eng.kernel_ms[q] / eng.samples[q] * eng.launches[q] : 0.0;
            if (bytes) bytes[q] = b[q];
            if (flops) flops[q] = f[q];
            if (launches) launches[q] = eng.launches[q];
        }
        return SYLV_OK;
    }

    int init(const AdiArgs& a) {
        stream = a.stream;
        n = a.n; m = a.m; r = a.r; kmax = a.o.kmax; max_inner = a.o.max_inner;
        std::vector<long long> rows;
        for (int l = 0; l < r; ++l) { rows.push_back(n); rows.push_back(m); }
        // BiCGstab: the r columns of each side form one group
        const std::vector<long long> grows{(long long)n, (long long)m};
        int rpc = a.o.rows_per_chunk > 0 ? a.o.rows_per_chunk
                  : a.o.inner == SYLV_INNER_BICGSTAB ? bicg_rows_per_chunk<T, S, C>(grows)
                                                     : sweep_rows_per_chunk<T, S, C>(rows, a.o.ortho);
        real_pairs = (a.o.real_pairs && sizeof(T) == sizeof(cplx)) ? 1 : 0;
        // a pair that starts at step kmax ends at kmax + 1
        const int ksl = kmax + real_pairs;
        SYLV_TRY(f.alloc((size_t)n * r));
        SYLV_TRY(g.alloc((size_t)m * r));
        SYLV_TRY(w.alloc((size_t)n * r));
        SYLV_TRY(t.alloc((size_t)m * r));
        if (real_pairs) {
            // real factors; the solves write complex work blocks
            SYLV_TRY(Zr.alloc((size_t)n * r * ksl));
            SYLV_TRY(Yr.alloc((size_t)m * r * ksl));
            SYLV_TRY(core_rec.alloc((size_t)ksl * 5));
            SYLV_TRY(XA.alloc((size_t)n * r));
            SYLV_TRY(XB.alloc((size_t)m * r));
            SYLV_TRY(XA2.alloc((size_t)n * r));
            SYLV_TRY(XB2.alloc((size_t)m * r));
            SYLV_TRY(RsA.alloc((size_t)n * r));
            SYLV_TRY(RsB.alloc((size_t)m * r));
            SYLV_CK(cudaMemset(core_rec.p, 0, core_rec.count * sizeof(double)));
        } else {
            SYLV_TRY(Z.alloc((size_t)n * r * kmax));
            SYLV_TRY(Y.alloc((size_t)m * r * kmax));
        }
        SYLV_TRY(gam.alloc((size_t)r * kmax));
        SYLV_TRY(hist.alloc((size_t)ksl * SYLV_HIST_COLS));
        SYLV_TRY(alpha.alloc(a.nshift));
        SYLV_TRY(beta.alloc(a.nshift));
        if (a.o.jacobi) {
            SYLV_TRY(pinvA.alloc(n));
            SYLV_TRY(pinvB.alloc(m));
        }
        if (scaled_op_possible(a.A->desc)) SYLV_TRY(avalA.alloc((size_t)a.A->desc.ndiag * n));
        if (scaled_op_possible(a.Bt->desc)) SYLV_TRY(avalB.alloc((size_t)a.Bt->desc.ndiag * m));
        SYLV_TRY(st.alloc(1));
        SYLV_CK(cudaMemset(st.p, 0, sizeof(AdiState<T>)));
        if (Z.p) SYLV_CK(cudaMemset(Z.p, 0, Z.count * sizeof(T)));
        if (Y.p) SYLV_CK(cudaMemset(Y.p, 0, Y.count * sizeof(T)));
        SYLV_CK(cudaMemset(hist.p, 0, hist.count * sizeof(double)));
        std::vector<T> ha(a.nshift), hb(a.nshift);
        for (int i = 0; i < a.nshift; ++i) {
            ha[i] = make_scalar<T>(a.alpha[i].re, a.alpha[i].im);
            hb[i] = make_scalar<T>(a.beta[i].re, a.beta[i].im);
        }
        SYLV_CK(cudaMemcpy(alpha.p, ha.data(), a.nshift * sizeof(T), cudaMemcpyHostToDevice));
        SYLV_CK(cudaMemcpy(beta.p, hb.data(), a.nshift * sizeof(T), cudaMemcpyHostToDevice));
        SYLV_TRY(set_rhs(a.f, a.g, 0));
        // 2r column systems: A side uses operator 0, B side operator 1 (B^T).
        std::vector<int> sn, so;
        std::vector<T*> pv;
        std::vector<C*> av;
        for (int l = 0; l < r; ++l) { sn.push_back(n); so.push_back(0); pv.push_back(pinvA.p); av.push_back(avalA.p); }
        for (int l = 0; l < r; ++l) { sn.push_back(m); so.push_back(1); pv.push_back(pinvB.p); av.push_back(avalB.p); }
        std::vector<OpDesc> ops{a.A->desc, a.Bt->desc};
        eng.ortho = a.o.ortho;
        eng.inner = a.o.inner;
        if (a.o.autotune && a.o.rows_per_chunk <= 0) {
            SYLV_TRY((autotune_rpc<T, S, C>(sn, so, ops, pv, av, a.o.restart, a.o.ortho, a.o.inner, stream, &tune)));
            if (tune.chosen > 0) rpc = tune.chosen;
        }
        SYLV_TRY(eng.setup(sn, so, ops, pv, av, {}, 0, a.o.restart, rpc, stream));
        const int nchA = (n + rpc - 1) / rpc, nchB = (m + rpc - 1) / rpc;
        SYLV_TRY(gpart.alloc((size_t)(nchA + nchB) * SYLV_GSTRIDE));
        // chunk partials, then the two reduced Gram sets of k_adi_pair_finish
        if (real_pairs) SYLV_TRY(pgpart.alloc((size_t)(nchA + nchB + 2) * SYLV_PGSTRIDE));
        SYLV_CK(cudaHostAlloc((void**)&h_done, sizeof(int), cudaHostAllocMapped));
        *h_done = 0;
        SYLV_CK(cudaHostGetDevicePointer((void**)&d_hdone, h_done, 0));
        d.n = n; d.m = m; d.r = r; d.kmax = kmax; d.nshift = a.nshift;
        d.strategy = a.o.strategy; d.bl_clamp = a.o.bl_clamp; d.max_inner = max_inner;
        d.tau = a.tau; d.xi = a.o.xi;
        d.dminA = a.o.dmin_A; d.dminB = a.o.dmin_B; d.dmaxA = a.o.dmax_A; d.dmaxB = a.o.dmax_B;
        d.fixed_tol = a.o.fixed_tol;
        d.alpha = alpha.p; d.beta = beta.p;
        d.f = f.p; d.g = g.p; d.w = w.p; d.t = t.p; d.Z = Z.p; d.Y = Y.p; d.gam = gam.p;
        d.hist = hist.p;
        d.opA = a.A->desc; d.opB = a.Bt->desc;
        d.pinvA = pinvA.p; d.pinvB = pinvB.p;
        d.avalA = avalA.p; d.avalB = avalB.p;
        d.sd = eng.d_sd.p; d.st = eng.d_st.p; d.ctl = eng.d_ctl.p;
        d.gpart = gpart.p; d.nchA = nchA; d.nchB = nchB; d.rpc = rpc;
        d.s = st.p; d.h_done = d_hdone;
        d.real_pairs = real_pairs;
        d.XA = XA.p; d.XB = XB.p; d.XA2 = XA2.p; d.XB2 = XB2.p;
        d.Zr = Zr.p; d.Yr = Yr.p; d.core = core_rec.p; d.RsA = RsA.p; d.RsB = RsB.p; d.pgpart = pgpart.p;
        graph_on = a.o.driver == 0 ? 1 : 0;
        eng.restart_every = a.o.restart_every;
        return SYLV_OK;
    }

    int set_rhs(const double* hf, const double* hg, int on_device) override {
        if (!hf || !hg) { set_error("set_rhs: null f or g"); return SYLV_ERR_INVALID; }
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        SYLV_CK(cudaMemcpyAsync(f.p, hf, (size_t)n * r * sizeof(double), kind, stream));
        SYLV_CK(cudaMemcpyAsync(g.p, hg, (size_t)m * r * sizeof(double), kind, stream));
        if (!on_device) SYLV_CK(cudaStreamSynchronize(stream));
        return SYLV_OK;
    }

    // event pairs around the outer-step kernels when profiling
    cudaEvent_t aev[4] = {};
    int ensure_events() {
        if (!aev[0])
            for (auto& e : aev) SYLV_CK(cudaEventCreate(&e));
        return SYLV_OK;
    }
    int add_ms(int kid, cudaEvent_t a, cudaEvent_t b) {
        float ms = 0.f;
        SYLV_CK(cudaEventElapsedTime(&ms, a, b));
        eng.kernel_ms[kid] += ms;
        eng.samples[kid] += 1;
        return SYLV_OK;
    }

    // ---- device-driven solve: one CUDA graph with conditional nodes ----
    //   gram(init) -> WHILE(h_outer) { controller -> step_init ->
    //       WHILE(h_loop) { spmv -> pass2 -> pass3 -> IF(h_restart) { update -> residual } }
    //       -> gram(update) }
    // The kernels set the conditions (pass3/residual: grid-level last block;
    // controller and gram: their deciding thread), so no host round trip
    // happens inside a solve.
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_on = 1;             // 0: host-driven loop (used while profiling)
    int h_one = 1, h_zero = 0;

    int add_kernel(cudaGraphNode_t* node, cudaGraph_t g, cudaGraphNode_t* dep, void* func, int grid,
                   int block, void** args, int smem = 0) {
        cudaKernelNodeParams kp = {};
        kp.func = func;
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(block);
        kp.sharedMemBytes = smem;
        kp.kernelParams = args;
        kp.extra = nullptr;
        SYLV_CK(cudaGraphAddKernelNode(node, g, dep, dep ? 1 : 0, &kp));
        return SYLV_OK;
    }

    int add_cond(cudaGraphNode_t* node, cudaGraph_t g, cudaGraphNode_t* dep, cudaGraphConditionalHandle h,
                 cudaGraphConditionalNodeType type, cudaGraph_t* body) {
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = type;
        p.conditional.size = 1;
        SYLV_CK(cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &p));
        *body = p.conditional.phGraph_out[0];
        return SYLV_OK;
    }

    // The graph of a solve; if the device-updatable step-kernel nodes are
    // refused at instantiation, the graph is built again without them.
    int build_graph() {
        int rc = build_graph_once(true);
        if (rc != SYLV_OK && eng.dyn_grid) {
            (void)cudaGetLastError();
            if (gexec) cudaGraphExecDestroy(gexec);
            if (graph) cudaGraphDestroy(graph);
            graph = nullptr;
            gexec = nullptr;
            rc = build_graph_once(false);
        }
        return rc;
    }

    int build_graph_once(bool try_dyn) {
        const int nb = d.nchA + d.nchB;
        const int ni = eng.nitems;
        int one = 1, zero = 0, mode0 = 0;
        cudaGraph_t g;
        SYLV_CK(cudaGraphCreate(&g, 0));
        graph = g;
        cudaGraphConditionalHandle h_outer, h_loop, h_restart;
        // every condition starts at 0 on each launch: a loop runs only while a
        // kernel has explicitly asked for another pass
        SYLV_CK(cudaGraphConditionalHandleCreate(&h_outer, g, 0, cudaGraphCondAssignDefault));
        void* a_init[] = {&d, &one};
        void* a_upd[] = {&d, &zero};
        void* a_d[] = {&d};
        cudaGraphNode_t n_init, n_outer, n_ctrl, n_step, n_loop, n_gram, n1, n2, n3, n_if, n4, n5;
        SYLV_TRY(add_kernel(&n_init, g, nullptr, (void*)k_adi_gram<T, S, C>, nb, SYLV_BLOCK, a_init));
        cudaGraph_t outer_body, loop_body, if_body;
        SYLV_TRY(add_cond(&n_outer, g, &n_init, h_outer, cudaGraphCondTypeWhile, &outer_body));
        SYLV_CK(cudaGraphConditionalHandleCreate(&h_loop, outer_body, 0, cudaGraphCondAssignDefault));
        SYLV_TRY(add_kernel(&n_ctrl, outer_body, nullptr, (void*)k_adi_controller<T, S, C>, 1, 32, a_d));
        SYLV_TRY(add_kernel(&n_step, outer_body, &n_ctrl, (void*)k_adi_step_init<T, S, C>, nb, SYLV_BLOCK, a_d));
        SYLV_TRY(add_cond(&n_loop, outer_body, &n_step, h_loop, cudaGraphCondTypeWhile, &loop_body));
        SYLV_TRY(add_kernel(&n_gram, outer_body, &n_loop, (void*)k_adi_gram<T, S, C>, nb, SYLV_BLOCK, a_upd));
        SYLV_CK(cudaGraphConditionalHandleCreate(&h_restart, loop_body, 0, cudaGraphCondAssignDefault));
        auto* sdp = eng.d_sd.p;
        auto* stp = eng.d_st.p;
        auto* opp = eng.d_ops.p;
        auto* itp = eng.d_items.p;
        auto* ctp = eng.d_ctl.p;
        void* a1[] = {&sdp, &stp, &opp, &itp, &ctp, &mode0};
        void* a2[] = {&sdp, &stp, &itp, &ctp};
        int nsysb = eng.nsys;
        void* ab[] = {&sdp, &stp, &itp, &ctp, &nsysb};
        void* a3[] = {&sdp, &stp, &itp, &ctp, &mode0};
        void* a4[] = {&sdp, &stp, &itp, &ctp};
        void* a5[] = {&sdp, &stp, &opp, &itp, &ctp};
        const int sm = sweep_smem_bytes<S, C>();
        auto* grp = eng.d_groups.p;
        auto* gip = eng.d_gitems.p;
        int ngi = eng.ngitems;
        void* br[] = {&sdp, &stp, &opp, &grp, &gip, &ngi, &ctp};
        if (eng.inner == 1) {
            SYLV_TRY(eng.add_bicg_nodes(loop_body, nullptr, &n3, try_dyn));
        } else if (eng.ortho == 1) {
            SYLV_TRY(add_kernel(&n1, loop_body, nullptr, (void*)k_dcgs_a<T, S, C>, ni, SYLV_BLOCK, a5,
                                dcgs_a_smem_bytes<T, S, C>()));
            SYLV_TRY(add_kernel(&n3, loop_body, &n1, (void*)k_dcgs_b<T, S, C>, ni + nsysb, SYLV_BLOCK, ab,
                                dcgs_b_smem_bytes<T, S, C>()));
        } else {
            SYLV_TRY(add_kernel(&n1, loop_body, nullptr, (void*)k_arnoldi_spmv<T, S, C>, ni, SYLV_BLOCK, a1, sm));
            SYLV_TRY(add_kernel(&n2, loop_body, &n1, (void*)k_cgs_pass2<T, S, C>, ni, SYLV_BLOCK, a2, sm));
            SYLV_TRY(add_kernel(&n3, loop_body, &n2, (void*)k_cgs_pass3<T, S, C>, ni, SYLV_BLOCK, a3, sm));
        }
        SYLV_TRY(add_cond(&n_if, loop_body, &n3, h_restart, cudaGraphCondTypeIf, &if_body));
        const int rg = eng.restart_grid();
        if (eng.inner == 1) {
            SYLV_TRY(add_kernel(&n5, if_body, nullptr, (void*)k_bicg_resid<T, S, C>, rg, SYLV_BLOCK, br));
        } else {
            SYLV_TRY(add_kernel(&n4, if_body, nullptr, (void*)k_restart_update<T, S, C>, rg, SYLV_BLOCK, a4));
            SYLV_TRY(add_kernel(&n5, if_body, &n4, (void*)k_restart_residual<T, S, C>, rg, SYLV_BLOCK, a5));
        }
        SYLV_CK(cudaGraphInstantiate(&gexec, g, 0));
        // kernels of the graph update nodes of the graph: upload it first
        if (eng.dyn_grid) SYLV_CK(cudaGraphUpload(gexec, stream));
        // the kernels read the handles and the decision parameters from the control block
        BatchCtl c{};
        SYLV_CK(cudaMemcpy(&c, eng.d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost));
        c.h_outer = h_outer;
        c.h_loop = h_loop;
        c.h_restart = h_restart;
        c.nsys = eng.nsys;
        c.max_ticks = max_inner + 8;
        c.graph = 0;
        eng.set_dyn_fields(c);
        SYLV_CK(cudaMemcpy(eng.d_ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice));
        return SYLV_OK;
    }

    unsigned long long device_launches() const {
        BatchCtl c{};
        if (cudaMemcpy(&c, eng.d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
        unsigned long long s = 0;
        for (int q = 0; q < K_COUNT; ++q) s += c.launch_count[q];
        return s;
    }

    int finish_solve(unsigned long long l0) {
        SYLV_CK(cudaStreamSynchronize(stream));
        SYLV_TRY(eng.take_stage_fault());
        launches_last = (long long)(device_launches() - l0);
        AdiState<T> s;
        SYLV_CK(cudaMemcpy(&s, st.p, sizeof(s), cudaMemcpyDeviceToHost));
        BatchCtl c{};
        SYLV_CK(cudaMemcpy(&c, eng.d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost));
        solved = 1;
        if (s.status == 2) { set_error("non-finite value during the solve"); last_status = SYLV_ERR_NONFINITE; }
        else if (s.status == 1 || !s.done) { set_error("kmax outer steps without reaching tau"); last_status = SYLV_ERR_MAXIT; }
        else if (s.stalled > 0) { set_error("%d inner solves reached max_inner", s.stalled); last_status = SYLV_ERR_INNER_STALL; }
        else last_status = SYLV_OK;
        return last_status;
    }

    int solve_graph() {
        if (!gexec) SYLV_TRY(build_graph());
        const unsigned long long l0 = device_launches();
        BatchCtl* dc = eng.d_ctl.p;
        SYLV_CK(cudaMemcpyAsync(&dc->graph, &h_one, sizeof(int), cudaMemcpyHostToDevice, stream));
        SYLV_CK(cudaGraphLaunch(gexec, stream));
        SYLV_CK(cudaMemcpyAsync(&dc->graph, &h_zero, sizeof(int), cudaMemcpyHostToDevice, stream));
        ticks = -1;   // not tracked on the host in this mode
        return finish_solve(l0);
    }

    int solve() override {
        if (real_pairs) return solve_pairs();
        if (graph_on && !eng.profile) return solve_graph();
        return solve_host();
    }

    int launch_pair_update(int nb) {
        switch (r) {
            case 1:
                k_adi_pair_update<T, S, C, 1><<<nb, SYLV_BLOCK, 0, stream>>>(d);
                k_adi_pair_finish<T, S, C, 1><<<1, 32, 0, stream>>>(d);
                break;
            case 2:
                k_adi_pair_update<T, S, C, 2><<<nb, SYLV_BLOCK, 0, stream>>>(d);
                k_adi_pair_finish<T, S, C, 2><<<1, 32, 0, stream>>>(d);
                break;
            case 3:
                k_adi_pair_update<T, S, C, 3><<<nb, SYLV_BLOCK, 0, stream>>>(d);
                k_adi_pair_finish<T, S, C, 3><<<1, 32, 0, stream>>>(d);
                break;
            default:
                k_adi_pair_update<T, S, C, 4><<<nb, SYLV_BLOCK, 0, stream>>>(d);
                k_adi_pair_finish<T, S, C, 4><<<1, 32, 0, stream>>>(d);
                break;
        }
        SYLV_CK(cudaGetLastError());
        eng.launches[K_GRAM]++;
        return SYLV_OK;
    }

    // Host-driven solve with the real double step of conjugate pairs: per
    // (double) step, controller -> set-up -> first solves -> pair_mid ->
    // (second solves of real-shift sides) -> pair update.
    int solve_pairs() {
        const int nb = d.nchA + d.nchB;
        const unsigned long long dl0 = device_launches();
        *h_done = 0;
        k_adi_gram<T, S, C><<<nb, SYLV_BLOCK, 0, stream>>>(d, 1);
        SYLV_CK(cudaGetLastError());
        eng.launches[K_GRAM]++;
        long long t0 = eng.ticks;
        for (int step = 0; step <= kmax + 1; ++step) {
            SYLV_CK(cudaStreamSynchronize(stream));
            if (*(volatile int*)h_done) break;
            *eng.h_flag = 1;
            k_adi_controller<T, S, C><<<1, 32, 0, stream>>>(d);
            k_adi_step_init<T, S, C><<<nb, SYLV_BLOCK, 0, stream>>>(d);
            SYLV_CK(cudaGetLastError());
            eng.launches[K_CTRL]++; eng.launches[K_STEP]++;
            SYLV_TRY(eng.run((long long)max_inner + 8));
            k_adi_pair_mid<T, S, C><<<nb, SYLV_BLOCK, 0, stream>>>(d);
            SYLV_CK(cudaGetLastError());
            SYLV_CK(cudaStreamSynchronize(stream));
            if (*(volatile int*)eng.h_flag) SYLV_TRY(eng.run((long long)max_inner + 8));
            SYLV_TRY(launch_pair_update(nb));
        }
        SYLV_CK(cudaStreamSynchronize(stream));
        ticks = eng.ticks - t0;
        return finish_solve(dl0);
    }

    int is_real() const override { return sizeof(T) == sizeof(double) || real_pairs; }

    int tuning(int* chosen, int* cand, double* ms, int cap, int* count) const override {
        if (chosen) *chosen = tune.chosen > 0 ? tune.chosen : eng.h_sd[0].rows_per_chunk;
        const int nc = (int)tune.cand.size();
        for (int q = 0; q < nc && q < cap; ++q) {
            if (cand) cand[q] = tune.cand[q];
            if (ms) ms[q] = tune.ms[q];
        }
        if (count) *count = nc;
        return SYLV_OK;
    }

    int core(double* G, int ld, int* kr) const override {
        AdiState<T> s;
        SYLV_CK(cudaMemcpy(&s, st.p, sizeof(s), cudaMemcpyDeviceToHost));
        const int steps = solved ? s.k - 1 : 0;
        const int ncol = steps * r;
        if (kr) *kr = ncol;
        if (!is_real()) {
            set_error("complex factors: the core is the diagonal gamma of sylv_adi_factors");
            return SYLV_ERR_UNSUPPORTED;
        }
        if (!G) return SYLV_OK;
        if (ld < ncol) { set_error("core: ld %d < kr %d", ld, ncol); return SYLV_ERR_INVALID; }
        for (int c = 0; c < ncol; ++c)
            for (int q = 0; q < ncol; ++q) G[q + (size_t)c * ld] = 0.0;
        if (!real_pairs) {
            std::vector<double> gh(ncol);
            if (ncol) SYLV_CK(cudaMemcpy(gh.data(), gam.p, ncol * sizeof(double), cudaMemcpyDeviceToHost));
            for (int c = 0; c < ncol; ++c) G[c + (size_t)c * ld] = gh[c];
            return SYLV_OK;
        }
        std::vector<double> rec((size_t)std::max(steps, 1) * 5);
        if (steps) SYLV_CK(cudaMemcpy(rec.data(), core_rec.p, (size_t)steps * 5 * sizeof(double), cudaMemcpyDeviceToHost));
        int c0 = 0;
        for (int k = 0; k < steps; ++k) {
            const double* e = &rec[(size_t)k * 5];
            if (e[0] == 1.0) {
                for (int l = 0; l < r; ++l) G[(c0 + l) + (size_t)(c0 + l) * ld] = e[1];
                c0 += r;
            } else if (e[0] == 2.0) {
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q)
                        for (int l = 0; l < r; ++l) G[(c0 + p * r + l) + (size_t)(c0 + q * r + l) * ld] = e[1 + 2 * p + q];
                c0 += 2 * r;
            }
        }
        return SYLV_OK;
    }

    int solve_host() {
        const int nb = d.nchA + d.nchB;
        const bool prof = eng.profile != 0;
        if (prof) SYLV_TRY(ensure_events());
        const unsigned long long dl0 = device_launches();
        long long l0 = 0;
        for (int q = 0; q < K_COUNT; ++q) l0 += eng.launches[q];
        *h_done = 0;
        if (prof) SYLV_CK(cudaEventRecord(aev[2], stream));
        k_adi_gram<T, S, C><<<nb, SYLV_BLOCK, 0, stream>>>(d, 1);
        if (prof) SYLV_CK(cudaEventRecord(aev[3], stream));
        SYLV_CK(cudaGetLastError());
        eng.launches[K_GRAM]++;
        long long t0 = eng.ticks;
        bool have_step = false;
        for (int step = 0; step <= kmax; ++step) {
            SYLV_CK(cudaStreamSynchronize(stream));
            if (prof) {
                SYLV_TRY(add_ms(K_GRAM, aev[2], aev[3]));
                if (have_step) SYLV_TRY(add_ms(K_CTRL, aev[0], aev[1]));
            }
            if (*(volatile int*)h_done) break;
            *eng.h_flag = 1;
            if (prof) SYLV_CK(cudaEventRecord(aev[0], stream));
            k_adi_controller<T, S, C><<<1, 32, 0, stream>>>(d);
            k_adi_step_init<T, S, C><<<nb, SYLV_BLOCK, 0, stream>>>(d);
            if (prof) SYLV_CK(cudaEventRecord(aev[1], stream));
            SYLV_CK(cudaGetLastError());
            eng.launches[K_CTRL]++; eng.launches[K_STEP]++;
            have_step = true;
            SYLV_TRY(eng.run((long long)max_inner + 8));
            if (prof) SYLV_CK(cudaEventRecord(aev[2], stream));
            k_adi_gram<T, S, C><<<nb, SYLV_BLOCK, 0, stream>>>(d, 0);
            if (prof) SYLV_CK(cudaEventRecord(aev[3], stream));
            SYLV_CK(cudaGetLastError());
            eng.launches[K_GRAM]++;
        }
        SYLV_CK(cudaStreamSynchronize(stream));
        ticks = eng.ticks - t0;
        (void)l0;
        return finish_solve(dl0);
    }

    int info(sylv_info* out) const override {
        AdiState<T> s;
        SYLV_CK(cudaMemcpy(&s, st.p, sizeof(s), cudaMemcpyDeviceToHost));
        std::memset(out, 0, sizeof(*out));
        out->status = last_status;
        out->steps = solved ? s.k - 1 : 0;
        out->kr = out->steps * r;
        out->is_complex = is_real() ? 0 : 1;
        out->rel_res_comp = s.nfg > 0 ? s.res / s.nfg : 0.0;
        out->norm_fg = s.nfg;
        out->inner_its_A = s.itsA;
        out->inner_its_B = s.itsB;
        out->inner_restarts = s.cycles;
        out->stalled_solves = s.stalled;
        out->ticks = (int32_t)ticks;
        out->launches = launches_last;
        return SYLV_OK;
    }

    int history(double* buf, int cap, int* rows) const override {
        AdiState<T> s;
        SYLV_CK(cudaMemcpy(&s, st.p, sizeof(s), cudaMemcpyDeviceToHost));
        int nrow = solved ? std::min(cap, s.k - 1) : 0;
        if (nrow > 0)
            SYLV_CK(cudaMemcpy(buf, hist.p, (size_t)nrow * SYLV_HIST_COLS * sizeof(double), cudaMemcpyDeviceToHost));
        if (rows) *rows = nrow;
        return SYLV_OK;
    }

    int factors(void* Zo, void* Yo, void* go, int on_device, int* kr) const override {
        AdiState<T> s;
        SYLV_CK(cudaMemcpy(&s, st.p, sizeof(s), cudaMemcpyDeviceToHost));
        const int steps = solved ? s.k - 1 : 0;
        const size_t ncol = (size_t)steps * r;
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (kr) *kr = (int)ncol;
        if (real_pairs) {
            if (go) { set_error("real double steps: the core has 2 x 2 blocks, use sylv_adi_core (gamma must be NULL)"); return SYLV_ERR_INVALID; }
            if (Zo && ncol) SYLV_CK(cudaMemcpy(Zo, Zr.p, ncol * n * sizeof(double), kind));
            if (Yo && ncol) SYLV_CK(cudaMemcpy(Yo, Yr.p, ncol * m * sizeof(double), kind));
            return SYLV_OK;
        }
        if (Zo && ncol) SYLV_CK(cudaMemcpy(Zo, Z.p, ncol * n * sizeof(T), kind));
        if (Yo && ncol) SYLV_CK(cudaMemcpy(Yo, Y.p, ncol * m * sizeof(T), kind));
        if (go && ncol) SYLV_CK(cudaMemcpy(go, gam.p, ncol * sizeof(T), kind));
        return SYLV_OK;
    }
};

template <typename T, typename S, typename C>
int make_adi_t(const AdiArgs& a, AdiBase** out) {
    Adi<T, S, C>* p = new (std::nothrow) Adi<T, S, C>();
    if (!p) { set_error("host allocation failed"); return SYLV_ERR_NOMEM; }
    int rc = p->init(a);
    if (rc != SYLV_OK) { delete p; return rc; }
    *out = p;
    return SYLV_OK;
}

}  // namespace sylv
