// batch.cuh - many independent Sylvester equations solved in one device loop.
//
// Every instance runs its own inexact LR-ADI iteration (Algorithm 1) with its
// own operators, rank, shifts and tolerance.  All 2 r_i column systems of all
// instances share one set of GMRES sweep launches (one work list of
// (system, row chunk) items), and instances move between outer steps on their
// own: a device iteration of the batch is
//
//   outer  : instances whose inner solves are all done (or that have not
//            started) take the factor update + Grams + stop test, then the
//            controller of their next step (Sec. 3.3)
//   step   : shifted-operator set-up and zeroed solution slots for the
//            instances that just began a step
//   sweeps : Arnoldi step of every active system, restart kernels on demand
//
// replayed by one CUDA graph WHILE node until every instance has finished.
#pragma once
#include "engine.cuh"

namespace sylv {

enum BatchStage : int { BST_INIT = 0, BST_INNER = 1, BST_SETUP = 2, BST_DONE = 3 };

struct BItem {
    int inst;     // instance
    int bi;       // block of that instance: A-side chunks first, then B side
};

// Outer-step kernel of a batch: gram(init) for new instances, gram(update)
// for instances whose 2r inner solves are all done; the instance's last
// block then finishes the step and starts the next one.
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_batch_outer(const AdiDev<T, S, C>* __restrict__ ds, const BItem* __restrict__ items, BatchCtl* ctl) {
    count_launch(ctl, K_GRAM);
    const BItem it = items[blockIdx.x];
    const AdiDev<T, S, C>& d = ds[it.inst];
    AdiState<T>* s = d.s;
    const int stage = s->stage;
    int init = 0;
    if (stage == BST_INIT) {
        init = 1;
    } else if (stage == BST_INNER) {
        // no sweep kernel runs concurrently: every block sees the same phases
        for (int q = 0; q < 2 * d.r; ++q)
            if (d.st[q].phase != PH_DONE) return;
    } else {
        return;
    }
    if (!adi_gram_body(d, init, it.bi)) return;
    if (s->done) {
        s->stage = BST_DONE;
        if (atomicSub(&ctl->n_inst_open, 1) == 1 && ctl->h_open) {
            *(volatile int*)ctl->h_open = 0;
            __threadfence_system();
        }
    } else {
        adi_begin_step(d);
        atomicAdd(&ctl->n_active, 2 * d.r);
        s->stage = BST_SETUP;
    }
}

// Set-up of the step an instance just began (Jacobi inverse, pre-scaled
// stencil diagonals, zeroed Z / Y slots); the last block hands the instance
// to the sweeps.
template <typename T, typename S, typename C>
__global__ void __launch_bounds__(SYLV_BLOCK)
k_batch_step(const AdiDev<T, S, C>* __restrict__ ds, const BItem* __restrict__ items, BatchCtl* ctl) {
    count_launch(ctl, K_STEP);
    const BItem it = items[blockIdx.x];
    const AdiDev<T, S, C>& d = ds[it.inst];
    AdiState<T>* s = d.s;
    if (s->stage != BST_SETUP) return;
    adi_step_rows(d, it.bi);
    if (!last_block(&s->counter, d.nchA + d.nchB)) return;
    if (threadIdx.x == 0) {
        s->counter = 0;
        s->stage = BST_INNER;
    }
}

// Device buffers of all instances carved from one allocation.
struct Arena {
    size_t bytes = 0;
    size_t take(size_t n) {
        const size_t off = bytes;
        bytes += (n + 255) / 256 * 256;
        return off;
    }
};

template <typename T, typename S, typename C>
struct Batch : BatchBase {
    Engine<T, S, C> eng;
    cudaStream_t stream = nullptr;
    int count = 0, kmax = 0, max_inner = 0, rpc = 0, nbitems = 0;
    std::vector<AdiDev<T, S, C>> hd;
    std::vector<int> inst_n, inst_m, inst_r;
    Dev<unsigned char> arena;
    Dev<AdiDev<T, S, C>> d_ds;
    Dev<BItem> d_items;
    Dev<AdiState<T>> st;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int h_one = 1, h_zero = 0;
    int solved = 0;
    std::vector<int> inst_status;
    long long launches_last = 0;

    TuneResult tune;                // chunk-size autotuner (opts.autotune)
    int driver = 0;                 // 0: one CUDA graph per solve; 1: host-driven device iterations
    int restart_every = 1;
    int* h_open = nullptr;          // mapped host word (host-driven solves)
    int* d_hopen = nullptr;
    cudaEvent_t bev[4][3] = {};     // events around the outer kernels of sampled iterations
    int bpend[4] = {0, 0, 0, 0};

    ~Batch() override {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (h_open) cudaFreeHost(h_open);
        for (auto& row : bev)
            for (auto& e : row)
                if (e) cudaEventDestroy(e);
    }

    int profile(int on) override {
        SYLV_TRY(eng.set_profile(on));
        for (int sl = 0; sl < 4; ++sl) bpend[sl] = 0;
        if (on && !bev[0][0])
            for (auto& row : bev)
                for (auto& e : row) SYLV_CK(cudaEventCreate(&e));
        return SYLV_OK;
    }

    int kernel_stats(double* ms, double* bytes, double* flops, long long* launches) const override {
        double b[K_COUNT], f[K_COUNT];
        SYLV_TRY(eng.read_work(b, f));
        for (int q = 0; q < K_COUNT; ++q) {
            if (ms) ms[q] = eng.samples[q] > 0 ? eng.kernel_ms[q] / eng.samples[q] * eng.launches[q] : 0.0;
            if (bytes) bytes[q] = b[q];
            if (flops) flops[q] = f[q];
            if (launches) launches[q] = eng.launches[q];
        }
        return SYLV_OK;
    }

    int harvest_outer(int slot) {
        if (!bpend[slot]) return SYLV_OK;
        SYLV_CK(cudaEventSynchronize(bev[slot][2]));
        float m0 = 0.f, m1 = 0.f;
        SYLV_CK(cudaEventElapsedTime(&m0, bev[slot][0], bev[slot][1]));
        SYLV_CK(cudaEventElapsedTime(&m1, bev[slot][1], bev[slot][2]));
        eng.kernel_ms[K_GRAM] += m0; eng.samples[K_GRAM] += 1;
        eng.kernel_ms[K_STEP] += m1; eng.samples[K_STEP] += 1;
        bpend[slot] = 0;
        return SYLV_OK;
    }

    // Host-driven solve: the host launches every device iteration (outer
    // kernel, step set-up, inner sweeps, restart kernels every restart_every
    // iterations) until the device clears *h_open (every instance finished),
    // with at most about eight iterations in flight; with profiling, the
    // kernels of every fourth iteration are bracketed by CUDA events.
    int solve_host() {
        SYLV_CK(cudaMemsetAsync(st.p, 0, (size_t)count * sizeof(AdiState<T>), stream));
        BatchCtl c{};
        SYLV_CK(cudaMemcpy(&c, eng.d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost));
        unsigned long long l0 = 0;
        for (int q = 0; q < K_COUNT; ++q) l0 += c.launch_count[q];
        c.n_active = 0; c.ticks = 0; c.capped = 0; c.n_inst_open = count; c.graph = 0;
        c.h_flag = nullptr;           // the inner-solve flag is not the end of a batch
        c.h_open = d_hopen;
        for (int q = 0; q < K_COUNT; ++q) c.gdone[q] = 0;
        SYLV_CK(cudaMemcpyAsync(eng.d_ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice, stream));
        SYLV_CK(cudaStreamSynchronize(stream));
        *h_open = 1;
        const long long max_ticks = (long long)(kmax + 2) * (max_inner + 8);
        const int D = 4, G = eng.pdl ? 4 : 1, DE = eng.pdl ? 2 : D;
        long long t = 0, grp = 0;
        int rc = SYLV_OK;
        while (*(volatile int*)h_open != 0) {
            if (t >= max_ticks) {
                set_error("batch: instances did not finish within %lld device iterations", max_ticks);
                rc = SYLV_ERR_INNER_STALL;
                break;
            }
            const int slot = (int)(t % D);
            if (eng.pending[slot]) SYLV_TRY(eng.harvest(slot));
            SYLV_TRY(harvest_outer(slot));
            const bool sampled = eng.profile && (eng.tick_no % eng.prof_every) == 0;
            if (sampled) SYLV_CK(cudaEventRecord(bev[slot][0], stream));
            k_batch_outer<T, S, C><<<nbitems, SYLV_BLOCK, 0, stream>>>(d_ds.p, d_items.p, eng.d_ctl.p);
            if (sampled) SYLV_CK(cudaEventRecord(bev[slot][1], stream));
            k_batch_step<T, S, C><<<nbitems, SYLV_BLOCK, 0, stream>>>(d_ds.p, d_items.p, eng.d_ctl.p);
            if (sampled) {
                SYLV_CK(cudaEventRecord(bev[slot][2], stream));
                bpend[slot] = 1;
            }
            SYLV_CK(cudaGetLastError());
            eng.launches[K_GRAM]++; eng.launches[K_STEP]++;
            SYLV_TRY(eng.launch_tick(0, slot, restart_every <= 1 || t % restart_every == 0));
            ++t;
            if (t % G == 0) {
                SYLV_CK(cudaEventRecord(eng.ev[grp % DE], stream));
                ++grp;
                if (grp >= DE) SYLV_CK(cudaEventSynchronize(eng.ev[grp % DE]));
            }
        }
        SYLV_CK(cudaStreamSynchronize(stream));
        for (int sl = 0; sl < D; ++sl) {
            if (eng.pending[sl]) SYLV_TRY(eng.harvest(sl));
            SYLV_TRY(harvest_outer(sl));
        }
        eng.ticks += t;
        SYLV_CK(cudaMemcpy(&c, eng.d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost));
        unsigned long long l1 = 0;
        for (int q = 0; q < K_COUNT; ++q) l1 += c.launch_count[q];
        launches_last = (long long)(l1 - l0);
        ticks_last = t;
        const int frc = finish();
        return rc != SYLV_OK ? rc : frc;
    }

    int tuning(int* chosen, int* cand, double* ms, int cap, int* count) const override {
        if (chosen) *chosen = rpc;
        const int nc = (int)tune.cand.size();
        for (int q = 0; q < nc && q < cap; ++q) {
            if (cand) cand[q] = tune.cand[q];
            if (ms) ms[q] = tune.ms[q];
        }
        if (count) *count = nc;
        return SYLV_OK;
    }

    int set_rhs(int i, const double* hf, const double* hg) override {
        if (!hf || !hg) { set_error("batch set_rhs: null f or g"); return SYLV_ERR_INVALID; }
        SYLV_CK(cudaMemcpyAsync((void*)hd[i].f, hf, (size_t)inst_n[i] * inst_r[i] * sizeof(double),
                                cudaMemcpyHostToDevice, stream));
        SYLV_CK(cudaMemcpyAsync((void*)hd[i].g, hg, (size_t)inst_m[i] * inst_r[i] * sizeof(double),
                                cudaMemcpyHostToDevice, stream));
        SYLV_CK(cudaStreamSynchronize(stream));
        return SYLV_OK;
    }

    int init(const std::vector<BatchProb>& ps, const sylv_opts& o, cudaStream_t s) {
        stream = s;
        count = (int)ps.size();
        kmax = o.kmax;
        max_inner = o.max_inner;
        std::vector<long long> rows, grows;
        for (const auto& p : ps) {
            for (int l = 0; l < p.r; ++l) { rows.push_back(p.n); rows.push_back(p.m); }
            grows.push_back(p.n);
            grows.push_back(p.m);
        }
        rpc = o.rows_per_chunk > 0 ? o.rows_per_chunk
              : o.inner == SYLV_INNER_BICGSTAB ? bicg_rows_per_chunk<T, S, C>(grows)
                                               : sweep_rows_per_chunk<T, S, C>(rows, o.ortho);
        if (o.autotune && o.rows_per_chunk <= 0) {
            // the systems of the batch with their operators; the Jacobi inverse
            // is left out of the probe and the stencil pointers only identify
            // the operators (the probe fills its own stencil values)
            std::vector<int> tn, to;
            std::vector<T*> tp;
            std::vector<C*> ta;
            std::vector<OpDesc> tops;
            for (int i = 0; i < (int)ps.size(); ++i) {
                const BatchProb& p = ps[i];
                tops.push_back(p.A->desc);
                tops.push_back(p.Bt->desc);
                for (int side = 0; side < 2; ++side)
                    for (int l = 0; l < p.r; ++l) {
                        tn.push_back(side ? p.m : p.n);
                        to.push_back(2 * i + side);
                        tp.push_back(nullptr);
                        const bool sc = scaled_op_possible(side ? p.Bt->desc : p.A->desc);
                        ta.push_back(sc ? reinterpret_cast<C*>((uintptr_t)(2 * i + side + 1) * 256) : nullptr);
                    }
            }
            SYLV_TRY((autotune_rpc<T, S, C>(tn, to, tops, tp, ta, o.restart, o.ortho, o.inner, s, &tune)));
            if (tune.chosen > 0) rpc = tune.chosen;
        }
        rpc = (rpc + 31) / 32 * 32;
        // the outer-step kernels (factor update, Grams, step set-up) touch each
        // row a few times per outer step: their work items are at least 4096
        // rows, whatever chunk the inner kernels take (fewer blocks, fewer
        // chunk partials in the Gram reductions)
        const int orpc = std::max(rpc, 4096);
        // ---- layout of every instance's buffers in one arena ----
        struct Off { size_t f, g, w, t, Z, Y, gam, hist, alpha, beta, pinvA, pinvB, avalA, avalB, gpart; };
        std::vector<Off> off(count);
        Arena ar;
        for (int i = 0; i < count; ++i) {
            const BatchProb& p = ps[i];
            const int nchA = (p.n + orpc - 1) / orpc, nchB = (p.m + orpc - 1) / orpc;
            Off& q = off[i];
            q.f = ar.take((size_t)p.n * p.r * sizeof(double));
            q.g = ar.take((size_t)p.m * p.r * sizeof(double));
            q.w = ar.take((size_t)p.n * p.r * sizeof(T));
            q.t = ar.take((size_t)p.m * p.r * sizeof(T));
            q.Z = ar.take((size_t)p.n * p.r * kmax * sizeof(T));
            q.Y = ar.take((size_t)p.m * p.r * kmax * sizeof(T));
            q.gam = ar.take((size_t)p.r * kmax * sizeof(T));
            q.hist = ar.take((size_t)kmax * SYLV_HIST_COLS * sizeof(double));
            q.alpha = ar.take((size_t)p.nshift * sizeof(T));
            q.beta = ar.take((size_t)p.nshift * sizeof(T));
            q.pinvA = o.jacobi ? ar.take((size_t)p.n * sizeof(T)) : (size_t)-1;
            q.pinvB = o.jacobi ? ar.take((size_t)p.m * sizeof(T)) : (size_t)-1;
            q.avalA = scaled_op_possible(p.A->desc) ? ar.take((size_t)p.A->desc.ndiag * p.n * sizeof(C)) : (size_t)-1;
            q.avalB = scaled_op_possible(p.Bt->desc) ? ar.take((size_t)p.Bt->desc.ndiag * p.m * sizeof(C)) : (size_t)-1;
            q.gpart = ar.take((size_t)(nchA + nchB) * SYLV_GSTRIDE * sizeof(T));
        }
        SYLV_TRY(arena.alloc(ar.bytes));
        SYLV_CK(cudaMemset(arena.p, 0, ar.bytes));
        unsigned char* base = arena.p;
        auto at = [&](size_t o_) { return o_ == (size_t)-1 ? nullptr : (void*)(base + o_); };
        // ---- the column systems of all instances: one engine ----
        std::vector<int> sn, so;
        std::vector<T*> pv;
        std::vector<C*> av;
        std::vector<OpDesc> ops;
        for (int i = 0; i < count; ++i) {
            const BatchProb& p = ps[i];
            ops.push_back(p.A->desc);
            ops.push_back(p.Bt->desc);
            for (int l = 0; l < p.r; ++l) {
                sn.push_back(p.n); so.push_back(2 * i);
                pv.push_back((T*)at(off[i].pinvA)); av.push_back((C*)at(off[i].avalA));
            }
            for (int l = 0; l < p.r; ++l) {
                sn.push_back(p.m); so.push_back(2 * i + 1);
                pv.push_back((T*)at(off[i].pinvB)); av.push_back((C*)at(off[i].avalB));
            }
        }
        eng.ortho = o.ortho;
        eng.inner = o.inner;
        eng.restart_every = o.restart_every;
        driver = o.driver;
        restart_every = o.restart_every;
        SYLV_TRY(eng.setup(sn, so, ops, pv, av, {}, 0, o.restart, rpc, stream));
        SYLV_CK(cudaHostAlloc((void**)&h_open, sizeof(int), cudaHostAllocMapped));
        *h_open = 0;
        SYLV_CK(cudaHostGetDevicePointer((void**)&d_hopen, h_open, 0));
        SYLV_TRY(st.alloc(count));
        SYLV_CK(cudaMemset(st.p, 0, (size_t)count * sizeof(AdiState<T>)));
        // ---- per-instance descriptors and the outer-kernel work list ----
        hd.resize(count);
        std::vector<BItem> items;
        int sbase = 0;
        for (int i = 0; i < count; ++i) {
            const BatchProb& p = ps[i];
            AdiDev<T, S, C>& d = hd[i];
            d = AdiDev<T, S, C>{};
            d.n = p.n; d.m = p.m; d.r = p.r; d.kmax = kmax; d.nshift = p.nshift;
            d.strategy = o.strategy; d.bl_clamp = o.bl_clamp; d.max_inner = max_inner;
            d.tau = p.tau; d.xi = o.xi;
            d.dminA = p.dminA; d.dminB = p.dminB; d.dmaxA = o.dmax_A; d.dmaxB = o.dmax_B;
            d.fixed_tol = p.fixed_tol;
            d.alpha = (const T*)at(off[i].alpha); d.beta = (const T*)at(off[i].beta);
            d.f = (const double*)at(off[i].f); d.g = (const double*)at(off[i].g);
            d.w = (T*)at(off[i].w); d.t = (T*)at(off[i].t);
            d.Z = (T*)at(off[i].Z); d.Y = (T*)at(off[i].Y); d.gam = (T*)at(off[i].gam);
            d.hist = (double*)at(off[i].hist);
            d.opA = p.A->desc; d.opB = p.Bt->desc;
            d.pinvA = (T*)at(off[i].pinvA); d.pinvB = (T*)at(off[i].pinvB);
            d.avalA = (C*)at(off[i].avalA); d.avalB = (C*)at(off[i].avalB);
            d.sd = eng.d_sd.p + sbase; d.st = eng.d_st.p + sbase; d.ctl = eng.d_ctl.p;
            d.gpart = (T*)at(off[i].gpart);
            d.nchA = (p.n + orpc - 1) / orpc; d.nchB = (p.m + orpc - 1) / orpc; d.rpc = orpc;
            d.s = st.p + i; d.h_done = nullptr;
            for (int b = 0; b < d.nchA + d.nchB; ++b) items.push_back({i, b});
            sbase += 2 * p.r;
            std::vector<T> ha(p.nshift), hb(p.nshift);
            for (int k = 0; k < p.nshift; ++k) {
                ha[k] = make_scalar<T>(p.alpha[k].re, p.alpha[k].im);
                hb[k] = make_scalar<T>(p.beta[k].re, p.beta[k].im);
            }
            SYLV_CK(cudaMemcpy((void*)d.alpha, ha.data(), p.nshift * sizeof(T), cudaMemcpyHostToDevice));
            SYLV_CK(cudaMemcpy((void*)d.beta, hb.data(), p.nshift * sizeof(T), cudaMemcpyHostToDevice));
            SYLV_CK(cudaMemcpy((void*)d.f, p.f, (size_t)p.n * p.r * sizeof(double), cudaMemcpyHostToDevice));
            SYLV_CK(cudaMemcpy((void*)d.g, p.g, (size_t)p.m * p.r * sizeof(double), cudaMemcpyHostToDevice));
            inst_n.push_back(p.n); inst_m.push_back(p.m); inst_r.push_back(p.r);
        }
        nbitems = (int)items.size();
        SYLV_TRY(d_ds.alloc(count));
        SYLV_TRY(d_items.alloc(items.size()));
        SYLV_CK(cudaMemcpy(d_ds.p, hd.data(), (size_t)count * sizeof(AdiDev<T, S, C>), cudaMemcpyHostToDevice));
        SYLV_CK(cudaMemcpy(d_items.p, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice));
        inst_status.assign(count, SYLV_ERR_NOT_SOLVED);
        return SYLV_OK;
    }

    int add_kernel(cudaGraphNode_t* node, cudaGraph_t g, cudaGraphNode_t* dep, void* func, int grid, void** args,
                   int smem = 0) {
        cudaKernelNodeParams kp = {};
        kp.func = func;
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(SYLV_BLOCK);
        kp.sharedMemBytes = smem;
        kp.kernelParams = args;
        SYLV_CK(cudaGraphAddKernelNode(node, g, dep, dep ? 1 : 0, &kp));
        return SYLV_OK;
    }

    // WHILE(h_loop) { IF(h_bouter) { outer -> step } -> spmv -> pass2 -> pass3 ->
    //                 IF(h_restart) { update -> residual } }
    // h_loop starts at 1 on each launch; afterwards only the grid-level
    // decisions of pass 3 / the restart residual keep it set (sweep 1 clears
    // it first), and they keep it while a system is active or an instance
    // has not finished.  h_bouter starts at 1 (every instance takes its
    // initial Grams); sweep 1 clears it and a system that finishes sets it,
    // so the outer-step kernels run only in the device iterations after one
    // did (an instance moves on only when all its systems are done).
    // If the device-updatable step-kernel nodes are refused at
    // instantiation, the graph is built again without them.
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
        cudaGraph_t g;
        SYLV_CK(cudaGraphCreate(&g, 0));
        graph = g;
        cudaGraphConditionalHandle h_loop, h_restart;
        SYLV_CK(cudaGraphConditionalHandleCreate(&h_loop, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams lp = {};
        lp.type = cudaGraphNodeTypeConditional;
        lp.conditional.handle = h_loop;
        lp.conditional.type = cudaGraphCondTypeWhile;
        lp.conditional.size = 1;
        cudaGraphNode_t n_loop;
        SYLV_CK(cudaGraphAddNode(&n_loop, g, nullptr, nullptr, 0, &lp));
        cudaGraph_t body = lp.conditional.phGraph_out[0];
        SYLV_CK(cudaGraphConditionalHandleCreate(&h_restart, body, 0, cudaGraphCondAssignDefault));
        cudaGraphConditionalHandle h_bouter;
        SYLV_CK(cudaGraphConditionalHandleCreate(&h_bouter, body, 1, cudaGraphCondAssignDefault));
        auto* dsp = d_ds.p;
        auto* bip = d_items.p;
        auto* sdp = eng.d_sd.p;
        auto* stp = eng.d_st.p;
        auto* opp = eng.d_ops.p;
        auto* itp = eng.d_items.p;
        auto* ctp = eng.d_ctl.p;
        int mode0 = 0;
        void* ao[] = {&dsp, &bip, &ctp};
        void* a1[] = {&sdp, &stp, &opp, &itp, &ctp, &mode0};
        void* a2[] = {&sdp, &stp, &itp, &ctp};
        int nsysb = eng.nsys;
        void* ab[] = {&sdp, &stp, &itp, &ctp, &nsysb};
        void* a3[] = {&sdp, &stp, &itp, &ctp, &mode0};
        void* a4[] = {&sdp, &stp, &itp, &ctp};
        void* a5[] = {&sdp, &stp, &opp, &itp, &ctp};
        const int ni = eng.nitems;
        cudaGraphNode_t n_o, n_s, n1, n2, n3, n_if, n4, n5, n_ob;
        cudaGraphNodeParams op = {};
        op.type = cudaGraphNodeTypeConditional;
        op.conditional.handle = h_bouter;
        op.conditional.type = cudaGraphCondTypeIf;
        op.conditional.size = 1;
        SYLV_CK(cudaGraphAddNode(&n_ob, body, nullptr, nullptr, 0, &op));
        cudaGraph_t ob_body = op.conditional.phGraph_out[0];
        SYLV_TRY(add_kernel(&n_o, ob_body, nullptr, (void*)k_batch_outer<T, S, C>, nbitems, ao));
        SYLV_TRY(add_kernel(&n_s, ob_body, &n_o, (void*)k_batch_step<T, S, C>, nbitems, ao));
        n_s = n_ob;               // the inner kernels follow the IF node
        const int sm = sweep_smem_bytes<S, C>();
        auto* grp = eng.d_groups.p;
        auto* gip = eng.d_gitems.p;
        int ngi = eng.ngitems;
        void* br[] = {&sdp, &stp, &opp, &grp, &gip, &ngi, &ctp};
        if (eng.inner == 1) {
            SYLV_TRY(eng.add_bicg_nodes(body, &n_s, &n3, try_dyn));
        } else if (eng.ortho == 1) {
            SYLV_TRY(add_kernel(&n1, body, &n_s, (void*)k_dcgs_a<T, S, C>, ni, a5, dcgs_a_smem_bytes<T, S, C>()));
            SYLV_TRY(add_kernel(&n3, body, &n1, (void*)k_dcgs_b<T, S, C>, ni + nsysb, ab, dcgs_b_smem_bytes<T, S, C>()));
        } else {
            SYLV_TRY(add_kernel(&n1, body, &n_s, (void*)k_arnoldi_spmv<T, S, C>, ni, a1, sm));
            SYLV_TRY(add_kernel(&n2, body, &n1, (void*)k_cgs_pass2<T, S, C>, ni, a2, sm));
            SYLV_TRY(add_kernel(&n3, body, &n2, (void*)k_cgs_pass3<T, S, C>, ni, a3, sm));
        }
        cudaGraphNodeParams ip = {};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = h_restart;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        SYLV_CK(cudaGraphAddNode(&n_if, body, &n3, nullptr, 1, &ip));
        cudaGraph_t if_body = ip.conditional.phGraph_out[0];
        const int rg = eng.restart_grid();
        if (eng.inner == 1) {
            SYLV_TRY(add_kernel(&n5, if_body, nullptr, (void*)k_bicg_resid<T, S, C>, rg, br));
        } else {
            SYLV_TRY(add_kernel(&n4, if_body, nullptr, (void*)k_restart_update<T, S, C>, rg, a4));
            SYLV_TRY(add_kernel(&n5, if_body, &n4, (void*)k_restart_residual<T, S, C>, rg, a5));
        }
        SYLV_CK(cudaGraphInstantiate(&gexec, g, 0));
        // kernels of the graph update nodes of the graph: upload it first
        if (eng.dyn_grid) SYLV_CK(cudaGraphUpload(gexec, stream));
        BatchCtl c{};
        SYLV_CK(cudaMemcpy(&c, eng.d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost));
        c.h_loop = h_loop;
        c.h_restart = h_restart;
        c.h_bouter = h_bouter;
        c.bouter = 1;
        c.nsys = eng.nsys;
        eng.set_dyn_fields(c);
        SYLV_CK(cudaMemcpy(eng.d_ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice));
        return SYLV_OK;
    }

    int solve() override {
        if (driver == 1 || eng.profile) return solve_host();
        if (!gexec) SYLV_TRY(build_graph());
        // fresh outer states; the control block's counters for this launch
        SYLV_CK(cudaMemsetAsync(st.p, 0, (size_t)count * sizeof(AdiState<T>), stream));
        BatchCtl c{};
        SYLV_CK(cudaMemcpy(&c, eng.d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost));
        unsigned long long l0 = 0;
        for (int q = 0; q < K_COUNT; ++q) l0 += c.launch_count[q];
        c.n_active = 0;
        c.ticks = 0;
        c.capped = 0;
        c.n_inst_open = count;
        c.max_ticks = (kmax + 2) * (max_inner + 8);
        for (int q = 0; q < K_COUNT; ++q) c.gdone[q] = 0;
        c.graph = 1;
        SYLV_CK(cudaMemcpyAsync(eng.d_ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice, stream));
        SYLV_CK(cudaStreamSynchronize(stream));     // c lives on this stack frame
        SYLV_CK(cudaGraphLaunch(gexec, stream));
        BatchCtl* dc = eng.d_ctl.p;
        SYLV_CK(cudaMemcpyAsync(&dc->graph, &h_zero, sizeof(int), cudaMemcpyHostToDevice, stream));
        SYLV_CK(cudaStreamSynchronize(stream));
        SYLV_CK(cudaMemcpy(&c, eng.d_ctl.p, sizeof(c), cudaMemcpyDeviceToHost));
        unsigned long long l1 = 0;
        for (int q = 0; q < K_COUNT; ++q) l1 += c.launch_count[q];
        launches_last = (long long)(l1 - l0);
        ticks_last = c.ticks;
        return finish();
    }

    // Per-instance status of the finished solve (SYLV_OK or the first failure).
    int finish() {
        SYLV_TRY(eng.take_stage_fault());
        std::vector<AdiState<T>> hs(count);
        SYLV_CK(cudaMemcpy(hs.data(), st.p, (size_t)count * sizeof(AdiState<T>), cudaMemcpyDeviceToHost));
        solved = 1;
        int first_bad = -1;
        for (int i = 0; i < count; ++i) {
            const AdiState<T>& s = hs[i];
            int rc;
            if (s.status == 2) rc = SYLV_ERR_NONFINITE;
            else if (s.stage != BST_DONE) rc = SYLV_ERR_INNER_STALL;   // stopped by the iteration cap
            else if (s.status == 1) rc = SYLV_ERR_MAXIT;
            else if (s.stalled > 0) rc = SYLV_ERR_INNER_STALL;
            else rc = SYLV_OK;
            inst_status[i] = rc;
            if (rc != SYLV_OK && first_bad < 0) first_bad = i;
        }
        if (first_bad >= 0) {
            set_error("batch instance %d: status %d (info() per instance)", first_bad, inst_status[first_bad]);
            return inst_status[first_bad];
        }
        return SYLV_OK;
    }
    long long ticks_last = 0;

    int state(int i, AdiState<T>* s) const {
        SYLV_CK(cudaMemcpy(s, st.p + i, sizeof(*s), cudaMemcpyDeviceToHost));
        return SYLV_OK;
    }

    int info(int i, sylv_info* out) const override {
        AdiState<T> s;
        SYLV_TRY(state(i, &s));
        std::memset(out, 0, sizeof(*out));
        out->status = inst_status[i];
        out->steps = solved ? s.k - 1 : 0;
        if (out->steps < 0) out->steps = 0;
        out->kr = out->steps * inst_r[i];
        out->is_complex = sizeof(T) == sizeof(cplx);
        out->rel_res_comp = s.nfg > 0 ? s.res / s.nfg : 0.0;
        out->norm_fg = s.nfg;
        out->inner_its_A = s.itsA;
        out->inner_its_B = s.itsB;
        out->inner_restarts = s.cycles;
        out->stalled_solves = s.stalled;
        out->ticks = (int32_t)ticks_last;
        out->launches = launches_last;
        return SYLV_OK;
    }

    int history(int i, double* buf, int cap, int* rows) const override {
        AdiState<T> s;
        SYLV_TRY(state(i, &s));
        const int nrow = solved ? std::max(0, std::min(cap, s.k - 1)) : 0;
        if (nrow > 0)
            SYLV_CK(cudaMemcpy(buf, hd[i].hist, (size_t)nrow * SYLV_HIST_COLS * sizeof(double), cudaMemcpyDeviceToHost));
        if (rows) *rows = nrow;
        return SYLV_OK;
    }

    int factors(int i, void* Zo, void* Yo, void* go, int on_device, int* kr) const override {
        AdiState<T> s;
        SYLV_TRY(state(i, &s));
        const int steps = solved ? std::max(0, s.k - 1) : 0;
        const size_t ncol = (size_t)steps * inst_r[i];
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (Zo && ncol) SYLV_CK(cudaMemcpy(Zo, hd[i].Z, ncol * inst_n[i] * sizeof(T), kind));
        if (Yo && ncol) SYLV_CK(cudaMemcpy(Yo, hd[i].Y, ncol * inst_m[i] * sizeof(T), kind));
        if (go && ncol) SYLV_CK(cudaMemcpy(go, hd[i].gam, ncol * sizeof(T), kind));
        if (kr) *kr = (int)ncol;
        return SYLV_OK;
    }

    int stats(long long* launches, double* bytes, double* flops, long long* ticks) const override {
        double b[K_COUNT], f[K_COUNT];
        SYLV_TRY(eng.read_work(b, f));
        double bs = 0.0, fs = 0.0;
        for (int q = 0; q < K_COUNT; ++q) { bs += b[q]; fs += f[q]; }
        if (launches) *launches = launches_last;
        if (bytes) *bytes = bs;
        if (flops) *flops = fs;
        if (ticks) *ticks = ticks_last;
        return SYLV_OK;
    }
};

template <typename T, typename S, typename C>
int make_batch_t(const std::vector<BatchProb>& ps, const sylv_opts& o, cudaStream_t s, BatchBase** out) {
    Batch<T, S, C>* p = new (std::nothrow) Batch<T, S, C>();
    if (!p) { set_error("host allocation failed"); return SYLV_ERR_NOMEM; }
    int rc = p->init(ps, o, s);
    if (rc != SYLV_OK) { delete p; return rc; }
    *out = p;
    return SYLV_OK;
}

}  // namespace sylv
