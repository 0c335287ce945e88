#!/usr/bin/env python
"""Time to relative residual 1e-8 of the inexact LR-ADI Sylvester solver on GB300.

Headline workload (default ``--workload batch64``): 64 independent 2D
Sylvester instances A_i X + X B_i = -f_i g_i^* solved together by the batched
solver - N_A, N_B ~ U{64..256} (n, m from 4096 to 65536), r ~ U{1, 2, 4},
convection magnitudes ~ U[0, 50], 10 real shift pairs each, "mid" inner
tolerances without back-looking, tau = 1e-8 - with BiCGstab inner solves in
mixed precision (float32 vectors and products, float64 solutions, restart
residuals and outer iteration) and one CUDA graph per solve.  One step = one
solve of all 64 instances.  The working set (about 1 GB) exceeds the 129 MB
L2, so the kernels' GB/s are HBM figures.

The line also carries the comparisons the benchmark asks for - the plain
float64 method, float64 with a fixed inner tolerance of 1e-12 (standing in
for exact solves), GMRES inner solves - on the batch and on the single 2D
workload (A: N = 512, B: N = 400, r = 2).  ``--workload mid2d|mid3d|large3d``
times a single instance instead.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-rel.residual 1e-8 (s) and SpMM/orthog HBM GB/s, mixed+batched vs FP64"
UNIT = "s"
L2_FLUSH_BYTES = 512 << 20
BATCH_COUNT = 64
# instances of the batch that the CPU oracle solves in full for its baseline
# (smallest first; the reference arm's step is the first of them)
CPU_SAMPLE = (32, 4, 28, 0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch64",
                    help="batch64 (64 instances, the headline), or one instance: mid2d, mid3d, large3d, small2d")
    ap.add_argument("--strategy", default="nobl_mid")
    ap.add_argument("--inner", default="bicgstab", choices=["gmres", "bicgstab"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"],
                    help="fp32: float32 inner vectors/basis, float64 outer iteration")
    ap.add_argument("--ortho", default="dcgs2", choices=["cgs2", "dcgs2"], help="GMRES orthogonalisation")
    ap.add_argument("--real-pairs", type=int, default=1, help="real double steps for complex shift pairs")
    ap.add_argument("--kmax", type=int, default=50, help="outer step cap (small values give short profiler cases)")
    ap.add_argument("--rows-per-chunk", type=int, default=0,
                    help="fixed rows per work item (0: autotuned; a fixed value gives profiler runs without the probe)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--clock-log", default=os.path.join(tempfile.gettempdir(), "sylv_clocks_rank{rank}.csv"),
                    help="where the nvidia-smi clock samples of the timed region are written")
    ap.add_argument("--gen-workers", type=int, default=min(16, os.cpu_count() or 1),
                    help="processes generating the batch instances")
    return ap.parse_args()


def max_over_ranks(value: float, device: str = "cuda") -> float:
    """The job's time: the largest per-rank value over the default process
    group (replicas; no data-path collective exists in the solver)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str):
        self.gpu = gpu_index
        self.proc = None
        self.path = path

    def start(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s, p in zip(sm, power) if p > 0.3 * max(power)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power)}


# ------------------------------------------------------------ CPU baseline
# The oracle (plain numpy / scipy float64, test infrastructure) runs in a
# fresh interpreter with one BLAS thread; its output is only timed.

def _oracle_script(body: str) -> str:
    return f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
from paper_2312_02891_gb300 import workloads as W
from oracle.lradi import lradi
{body}
"""


def run_oracle(body: str) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-c", _oracle_script(body)], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        raise RuntimeError(p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def oracle_batch_instances(indices, strategy, inner) -> dict:
    """Full oracle solves of the given batch instances: per instance the
    seconds of the solve (generation excluded), its rows x rank and its outer
    steps."""
    return run_oracle(f"""
out = {{}}
for i in {list(indices)!r}:
    p = W.batch_problems(1, base_seed=1000 + i)[0]
    t = time.perf_counter()
    r = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy={strategy!r}, jacobi=True, inner={inner!r})
    out[i] = [time.perf_counter() - t, (p.A.n + p.B.n) * p.r, r.steps, bool(r.converged)]
print(json.dumps(out))
""")


def oracle_single(workload, strategy, inner) -> dict:
    return run_oracle(f"""
p = W.problem_config({workload!r})
t = time.perf_counter()
r = lradi(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, strategy={strategy!r},
          jacobi=bool(p.opts.get('jacobi', False)), inner={inner!r})
print(json.dumps({{"s": time.perf_counter() - t, "steps": r.steps, "converged": bool(r.converged)}}))
""")


def batch_rows(probs) -> int:
    return sum((p.A.n + p.B.n) * p.r for p in probs)


def cpu_baseline_batch(probs, strategy, inner) -> dict:
    """Full oracle solves of four batch instances (about 10 s on one core),
    scaled to the 64-instance batch by rows x rank; one full oracle solve of
    the smallest 2D workload (n = 1024, m = 900) as a measured anchor."""
    res = oracle_batch_instances(CPU_SAMPLE, strategy, inner)
    ts = sum(v[0] for v in res.values())
    rs = sum(v[1] for v in res.values())
    est = ts * batch_rows(probs) / rs
    anchor = oracle_single("small2d", strategy, "gmres")
    return {"value": est, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"full oracle solves ({inner} inner, float64, one thread) of batch instances "
                       f"{list(CPU_SAMPLE)}: {ts:.1f} s for {rs} rows x rank, scaled by rows x rank to the "
                       f"{batch_rows(probs)} of the batch"),
            "instances": {str(k): {"s": round(v[0], 3), "rows_x_r": v[1], "steps": v[2]} for k, v in res.items()},
            "anchor_small2d_full_solve_s": round(anchor["s"], 3)}


# ------------------------------------------------------------------- main

def run_reference(a):
    """The oracle as it stands, one core, on the benchmark workload: each step
    is one full solve of the smallest instance of the batch (a bounded
    sample), timed as it runs; the scaled estimate of the whole batch is
    reported beside it."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if a.workload != "batch64":
        steps = []
        for s in range(a.warmup + a.steps):
            r = oracle_single(a.workload, a.strategy, a.inner)
            if s >= a.warmup:
                steps.append(r["s"])
        v = statistics.mean(steps)
        sample = f"full oracle solve of {a.workload} ({a.inner} inner, float64, one thread)"
        extra = {}
    else:
        i0 = CPU_SAMPLE[0]
        steps, rows0 = [], None
        for s in range(a.warmup + a.steps):
            res = oracle_batch_instances([i0], a.strategy, a.inner)
            t, rows0 = res[str(i0)][0], res[str(i0)][1]
            if s >= a.warmup:
                steps.append(t)
        v = statistics.mean(steps)
        total = sum((p.A.n + p.B.n) * p.r for p in [_instance_sizes(i) for i in range(BATCH_COUNT)])
        sample = (f"full oracle solve ({a.inner} inner, float64, one thread) of batch instance {i0} "
                  f"({rows0} rows x rank) per step")
        extra = {"extrapolated_batch64_s": v * total / rows0,
                 "extrapolation": f"per step time x {total} / {rows0} (rows x rank of the batch / of the sample)"}
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": a.workload, "strategy": a.strategy, "inner": a.inner},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": v, "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    line.update(extra)
    print(json.dumps(line), flush=True)
    return 0


class _Sizes:
    def __init__(self, n, m, r):
        self.A, self.B, self.r = type("O", (), {"n": n})(), type("O", (), {"n": m})(), r


def _instance_sizes(i: int):
    """Sizes of batch instance i without building it (the seeded size draw of
    workloads.batch_problems)."""
    from paper_2312_02891_gb300 import workloads as W
    u = W._uniform53(1000 + i, 9, 0, 0, 5)
    NA = 64 + int(u[0] * 193)
    NB = 64 + int(u[1] * 193)
    return _Sizes(NA * NA, NB * NB, (1, 2, 4)[int(u[2] * 3)])


FP64_NOMINAL_TFLOPS = 1.25   # GB300 float64 rate (nominal, dense)
KNAMES = {
    "bicgstab": {"arnoldi_spmv": "k_bicg_a (p update + product + rhat^* v)",
                 "cgs_pass2": "k_bicg_b (product + t^* s, t^* t, s^* s)",
                 "cgs_pass3": "k_bicg_c (x, r, q updates + rhat^* r, r^* r)",
                 "restart_residual": "k_bicg_resid (float64 true residual)",
                 "restart_update": "k_bicg_list (work list of the iteration)"},
    "dcgs2": {"arnoldi_spmv": "k_dcgs_a (product + all dots)", "cgs_pass3": "k_dcgs_b (basis update)"},
    "cgs2": {},
}
INNER_KERNELS = ("arnoldi_spmv", "cgs_pass2", "cgs_pass3")
# DRAM traffic / algorithmic bytes of a kernel from one ncu capture of the
# current kernels, keyed by (workload, precision, inner solver, kernel); a
# kernel changed after its capture, or another workload or precision, has no
# entry (traffic null).  BiCGstab:
# one launch of each step kernel with every column system of the batched
# workload active (dram__bytes_read.sum + dram__bytes_write.sum over the
# kernel's own byte model), profiles/bicgstab_batch64_fp32.md.
NCU_TRAFFIC_RATIO = {
    ("batch64", "fp32", "bicgstab", "arnoldi_spmv"): (172.304640 + 45.247232) / 239.5,    # k_bicg_a
    ("batch64", "fp32", "bicgstab", "cgs_pass2"): (138.174464 + 19.597824) / 171.5,       # k_bicg_b
    ("batch64", "fp32", "bicgstab", "cgs_pass3"): (266.494464 + 93.886464) / 402.2,       # k_bicg_c
}


def kernel_table(stats, names):
    total_ms = sum(v[0] for v in stats.values())
    return {names.get(k, k): {"ms": round(v[0], 3), "share": round(v[0] / total_ms, 4) if total_ms else None,
                              "launches": v[3],
                              "GBps": round(v[1] / (v[0] * 1e-3) / 1e9, 1) if v[0] > 0 else None,
                              "TFLOPs": round(v[2] / (v[0] * 1e-3) / 1e12, 4) if v[0] > 0 else None}
            for k, v in stats.items() if v[3] > 0}


def roofline_of(stats, names, hbm, hbm_src, inner, workload, precision):
    dom = max(INNER_KERNELS, key=lambda k: stats[k][0])
    ms, by, fl, la = stats[dom]
    ach = (by / la) / ((ms / la) * 1e-3) / 1e9 if ms > 0 else None
    ratio = NCU_TRAFFIC_RATIO.get((workload, precision, inner, dom))
    inner_ms = sum(stats[k][0] for k in INNER_KERNELS + ("restart_update", "restart_residual"))
    inner_by = sum(stats[k][1] for k in INNER_KERNELS + ("restart_update", "restart_residual"))
    return {"bound": "hbm", "kernel": names.get(dom, dom), "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": (ach / hbm) if ach else None, "peak_source": hbm_src,
            "traffic": (ratio * by / la) if ratio else None,
            "algorithmic_bytes_per_launch": by / la if la else None,
            "inner_kernels_GBps": inner_by / (inner_ms * 1e-3) / 1e9 if inner_ms else None,
            "inner_kernels_frac": (inner_by / (inner_ms * 1e-3) / 1e9 / hbm) if inner_ms else None}


def run_ours(a):
    import ctypes as C

    import numpy as np

    from paper_2312_02891_gb300 import workloads as W

    ws, rank, local = dist_env()
    batch = a.workload == "batch64"
    # the batch instances are generated in spawned processes before the first
    # GPU call (a process forked after it could hang)
    probs = W.batch_problems(BATCH_COUNT, workers=a.gen_workers) if (batch or not a.no_variants) else []
    p2d = W.problem_config("mid2d") if (not batch or not a.no_variants) else None
    single = None if batch else (p2d if a.workload == "mid2d" else W.problem_config(a.workload))

    import torch
    import paper_2312_02891_gb300 as P

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    def timed(solver, warmup, steps):
        """Mean device seconds per solve (CUDA events on the solver stream),
        L2 flushed before every timed solve."""
        for _ in range(warmup):
            solver.solve()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        st = 0
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[k][0].record(stream)
            st = solver.solve()
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        barrier()
        t = sum(s.elapsed_time(e) for s, e in ev) / 1e3 / steps
        return max_over_ranks(t, "cuda"), st

    def make_batch(**kw):
        o = dict(strategy=a.strategy, precision=a.precision, jacobi=1, restart=30, inner=a.inner,
                 ortho="cgs2" if a.inner == "bicgstab" else a.ortho, kmax=a.kmax,
                 autotune=0 if a.rows_per_chunk else 1, rows_per_chunk=a.rows_per_chunk)
        o.update(kw)
        return P.SylvesterADIBatch(probs, stream=stream, **o)

    def make_single(p, **kw):
        o = dict(strategy=a.strategy, precision=a.precision, jacobi=int(p.opts.get("jacobi", False)),
                 restart=p.opts.get("restart", 30), inner=a.inner, ortho=a.ortho, kmax=a.kmax,
                 autotune=0 if a.rows_per_chunk else 1, rows_per_chunk=a.rows_per_chunk)
        if np.iscomplexobj(p.alpha) or np.iscomplexobj(p.beta):
            o["real_pairs"] = a.real_pairs
        o.update(kw)
        return P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, stream=stream, **o)

    def batch_summary(bt, t, st, nsolve):
        infos = [bt.info(i) for i in range(len(probs))]
        bs = bt.stats()
        return {"s": t, "instances_per_s": len(probs) / t, "status": st,
                "converged": sum(1 for q, i_ in zip(probs, infos) if i_["status"] == 0 and i_["rel_res_comp"] < q.tau),
                "outer_steps_total": sum(i_["steps"] for i_ in infos),
                "inner_its_total": sum(i_["inner_its_A"] + i_["inner_its_B"] for i_ in infos),
                "ticks_per_solve": bs["ticks"], "launches_per_solve": bs["launches"],
                "algorithmic_GBps": bs["bytes"] / nsolve / t / 1e9}, infos

    def single_summary(sv, t, st):
        info = sv.info()
        return {"s": t, "status": st, "outer_steps": info["steps"], "inner_its_A": info["inner_its_A"],
                "inner_its_B": info["inner_its_B"], "rel_res_comp": info["rel_res_comp"],
                "launches_per_solve": info["launches"]}, info

    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as fh_:
            peaks = json.load(fh_)
    hbm = peaks.get("hbm_gbs")
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs, copy kernel)" if hbm else "fallback 6800 GB/s"
    hbm = hbm or 6800.0
    names = KNAMES["bicgstab" if a.inner == "bicgstab" else a.ortho]
    sampler = ClockSampler(local, a.clock_log.format(rank=rank))

    # ---------------- headline ----------------
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    if batch:
        head = make_batch()
        n_items = len(probs)
    else:
        head = make_single(single)
        n_items = 1
    torch.cuda.synchronize()
    footprint = free0 - torch.cuda.mem_get_info()[0]
    tuning = head.tuning()
    sampler.start()
    time.sleep(0.3)
    nsolve0 = a.warmup + a.steps
    t_solve, st = timed(head, a.warmup, a.steps)
    clocks = sampler.stop()
    if batch:
        main_sum, infos = batch_summary(head, t_solve, st, nsolve0)
        launches = main_sum["launches_per_solve"]
    else:
        main_sum, info = single_summary(head, t_solve, st)
        launches = info["launches"]

    # per-kernel CUDA events: one more solve, host-driven, every fourth
    # device iteration's kernels bracketed by events
    if batch:
        prof = make_batch(driver=1)
    else:
        prof = make_single(single, driver=1)
    prof.solve()
    prof.profile(True)
    prof.solve()
    stats = prof.kernel_stats()
    prof.profile(False)
    prof.close()
    roof = roofline_of(stats, names, hbm, hbm_src, a.inner, a.workload, a.precision)

    # ---------------- end to end through the public API, host buffers ----------------
    e2e_steps = max(1, min(a.steps, 3))
    if batch:
        fh = [torch.from_numpy(np.asfortranarray(q.f)).pin_memory() for q in probs]
        gh = [torch.from_numpy(np.asfortranarray(q.g)).pin_memory() for q in probs]
        outs = []
        for q, i_ in zip(probs, infos):
            kr = i_["kr"]
            outs.append((torch.empty((kr, q.A.n), dtype=torch.float64).pin_memory(),
                         torch.empty((kr, q.B.n), dtype=torch.float64).pin_memory(),
                         torch.empty(kr, dtype=torch.float64).pin_memory()))
        h2d = sum(f.numel() + g.numel() for f, g in zip(fh, gh)) * 8
        d2h = sum(z.numel() + y.numel() + g.numel() for z, y, g in outs) * 8
        lib = P.load()
        e2e = []
        for _ in range(e2e_steps):
            flush.zero_()
            barrier()
            t0 = time.perf_counter()
            for i in range(len(probs)):
                P.sylv_adi_batch_set_rhs(head.h, i, fh[i].numpy(), gh[i].numpy())
            head.solve()
            kro, isc = C.c_int32(), C.c_int32()
            for i, (z, y, g) in enumerate(outs):
                lib.sylv_adi_batch_factors(head.h, i, z.data_ptr(), y.data_ptr(), g.data_ptr(), 0,
                                           C.byref(kro), C.byref(isc))
            e2e.append(time.perf_counter() - t0)
    else:
        fh = torch.from_numpy(np.asfortranarray(single.f)).pin_memory()
        gh = torch.from_numpy(np.asfortranarray(single.g)).pin_memory()
        kr = info["kr"]
        real = info["is_complex"] == 0
        fdt = torch.float64 if real else torch.complex128
        Zh = torch.empty((kr, single.A.n), dtype=fdt).pin_memory()
        Yh = torch.empty((kr, single.B.n), dtype=fdt).pin_memory()
        gmh = torch.empty(kr, dtype=fdt).pin_memory()
        h2d = (single.A.n + single.B.n) * single.r * 8
        d2h = (Zh.numel() + Yh.numel() + gmh.numel()) * Zh.element_size()
        e2e = []
        for _ in range(e2e_steps):
            flush.zero_()
            barrier()
            t0 = time.perf_counter()
            P.sylv_adi_set_rhs(head.h, fh.numpy(), gh.numpy())
            head.solve()
            kro, isc = C.c_int32(), C.c_int32()
            P.load().sylv_adi_factors(head.h, Zh.data_ptr(), Yh.data_ptr(),
                                      None if head.opts.real_pairs else gmh.data_ptr(), 0, C.byref(kro),
                                      C.byref(isc))
            e2e.append(time.perf_counter() - t0)
    barrier()
    e2e_v = max_over_ranks(sum(e2e) / len(e2e), "cuda")
    head.close()

    # ---------------- comparisons ----------------
    variants = {}
    if not a.no_variants:
        if probs:
            for name, kw, w_, k_ in (
                    ("batch64_fp64", dict(precision="fp64"), 1, 1),
                    ("batch64_fp64_fixed_1e-12", dict(precision="fp64", strategy="fixed", fixed_tol=1e-12), 0, 1),
                    ("batch64_fp32_gmres_cgs2", dict(inner="gmres", ortho="cgs2"), 1, 1),
                    ("batch64_fp32_gmres_dcgs2", dict(inner="gmres", ortho="dcgs2"), 0, 1)):
                with make_batch(**kw) as bt:
                    tv, stv = timed(bt, w_, k_)
                    variants[name], _ = batch_summary(bt, tv, stv, w_ + k_)
            if batch:
                f = variants["batch64_fp64_fixed_1e-12"]["s"]
                variants["speedup_vs_fp64_fixed_1e-12"] = f / t_solve
                variants["speedup_vs_fp64_adaptive"] = variants["batch64_fp64"]["s"] / t_solve
                variants["speedup_vs_fp32_gmres_cgs2"] = variants["batch64_fp32_gmres_cgs2"]["s"] / t_solve
        if p2d is not None:
            for name, kw, w_, k_ in (
                    ("mid2d_fp32_bicgstab", dict(inner="bicgstab"), 1, 2),
                    ("mid2d_fp64_bicgstab", dict(inner="bicgstab", precision="fp64"), 1, 1),
                    ("mid2d_fp32_gmres_dcgs2", dict(inner="gmres", ortho="dcgs2", driver=1), 1, 2),
                    ("mid2d_fp64_gmres_dcgs2", dict(inner="gmres", ortho="dcgs2", precision="fp64"), 1, 1),
                    ("mid2d_fp64_fixed_1e-12", dict(inner="gmres", ortho="dcgs2", precision="fp64",
                                                    strategy="fixed", fixed_tol=1e-12), 0, 1)):
                with make_single(p2d, **kw) as sv:
                    tv, stv = timed(sv, w_, k_)
                    variants[name], _ = single_summary(sv, tv, stv)
            variants["mid2d_note"] = ("2D workload, one instance (A: N = 512, B: N = 400, r = 2): its working "
                                      "set stays in L2, so its kernel rates are not HBM figures")

    line = {
        "metric": METRIC, "value": t_solve, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("f32 inner vectors + f64 outer" if a.precision == "fp32" else a.precision),
        "data": "synthetic",
        "config": ({"workload": "batch64", "instances": len(probs), "n_range": [min(q.A.n for q in probs),
                                                                               max(q.A.n for q in probs)],
                    "m_range": [min(q.B.n for q in probs), max(q.B.n for q in probs)],
                    "r": sorted({q.r for q in probs}), "rows_x_r": batch_rows(probs)}
                   if batch else {"workload": a.workload, "n": single.A.n, "m": single.B.n, "r": single.r}),
        "roofline": roof,
        "autotune": {"rows_per_chunk": tuning["rows_per_chunk"],
                     "ms_per_device_iteration": {str(k): round(v, 4) for k, v in tuning["candidates"].items()}},
        "kernels": kernel_table(stats, names),
        "variants": variants,
        "gpu_launches": int(launches) * a.steps,
        "clocks": clocks,
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "steps": e2e_steps},
    }
    line["config"].update({"inner": a.inner, "precision": a.precision, "strategy": a.strategy, "tau": 1e-8,
                           "kmax": a.kmax, "driver": "graph (one CUDA graph per solve)" if batch else "host",
                           "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "flushed (512 MiB write) before every timed solve",
                           "device_bytes_of_solver": footprint})
    line["config"].update({k: v for k, v in main_sum.items() if k not in ("s",)})
    if rank == 0 and ws == 1 and not a.no_cpu_baseline and batch:
        line["cpu_baseline"] = cpu_baseline_batch(probs, a.strategy, a.inner)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
