#!/usr/bin/env python
"""Time to relative residual 1e-8 of the inexact LR-ADI Sylvester solver on GB300.

One step = one full solve of Algorithm 1 (all inner shifted GMRES solves,
factor updates, Gram residual norms, device controller) on the mid-size 2D
convection-diffusion workload: A from N=512 (n = 262144, omega = 50 (x, y)),
B from N=400 (m = 160000, omega = 20 (y, -x)), r = 2, 12 real shift pairs,
right-Jacobi GMRES(30), "mid" tolerances without back-looking, tau = 1e-8,
mixed precision (float32 Krylov basis and sweeps, float64 restart residuals,
least squares, factors and outer iteration).  The line also carries the
plain float64 run, the float64 run with a fixed inner tolerance of 1e-12,
the bfloat16-basis run, the graph-driven runs and the batched workload (64
independent instances in one device loop).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-rel.residual 1e-8 (s) and SpMM/orthog HBM GB/s, mixed+batched vs FP64"
UNIT = "s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mid2d")
    ap.add_argument("--strategy", default="nobl_mid")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload among the variants")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"],
                    help="precision of the headline solve (the benchmark line uses fp32: float32 "
                         "Krylov basis and sweeps, float64 outer iteration)")
    ap.add_argument("--ortho", default="dcgs2", choices=["cgs2", "dcgs2"],
                    help="Arnoldi orthogonalisation of the inner GMRES (all runs of the line)")
    ap.add_argument("--inner", default="gmres", choices=["gmres", "bicgstab"],
                    help="inner solver of the headline solve")
    ap.add_argument("--kmax", type=int, default=50,
                    help="outer step cap (a small value gives a short case for profilers)")
    ap.add_argument("--cpu-sample-its", type=int, default=60)
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

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
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

def cpu_sample(workload: str, its: int, threads: int = 1):
    """Oracle GMRES on the first outer step's A and B systems, `its` Arnoldi
    steps each (whole restart cycles), timed on this host; run in a fresh
    interpreter with `threads` BLAS / OpenMP threads (the sparse products of
    the oracle are single-threaded; its dense basis operations use them)."""
    code = f"""
import json, time, numpy as np, sys
sys.path.insert(0, {ROOT!r})
from paper_2312_02891_gb300 import workloads as W
from oracle.gmres import gmres
p = W.problem_config({workload!r})
S = p.A.to_scipy(); Bt = p.B.to_scipy().T.tocsr()
jac = bool(p.opts.get('jacobi', False)); m = p.opts.get('restart', 30)
out = {{}}
for side, M, sig, b in (('A', S, p.beta[0], p.f[:, 0]), ('B', Bt, np.conj(p.alpha[0]), p.g[:, 0])):
    t = time.perf_counter()
    r = gmres(M, sig, b, 1e-300, m, {its}, jac, 'cgs2')
    out[side] = (time.perf_counter() - t) / r.iters
print(json.dumps(out))
"""
    nt = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=nt, OPENBLAS_NUM_THREADS=nt, MKL_NUM_THREADS=nt)
    t0 = time.perf_counter()
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        raise RuntimeError(p.stderr)
    per_it = json.loads(p.stdout.strip().splitlines()[-1])
    return per_it, time.perf_counter() - t0


def golden(workload: str, strategy: str):
    path = os.path.join(ROOT, "tests", "golden", f"{workload}_{strategy}.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return None


def cpu_baseline(workload, strategy, its, gpu_info=None, threads: int = 1):
    per_it, wall = cpu_sample(workload, its, threads)
    g = golden(workload, strategy)
    if g is not None:
        itsA, itsB, src = g["inner_its_A"], g["inner_its_B"], "stored oracle run"
    else:
        itsA, itsB, src = gpu_info["inner_its_A"], gpu_info["inner_its_B"], "this GPU run"
    est = itsA * per_it["A"] + itsB * per_it["B"]
    return {"value": est, "unit": UNIT, "cores": int(threads), "kind": "oracle",
            "sample": (f"oracle GMRES(30) on step-1 A and B systems, {its} Arnoldi steps each, "
                       f"{per_it['A'] * 1e3:.2f} / {per_it['B'] * 1e3:.2f} ms per step (A/B), "
                       f"scaled by the inner-step totals of the {src} "
                       f"({itsA} A + {itsB} B); sample wall {wall:.1f} s")}


# ------------------------------------------------------------------- main

def run_reference(a):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    vals = []
    for s in range(a.warmup + a.steps):
        cb = cpu_baseline(a.workload, a.strategy, a.cpu_sample_its)
        if s >= a.warmup:
            vals.append(cb["value"])
    v = statistics.mean(vals)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": a.workload, "strategy": a.strategy},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": cb["sample"], "value": v,
                             "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


FP64_NOMINAL_TFLOPS = 1.25   # GB300 float64 rate (nominal, dense)
SWEEPS = ("arnoldi_spmv", "cgs_pass2", "cgs_pass3")
# with the delayed CGS2 the first and third counters hold its two kernels
DCGS2_NAMES = {"arnoldi_spmv": "k_dcgs_a (product + all dots)", "cgs_pass3": "k_dcgs_b (basis update)"}
# DRAM traffic / algorithmic bytes of the sweep kernels from one ncu capture
# of the current kernels (None once a kernel changes after its capture)
NCU_TRAFFIC_RATIO = {}


def run_ours(a):
    import ctypes as C

    import numpy as np
    import torch

    import paper_2312_02891_gb300 as P
    from paper_2312_02891_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    p = W.problem_config(a.workload)
    # the 64 batched instances are generated on a host thread meanwhile
    # (shift selection runs sparse LU solves; the solver calls release the GIL)
    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(max_workers=1)
    batch_future = None if (a.no_variants or a.no_batch) else pool.submit(W.batch_problems, 64)
    stream = torch.cuda.Stream()
    jac = int(p.opts.get("jacobi", False))
    rst = p.opts.get("restart", 30)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    n, m, r = p.A.n, p.B.n, p.r

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    def make(**kw):
        kw.setdefault("kmax", a.kmax)
        kw.setdefault("ortho", a.ortho)
        kw.setdefault("inner", a.inner)
        return P.SylvesterADI(p.A, p.B, p.f, p.g, p.alpha, p.beta, p.tau, stream=stream,
                              jacobi=jac, restart=rst, **kw)

    def timed(solver, warmup, steps, profile=False):
        """Mean device seconds per solve (CUDA events on the solver stream),
        L2 flushed before every timed solve."""
        for _ in range(warmup):
            solver.solve()
        if profile:
            solver.profile(True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
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
        solver.timed_solves = steps
        t = sum(s.elapsed_time(e) for s, e in ev) / 1e3 / steps
        return max_over_ranks(t, "cuda"), st

    def summary(solver, t, st):
        info = solver.info()
        stats = solver.kernel_stats()
        so_ms = sum(stats[k][0] for k in SWEEPS)
        so_by = sum(stats[k][1] for k in SWEEPS)
        return {"s": t, "status": st, "outer_steps": info["steps"], "inner_its_A": info["inner_its_A"],
                "inner_its_B": info["inner_its_B"], "rel_res_comp": info["rel_res_comp"],
                "launches_per_solve": info["launches"], "ticks_per_solve": info["ticks"],
                "spmm_orth_GBps": so_by / (so_ms * 1e-3) / 1e9 if so_ms else None,
                "kernel_ms_per_solve": {k: round(v[0] / max(1, solver.timed_solves), 2)
                                        for k, v in stats.items() if v[3] > 0}}, info, stats

    def kname(k):
        return DCGS2_NAMES.get(k, k) if a.ortho == "dcgs2" else k

    def kernel_table(stats):
        total_ms = sum(v[0] for v in stats.values())
        return {kname(k): {"ms": round(v[0], 3), "share": round(v[0] / total_ms, 4) if total_ms else None,
                    "launches": v[3],
                    "GBps": round(v[1] / (v[0] * 1e-3) / 1e9, 1) if v[0] > 0 else None,
                    "TFLOPs": round(v[2] / (v[0] * 1e-3) / 1e12, 4) if v[0] > 0 else None}
                for k, v in stats.items() if v[3] > 0}

    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as fh_:
            peaks = json.load(fh_)
    hbm = peaks.get("hbm_gbs")
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs, copy kernel)" if hbm else "fallback 6800 GB/s"
    hbm = hbm or 6800.0

    # ---- headline: mixed precision (float32 Krylov basis and sweeps, float64
    # outer iteration), adaptive inner tolerances; host driver with CUDA
    # events on every 4th device iteration for the per-kernel times ----
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    solver = make(strategy=a.strategy, precision=a.precision, driver=1)
    torch.cuda.synchronize()
    footprint = free0 - torch.cuda.mem_get_info()[0]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t_solve, st = timed(solver, a.warmup, a.steps, profile=True)
    clocks = sampler.stop()
    main_sum, info, stats = summary(solver, t_solve, st)
    solver.profile(False)

    # ---- end to end through the public API with host buffers ----
    fh = torch.from_numpy(np.asfortranarray(p.f)).pin_memory()
    gh = torch.from_numpy(np.asfortranarray(p.g)).pin_memory()
    kr = info["kr"]
    fdt = torch.complex128 if info["is_complex"] else torch.float64
    Zh = torch.empty((kr, n), dtype=fdt).pin_memory()
    Yh = torch.empty((kr, m), dtype=fdt).pin_memory()
    gmh = torch.empty(kr, dtype=fdt).pin_memory()
    e2e = []
    for k in range(a.steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        P.sylv_adi_set_rhs(solver.h, fh.numpy(), gh.numpy())
        solver.solve()
        kro, isc = C.c_int32(), C.c_int32()
        P.load().sylv_adi_factors(solver.h, Zh.data_ptr(), Yh.data_ptr(), gmh.data_ptr(), 0,
                                  C.byref(kro), C.byref(isc))
        e2e.append(time.perf_counter() - t0)
    barrier()
    e2e_v = max_over_ranks(sum(e2e) / len(e2e), "cuda")
    solver.close()

    # ---- comparison runs ----
    variants = {}
    if not a.no_variants:
        for name, kw, w_, k_, prof in (
                ("fp64", dict(strategy=a.strategy, precision="fp64"), 1, 2, True),
                ("fp64_fixed_1e-12", dict(strategy="fixed", fixed_tol=1e-12, precision="fp64"), 0, 1, True),
                ("bf16_basis", dict(strategy=a.strategy, precision="bf16"), 1, 2, True),
                # one CUDA graph per solve, device-set conditional nodes (no kernel events)
                ("fp32_graph", dict(strategy=a.strategy, precision="fp32", driver=0), 1, 3, False),
                ("fp64_graph", dict(strategy=a.strategy, precision="fp64", driver=0), 1, 2, False),
                ("fp32_cgs2", dict(strategy=a.strategy, precision="fp32", ortho="cgs2"), 1, 2, True),
                ("fp32_bicgstab", dict(strategy=a.strategy, precision="fp32", inner="bicgstab"), 1, 3, True),
                ("fp64_bicgstab", dict(strategy=a.strategy, precision="fp64", inner="bicgstab"), 1, 2, True),
                ("fp32_bicgstab_graph", dict(strategy=a.strategy, precision="fp32", inner="bicgstab", driver=0),
                 1, 3, False)):
            sv = make(**kw)
            tv, stv = timed(sv, w_, k_, profile=prof)
            variants[name], _, vst = summary(sv, tv, stv)
            variants[name]["strategy"] = kw["strategy"]
            if name == "fp64":
                # the float64 sweeps are bound by the float64 pipe
                dk = max(SWEEPS, key=lambda k_: vst[k_][0])
                ms_, by_, fl_, la_ = vst[dk]
                tf = (fl_ / la_) / ((ms_ / la_) * 1e-3) / 1e12
                variants[name]["roofline"] = {"bound": "alu", "kernel": dk, "achieved": tf,
                                              "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                                              "frac": tf / FP64_NOMINAL_TFLOPS}
            sv.close()
        fixed = variants["fp64_fixed_1e-12"]["s"]
        variants["speedup_mixed_adaptive_vs_fp64_fixed_1e-12"] = fixed / t_solve
        variants["speedup_mixed_adaptive_graph_vs_fp64_fixed_1e-12"] = fixed / variants["fp32_graph"]["s"]
        variants["speedup_fp64_adaptive_vs_fp64_fixed_1e-12"] = fixed / variants["fp64"]["s"]

        # ---- batched workload: 64 independent 2D instances in one device loop ----
        probs = batch_future.result() if batch_future is not None else []
        for prec, orth in ((("fp32", "cgs2"), ("fp32", "dcgs2"), ("fp64", "cgs2"), ("fp32", "bicgstab"))
                           if probs else ()):
            inner = "bicgstab" if orth == "bicgstab" else "gmres"
            with P.SylvesterADIBatch(probs, stream=stream, strategy=a.strategy, precision=prec, jacobi=1,
                                     restart=30, ortho="cgs2" if inner == "bicgstab" else orth,
                                     inner=inner) as bt:
                nsolve = 0
                bt.solve()
                nsolve += 1
                evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(2)]
                barrier()
                stb = 0
                for k in range(2):
                    with torch.cuda.stream(stream):
                        flush.zero_()
                        evb[k][0].record(stream)
                    stb = bt.solve()
                    nsolve += 1
                    with torch.cuda.stream(stream):
                        evb[k][1].record(stream)
                barrier()
                tb = max_over_ranks(sum(s_.elapsed_time(e_) for s_, e_ in evb) / 1e3 / 2, "cuda")
                infos = [bt.info(i) for i in range(len(probs))]
                bs = bt.stats()
                variants[f"batch64_{prec}_{orth}"] = {
                    "s": tb, "instances_per_s": len(probs) / tb, "status": stb,
                    "converged": sum(1 for q, i_ in zip(probs, infos) if i_["status"] == 0 and i_["rel_res_comp"] < q.tau),
                    "outer_steps_total": sum(i_["steps"] for i_ in infos),
                    "inner_its_total": sum(i_["inner_its_A"] + i_["inner_its_B"] for i_ in infos),
                    "ticks_per_solve": bs["ticks"], "launches_per_solve": bs["launches"],
                    "algorithmic_GBps": bs["bytes"] / nsolve / tb / 1e9,
                    "rows": sum((q.A.n + q.B.n) * q.r for q in probs)}
    pool.shutdown()

    # ---- roofline of the dominant kernel of the headline solve (HBM) ----
    dom = max(SWEEPS, key=lambda k: stats[k][0])
    ms, by, fl, la = stats[dom]
    ach_gb = (by / la) / ((ms / la) * 1e-3) / 1e9 if ms > 0 else None
    ratio = NCU_TRAFFIC_RATIO.get(dom)
    # time lower bound of a solve: all its algorithmic bytes (every kernel,
    # every launch of the timed solves) at the measured copy bandwidth
    solve_bytes = sum(v[1] for v in stats.values()) / max(1, a.steps)
    bound_s = solve_bytes / (hbm * 1e9)
    line = {
        "metric": METRIC, "value": t_solve, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 Krylov basis/sweeps + f64 outer" if a.precision == "fp32" else a.precision,
        "data": "synthetic",
        "config": {"workload": a.workload, "n": n, "m": m, "r": r, "restart": rst,
                   "jacobi": bool(jac), "strategy": a.strategy, "tau": p.tau, "precision": a.precision,
                   "kmax": a.kmax, "ortho": a.ortho,
                   "driver": "host (per-kernel CUDA events on every 4th device iteration)",
                   "shifts": len(p.alpha), "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "flushed (512 MiB write) before every timed solve",
                   "outer_steps": info["steps"], "inner_its_A": info["inner_its_A"],
                   "inner_its_B": info["inner_its_B"], "rel_res_comp": info["rel_res_comp"],
                   "status": st, "device_bytes_of_solver": footprint},
        "roofline": {"bound": "hbm", "kernel": kname(dom), "achieved": ach_gb, "peak": hbm, "unit": "GB/s",
                     "frac": (ach_gb / hbm) if ach_gb else None, "peak_source": hbm_src,
                     "traffic": (ratio * by / la) if ratio else None,
                     "sweeps_GBps": main_sum["spmm_orth_GBps"],
                     "sweeps_frac": (main_sum["spmm_orth_GBps"] / hbm) if main_sum["spmm_orth_GBps"] else None,
                     "solve_algorithmic_bytes": solve_bytes, "solve_time_lower_bound_s": bound_s,
                     "solve_time_over_bound": (t_solve / bound_s) if bound_s > 0 else None},
        "kernels": kernel_table(stats),
        "variants": variants,
        "gpu_launches": info["launches"] * a.steps,
        "clocks": clocks,
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": (n + m) * r * 8,
                "d2h_bytes_per_step": ((n + m) * kr + kr) * (16 if info["is_complex"] else 8)},
    }
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a.workload, a.strategy, a.cpu_sample_its, info)
        # the same oracle with every host core available to its dense operations
        ncores = os.cpu_count() or 1
        if ncores > 1:
            allc = cpu_baseline(a.workload, a.strategy, a.cpu_sample_its, info, threads=ncores)
            line["cpu_baseline"]["all_cores"] = {k: allc[k] for k in ("value", "unit", "cores", "sample")}
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
