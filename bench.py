#!/usr/bin/env python
"""Benchmark of the GA-NGMRES gradient-evaluation hot path on one GB300 per process.

Workload: 3D 256^3 mass-preserving (continuity) model, n_t = 16, H1 regularisation alpha = 1e-3,
GA-NGMRES(10; 4, 2), trajectory checkpointing every 4 steps, FP32 fields with FP64 reductions, inputs
= 64 anisotropic Gaussians (densities) displaced by a smooth velocity of up to 6 voxels (seeded,
synthetic). One step = one GA-NGMRES iteration (ga_step): preconditioner, Armijo line search (state
solves), reduced gradient(s) (state + adjoint solves, body force, spectral epilogue), window inner
products, least squares, combination and stop test.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). `value` is gradient evaluations per second over all ranks (each rank
runs an independent replica: the problem does not shard), `e2e` the same through host buffers,
`tts_s` the time to relative gradient 1e-2 from v = 0. The reference arm times the FP64 NumPy oracle
on the host cores on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "gradient evals/s & GA-NGMRES time to rel-grad 1e-2 at 256^3; HBM roofline frac"
UNIT = "grad_evals/s"
N = 256
NT = 16
SETTINGS = dict(nt=NT, model="continuity", reg_order=1, alpha=1e-3, ckpt_every=4, window=10, sigma=4,
                tau=2, max_iter=200, rel_tol=1e-2)
WORKLOAD_NAME = ("cont3d256: 256^3 continuity (mass-preserving), nt=16, H1 alpha=1e-3, "
                 "GA-NGMRES(10;4,2), checkpoint every 4, 64 anisotropic Gaussian densities, 6-voxel velocity")
CPU_SAMPLE_N = 80  # oracle sample grid of the default line (same recipe), scaled to 256^3 by voxel count
REF_SAMPLE_N = 48  # oracle sample grid of each step of the reference arm

# kernel classes timed with events inside the library (ga_prof_start)
PROF_SL_FWD, PROF_DERIV, PROF_FFT, PROF_SL_ADJ, PROF_DERIV_PAIR = 0, 1, 2, 3, 4

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one k_sl_tile2<1> launch from an ncu
# capture of this benchmark at 192^3 (`--sl-depth 12,8`: chained state steps at brick depth 12,
# 171.7 MB read + 55.7 MB written, mean of 3 launches), scaled to n^3 by the voxel count. Valid for the
# kernel as captured, at that brick depth; None while the kernel has changed since the last capture.
SL_FWD_TRAFFIC_192 = 227.4e6
SL_FWD_TRAFFIC_DEPTH = 12


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(ms, units, device="cuda"):
    """Whole-job figures of one timed region: the slowest rank's time and the units all ranks
    processed (a no-op without an initialised process group of more than one rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_inputs(n=N, seed=0):
    """The benchmark recipe on an n^3 grid (n an int) or on a given (n0, n1, n2) grid."""
    from synth.inputs import workload

    return workload("cont3d256", seed=seed, n=tuple(n) if isinstance(n, (tuple, list)) else (n, n, n))


def _oracle_worker(job):
    """One host process: the unmodified FP64 oracle on an n^3 sample of the benchmark recipe. Runs
    `warmup` untimed and `steps` timed evaluations of `kind` ('gradient' or 'objective') at
    v = v_true / 2 and returns the seconds of each timed evaluation."""
    n, kind, steps, warmup = job
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle.problem import Problem as OProblem

    w = make_inputs(n)
    P = OProblem(w["m0"], w["m1"], nt=NT, model="continuity", reg_order=1, alpha=1e-3)
    v = 0.5 * w["v_true"]
    fn = P.gradient if kind == "gradient" else P.objective
    for _ in range(warmup):
        fn(v)
    out = []
    for _ in range(steps):
        t0 = time.perf_counter()
        fn(v)
        out.append(time.perf_counter() - t0)
    return out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_oracle_pool(jobs):
    """Run oracle jobs in a pool of spawned processes, one per job, all concurrently (the pool is
    spawned, never forked: the parent may hold a CUDA context). Each child is held to one thread so
    the processes do not oversubscribe the cores."""
    import multiprocessing as mp

    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, jobs)
            wall = time.perf_counter() - t0
    finally:
        for k, val in saved.items():
            if val is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = val
    return res, wall


def cpu_baseline(n=CPU_SAMPLE_N, cores=None):
    """The FP64 oracle, as it stands (single-threaded NumPy), on every host core at once: each core
    runs one independent evaluation on an n^3 sample of the same recipe (three quarters of the cores
    a reduced gradient, the rest an objective). Throughput = gradient evaluations per second of all
    cores, scaled to 256^3 by the voxel count."""
    cores = cores or host_cores()
    n_obj = max(1, cores // 4) if cores > 1 else 0
    jobs = [(n, "gradient", 1, 0)] * (cores - n_obj) + [(n, "objective", 1, 0)] * n_obj
    res, wall = run_oracle_pool(jobs)
    tg = [t for r, j in zip(res, jobs) if j[1] == "gradient" for t in r]
    to = [t for r, j in zip(res, jobs) if j[1] == "objective" for t in r]
    scale = (N / n) ** 3
    t_grad = statistics.mean(tg)  # seconds per gradient on one core at n^3
    t_obj = statistics.mean(to) if to else None
    value = cores / (t_grad * scale)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} concurrent single-threaded FP64 oracle evaluations of the same recipe at {n}^3 "
                      f"(nt=16, v = v_true/2): {len(tg)} reduced gradients ({t_grad:.1f} s each) and {len(to)} "
                      f"objectives; throughput = cores / seconds per gradient, scaled to 256^3 by voxel count "
                      f"x{scale:.1f}; pool wall {wall:.1f} s",
            "s_per_grad_1core_256": t_grad * scale,
            "s_per_obj_1core_256": (t_obj * scale) if t_obj else None}


def run_reference(args):
    """The oracle arm: K timed steps after W warm-ups, each step one reduced gradient per host core at
    the reference sample size (all cores concurrently), scaled to 256^3 by voxel count."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n = REF_SAMPLE_N
    cores = host_cores()
    res, wall = run_oracle_pool([(n, "gradient", args.steps, args.warmup)] * cores)
    per = [t for r in res for t in r]
    t_grad = statistics.mean(per)
    scale = (N / n) ** 3
    value = cores / (t_grad * scale)
    sample = (f"each step: {cores} concurrent single-threaded FP64 oracle reduced gradients of the same recipe at "
              f"{n}^3 (nt=16), {t_grad:.2f} s each, scaled to 256^3 by voxel count x{scale:.0f}; pool wall "
              f"{wall:.1f} s for {args.warmup} warm-up + {args.steps} timed steps")
    cb = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_grad * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "sample": sample},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Configuration sweep after the paper's studies: hyperparameters w and p = (sigma, tau) (Sec. 3.3),
# regularisation parameter (Sec. 3.4) and mesh refinement with n_t proportional to n (Sec. 3.5).
SWEEP_W = (1, 5, 10, 15, 20, 25, 50)
SWEEP_P = ((1, 0), (5, 1), (1, 5), (5, 5), (4, 2), (2, 4), (6, 3), (3, 6))
SWEEP_ALPHA = (1e-1, 5e-2, 1e-2, 5e-3, 1e-3, 5e-4)
SWEEP_MESH = ((64, 4), (128, 8), (256, 16), (512, 32))


def run_sweep(args):
    """Solves of the 3D advection recipe (low-pass template of 256 signed blobs, |k| <= 4 velocity of
    2 voxels, H2, FP32 fields) for every configuration of the three studies; one JSON line with a row
    per solve: iterations, gradient/objective evaluations, PDE solves, relative mismatch (dist),
    relative gradient and time to solution."""
    import torch

    import paper_2510_08782_gb300 as ga
    from paper_2510_08782_gb300 import build
    from synth.inputs import workload

    build.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    parts = set(args.sweep_parts.split(","))
    data = {}

    def fields(n):
        if n not in data:
            w = workload("adv3d64", seed=0, n=(n, n, n))
            data[n] = (torch.from_numpy(w["m0"].astype(np.float32)).cuda(),
                       torch.from_numpy(w["m1"].astype(np.float32)).cuda())
        return data[n]

    def solve(n, nt, alpha, window, sigma, tau, rel_tol, method="ga-ngmres"):
        m0, m1 = fields(n)
        P = ga.Problem(m0, m1, nt=nt, model="advection", reg_order=2, alpha=alpha, prec="mixed", window=window,
                       sigma=sigma, tau=tau, max_iter=200, rel_tol=rel_tol, method=method)
        v = torch.zeros((3, n, n, n), dtype=torch.float32, device="cuda")
        mis0 = P.objective(v)  # the regulariser vanishes at v = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        err = None
        try:
            st, _ = P.solve(v)
        except ga.GaError as e:
            err = str(e)
            st = ga.Stats()
            ga.lib().ga_get_stats(P.ctx, st)
        torch.cuda.synchronize()
        row = {"n": n, "nt": nt, "alpha": alpha, "w": window, "p": [sigma, tau], "method": method,
               "iters": st.iters, "grad_evals": st.grad_evals, "obj_evals": st.obj_evals,
               "pde_solves": st.pde_solves, "converged": bool(st.converged), "grad": st.rel_grad_inf,
               "dist": st.mismatch / mis0 if mis0 > 0 else None, "tts_s": time.perf_counter() - t0,
               "t_grad_ms": st.t_grad_ms, "t_obj_ms": st.t_obj_ms, "error": err}
        P.close()
        del v
        return row

    def solve_inc(window, sigma, tau, method="ga-ngmres"):
        """One solve of the incompressible stand-in of Sec. 3.6 (2D 256^2 sinusoidal images, H3,
        alpha = 1e-4, n_t = 16, tolerance 1e-3) in FP64, with det grad y of the solution."""
        if "inc" not in data:
            w = workload("inc2d256", seed=0)
            data["inc"] = (w, torch.from_numpy(w["m0"]).cuda(), torch.from_numpy(w["m1"]).cuda())
        w, m0, m1 = data["inc"]
        P = ga.Problem(m0, m1, nt=w["nt"], model="incompressible", reg_order=w["reg_order"], alpha=w["alpha"],
                       prec="fp64", window=window, sigma=sigma, tau=tau, max_iter=200, rel_tol=w["rel_tol"],
                       method=method)
        v = torch.zeros((2,) + tuple(w["n"]), dtype=torch.float64, device="cuda")
        mis0 = P.objective(v)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        err = None
        try:
            st, _ = P.solve(v)
        except ga.GaError as e:
            err = str(e)
            st = P.stats()
        torch.cuda.synchronize()
        tts = time.perf_counter() - t0
        u = torch.empty_like(v)
        jd = torch.empty(tuple(w["n"]), dtype=torch.float64, device="cuda")
        P.deformation(v, u, jd)
        row = {"n": list(w["n"]), "nt": w["nt"], "alpha": w["alpha"], "w": window, "p": [sigma, tau],
               "method": method, "iters": st.iters, "grad_evals": st.grad_evals, "obj_evals": st.obj_evals,
               "pde_solves": st.pde_solves, "converged": bool(st.converged), "grad": st.rel_grad_inf,
               "dist": st.mismatch / mis0 if mis0 > 0 else None, "tts_s": tts,
               "det_min": float(jd.min()), "det_mean": float(jd.mean()), "det_max": float(jd.max()),
               "det_std": float(jd.std()), "error": err}
        P.close()
        return row

    rows = {"hyper": [], "alpha": [], "mesh": [], "inc": []}
    t_all = time.perf_counter()
    tol = args.sweep_tol  # the paper's default tolerance is 5e-2 (Sec. 3.1)
    if "hyper" in parts:  # Sec. 3.3: n = 128, n_t = 8, alpha = 1e-3
        for w in SWEEP_W:
            for sg, ta in SWEEP_P:
                rows["hyper"].append(solve(128, 8, 1e-3, w, sg, ta, tol))
        rows["hyper"].append(solve(128, 8, 1e-3, 0, 1, 0, tol, method="rpgd"))
        rows["hyper"].append(solve(128, 8, 1e-3, 10, 4, 2, tol, method="ga-aa"))
    if "alpha" in parts:  # Sec. 3.4
        for a in SWEEP_ALPHA:
            rows["alpha"].append(solve(128, 8, a, 0, 1, 0, tol, method="rpgd"))
            for w in (10, 25):
                for sg, ta in ((5, 1), (4, 2)):
                    rows["alpha"].append(solve(128, 8, a, w, sg, ta, tol))
    if "mesh" in parts:  # Sec. 3.5: w = 25, p = (4, 2), alpha = 1e-3, tolerance 1e-3
        for n, nt in SWEEP_MESH:
            if n > args.sweep_max_n:
                continue
            rows["mesh"].append(solve(n, nt, 1e-3, 25, 4, 2, 1e-3))
            data.pop(n, None)
            torch.cuda.empty_cache()
    if "inc" in parts:  # Sec. 3.6: incompressible flow, H3
        for w in (5, 10, 25):
            for sg, ta in ((4, 2), (5, 1), (2, 4)):
                rows["inc"].append(solve_inc(w, sg, ta))
        rows["inc"].append(solve_inc(0, 1, 0, method="rpgd"))
    total_s = time.perf_counter() - t_all
    if rank != 0:
        return 0
    allrows = rows["hyper"] + rows["alpha"] + rows["mesh"] + rows["inc"]
    conv = sum(r["converged"] for r in allrows)
    print(json.dumps({
        "metric": "configuration sweep: iterations and time to rel-grad per configuration (3D advection H2; "
                  "2D incompressible H3)",
        "value": conv, "unit": "converged runs", "n_gpus": 1, "steps": len(allrows), "warmup": 0,
        "ms_per_step": 1e3 * total_s / max(len(allrows), 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "sweep: adv3d64 recipe; hyperparameters and alpha at 128^3 (n_t = 8), "
                               "mesh 64..512 with n_t = n/16; incompressible: inc2d256 recipe (2D 256^2 "
                               "sinusoidal images, n_t = 16, H3, alpha = 1e-4, FP64)",
                   "tol": args.sweep_tol, "mesh_tol": 1e-3, "inc_tol": 1e-3},
        "gpu_launches": ga.ga_kernel_launches(), "sweep": rows}))
    return 0


GRAPH_MODES = {"off": False, "replay": True, "device": "device"}


def _batch_problem_worker(spec):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from synth.inputs import batch_problem

    w = batch_problem(spec)
    return {k: w[k] for k in ("n", "nt", "alpha", "m0", "m1")}


def batch_inputs(count=32, seed=0):
    """The seeded batch of uneven advection problems, generated on all host cores (spawned pool)."""
    import multiprocessing as mp

    from synth.inputs import batch_specs

    specs = batch_specs(count, seed=seed)
    with mp.get_context("spawn").Pool(min(len(specs), host_cores())) as pool:
        return pool.map(_batch_problem_worker, specs)


BATCH_NAME = ("batch: 32 independent 3D advection problems, grids drawn from {64,96,128,160}^3 (seeded), nt=4, "
              "H1, alpha in {1e-2,1e-3}, GA-NGMRES(5;4,2) to rel-grad 1e-2, FP32 fields with FP64 reductions")


def measure_batch(probs, graphs, steps, warmup, barrier=None):
    """Solve the batch with ga_solve_batch `warmup` + `steps` times from v = 0; returns seconds per
    batch (mean of the timed solves), problems/s and the per-problem statistics of the last solve.
    graphs: 'off' one host worker and stream per problem; 'device' the whole batch as one CUDA graph
    launch with the solver's decisions on the device; 'replay' host workers replaying evaluations."""
    import torch

    import paper_2510_08782_gb300 as ga

    barrier = barrier or torch.cuda.synchronize
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    streams = [torch.cuda.Stream() for _ in probs]
    ctxs, vs = [], []
    for w, st in zip(probs, streams):
        d0, d1 = dev(w["m0"]), dev(w["m1"])
        torch.cuda.synchronize()  # pooled streams do not order themselves after the default stream
        ctxs.append(ga.Problem(d0, d1, nt=w["nt"], model="advection", reg_order=1, alpha=w["alpha"],
                               prec="mixed", window=5, sigma=4, tau=2, max_iter=200, rel_tol=1e-2,
                               stream=st.cuda_stream, graphs=GRAPH_MODES[graphs]))
        vs.append(torch.zeros((3,) + tuple(w["n"]), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()

    def solve_all():
        for v in vs:
            v.zero_()
        torch.cuda.synchronize()
        return ga.ga_solve_batch([P.ctx for P in ctxs], np.float32, vs)

    for _ in range(warmup):
        solve_all()
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        stats, status = solve_all()
    barrier()
    dt = time.perf_counter() - t0
    per = [{"n": int(w["n"][0]), "alpha": w["alpha"], "iters": st.iters, "grad_evals": st.grad_evals,
            "obj_evals": st.obj_evals, "converged": bool(st.converged), "rel_grad_inf": st.rel_grad_inf}
           for w, st in zip(probs, stats)]
    for P in ctxs:
        P.close()
    del vs
    torch.cuda.synchronize()
    return {"graphs": graphs, "s_per_batch": dt / steps, "problems_per_s": len(probs) * steps / dt,
            "timed_solves": steps, "warmup_solves": warmup, "iters_total": sum(r["iters"] for r in per),
            "all_converged": all(r["converged"] for r in per), "per_problem": per}, dt


def run_batch(args):
    """Batched form: 32 independent 3D advection problems with grids drawn from {64,96,128,160}^3,
    n_t = 4, H1, alpha in {1e-2, 1e-3}, GA-NGMRES(5; 4, 2) to rel-grad 1e-2, FP32 fields. One step =
    one ga_solve_batch over all problems."""
    import torch

    import paper_2510_08782_gb300 as ga
    from paper_2510_08782_gb300 import build

    build.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:  # weak scaling: every rank solves its own batch of 32 (seeded by the rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    probs = batch_inputs(32, seed=rank)
    res, dt = measure_batch(probs, args.graphs, args.steps, args.warmup, barrier)
    dt, solved = aggregate_over_ranks(dt, len(probs) * args.steps)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0
    line = {"metric": "problems solved to rel-grad 1e-2 per second (batch of 32 uneven 3D advection problems)",
            "value": solved / dt, "unit": "problems/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_NAME + (", the whole batch one CUDA graph launch" if args.graphs == "device"
                                                 else ", one stream per problem"), "graphs": args.graphs},
            "gpu_launches": ga.ga_kernel_launches(), "per_problem": res["per_problem"]}
    print(json.dumps(line), flush=True)


# Algorithmic HBM bytes per voxel of the 256^3 continuity workload (d = 3, FP32, n_t = 16, checkpoints
# every 4 steps): a reduced gradient 4 [(22 + 1) n_t + 47] plus the checkpoint recompute
# 3/4 (d + 2) 4 n_t (27.85 GB + 4.0 GB at 256^3), an objective-only evaluation (line-search trial)
# 4 (5 n_t + 7) (5.84 GB), and per iteration the window's inner products and combination 2 (w + 2) d 4.
def bytes_per_voxel(nt=NT, window=10, d=3, s=4):
    grad = s * ((22 + 1) * nt + 47) + 0.75 * (d + 2) * s * nt
    obj = s * (5 * nt + 7)
    win = 2 * (window + 2) * d * s
    return grad, obj, win


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tts", action="store_true")
    ap.add_argument("--no-device-tts", action="store_true",
                    help="skip the device-driven (one graph launch) time-to-solution")
    ap.add_argument("--prof-class", type=int, default=PROF_SL_FWD)
    ap.add_argument("--grid", type=int, default=N, help="grid size (default 256; smaller only for smoke runs)")
    ap.add_argument("--shape", default=None,
                    help="n0,n1,n2 grid instead of --grid (small non-cubic cases for profiling captures)")
    ap.add_argument("--sweep-parts", default="hyper,alpha,mesh,inc",
                    help="--workload sweep: comma-separated subset of hyper, alpha, mesh, inc")
    ap.add_argument("--sweep-max-n", type=int, default=512, help="--workload sweep: largest mesh")
    ap.add_argument("--sweep-tol", type=float, default=5e-2,
                    help="--workload sweep: tolerance of the hyperparameter and alpha parts (mesh: 1e-3)")
    ap.add_argument("--workload", default="cont3d256", choices=["cont3d256", "batch", "sweep"],
                    help="cont3d256 (default) or batch: 32 independent advection problems of uneven size")
    ap.add_argument("--graphs", nargs="?", const="replay", default="off", choices=["off", "replay", "device"],
                    help="--workload batch: 'replay' each problem's repeated evaluations from CUDA graphs, or "
                         "'device': the whole batch as one graph launch with the solver's decisions on the device")
    ap.add_argument("--dto", action="store_true",
                    help="also time the discretise-then-optimise gradient (advection transport, same data)")
    ap.add_argument("--compare-methods", action="store_true",
                    help="also time the same solve with GA-AA and RPGD (mixed precision, same settings)")
    ap.add_argument("--no-fp64-tts", action="store_true",
                    help="skip the same GA-NGMRES solve on the FP64 GPU path and the per-result error of the "
                         "mixed path against it")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batch of 32 uneven advection problems (both batched forms)")
    ap.add_argument("--sl-depth", default=None,
                    help="STATE,ADJOINT: fix the transport steps' brick depths (4, 8 or 12) instead of the "
                         "setup autotuner's choice, e.g. for a profiler run, whose timing the autotuner "
                         "would otherwise measure")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "sweep":
        return run_sweep(args)

    import torch

    import paper_2510_08782_gb300 as ga
    from paper_2510_08782_gb300 import build

    ws, rank, local = dist_env()
    build.build()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.grid
    shape = tuple(int(x) for x in args.shape.split(",")) if args.shape else (n, n, n)
    w = make_inputs(shape)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    m0, m1 = dev(w["m0"]), dev(w["m1"])
    P = ga.Problem(m0, m1, prec="mixed", **SETTINGS)
    if args.sl_depth:
        ga.ga_op_set_sl_depth(P.ctx, *(int(x) for x in args.sl_depth.split(",")))
    v = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- warm-up (W GA-NGMRES iterations from v = 0) ----
    for _ in range(args.warmup):
        P.step(v)
    # ---- timed: K iterations of a fresh solve from v = 0 ----
    P.reset()
    v.zero_()
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except Exception:
            pass
    sampler = ClockSampler(gpu_index)
    barrier()
    launches0 = ga.ga_kernel_launches()
    ga.ga_prof_start(P.ctx, args.prof_class)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st = None
    for _ in range(args.steps):
        st = P.step(v)
    e1.record()
    barrier()
    clocks = sampler.stop()
    prof_ms, prof_n = ga.ga_prof_stop(P.ctx)
    launches = ga.ga_kernel_launches() - launches0
    deriv_tiles = ga.ga_op_get_tiles(P.ctx, 3)  # pencil pairs per CTA chosen by the setup autotuner
    ms = e0.elapsed_time(e1)
    grad_evals = st.grad_evals
    ms_max, total_evals = aggregate_over_ranks(ms, grad_evals)
    value = total_evals / (ms_max / 1e3)
    step_stats = st.as_dict()

    # ---- roofline of the dominant kernel: algorithmic bytes per launch / mean event duration ----
    nv = int(np.prod(shape))
    algo = {PROF_SL_FWD: ("sl_forward continuity step: read pi_j, mu, 3 displacement fields, write pi_{j+1}", 24),
            PROF_SL_ADJ: ("sl_adjoint continuity step: read lambda_{j+1}, 3 displacement fields, write lambda_j", 20),
            PROF_DERIV: ("fused FFT-derivative pass: read f, read multiplier, read+write accumulator", 16),
            PROF_FFT: ("3D real FFT (3 passes)", 24),
            PROF_DERIV_PAIR: ("body-force FFT-derivative pass over two time steps: read f, f2, multiplier, "
                              "multiplier2, read+write accumulator", 24)}[args.prof_class]
    hbm, peak_kind = peaks()
    per_launch_ms = prof_ms / max(prof_n, 1)
    bytes_per_launch = algo[1] * nv
    achieved = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
    sl_depth = ga.ga_op_get_sl_depth(P.ctx)  # brick depths (state, adjoint steps) chosen at setup
    traffic = None
    if args.prof_class == PROF_SL_FWD and SL_FWD_TRAFFIC_192 is not None and sl_depth[0] == SL_FWD_TRAFFIC_DEPTH:
        traffic = round(SL_FWD_TRAFFIC_192 * nv / 192.0 ** 3)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": traffic,
                "traffic_note": "bytes per launch of the chained state step from an ncu capture at 192^3 "
                                "(brick depth 12) scaled by voxel count; null for another brick depth",
                "kernel": algo[0],
                "bytes_per_launch": bytes_per_launch, "launches": prof_n, "mean_launch_ms": per_launch_ms,
                "peak_kind": f"{peak_kind} (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)"}
    # The semi-Lagrangian steps are bound by shared-memory bandwidth, not HBM: each interpolated field
    # reads 64 taps x 4 B per voxel from the staged tile. Peak: 128 B per clock per SM at the median SM
    # clock sampled during the timed region.
    taps_fields = {PROF_SL_FWD: 2, PROF_SL_ADJ: 1}.get(args.prof_class)
    if taps_fields:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
        smem_peak = sms * 128 * mhz * 1e6 / 1e9
        smem_bytes = 64 * 4 * taps_fields * nv
        smem_achieved = smem_bytes / (per_launch_ms / 1e3) / 1e9
        roofline["secondary"] = {"bound": "smem", "achieved": round(smem_achieved, 1), "peak": round(smem_peak, 1),
                                 "unit": "GB/s", "frac": round(smem_achieved / smem_peak, 4),
                                 "bytes_per_launch": smem_bytes,
                                 "peak_kind": f"nominal: {sms} SMs x 128 B/clock x {mhz:.0f} MHz (sampled)"}

    # ---- time to rel-grad 1e-2 from v = 0 (GA-NGMRES) ----
    tts = None
    if not args.no_tts:
        P.reset()
        v.zero_()
        barrier()
        t0 = time.perf_counter()
        try:
            stt, status = P.solve(v)
            err = None
        except ga.GaError as e:  # e.g. an exhausted line search: report it with the last statistics
            err = str(e)
            stt = ga.Stats()
            ga.lib().ga_get_stats(P.ctx, stt)
        torch.cuda.synchronize()
        tts = {"tts_s": time.perf_counter() - t0, "iters": stt.iters, "converged": bool(stt.converged),
               "rel_grad_inf": stt.rel_grad_inf, "grad_evals": stt.grad_evals, "obj_evals": stt.obj_evals,
               "pde_solves": stt.pde_solves, "mismatch": stt.mismatch, "obj": stt.obj, "error": err}
        # roofline of the whole solve: algorithmic bytes of its evaluations and window operations
        bg, bo, bw = bytes_per_voxel()
        tb = (stt.grad_evals * bg + stt.obj_evals * bo + stt.iters * bw) * nv
        hbm_peak, kind = peaks()
        tts["roofline"] = {"bound": "hbm", "algorithmic_bytes": tb, "achieved": round(tb / tts["tts_s"] / 1e9, 1),
                           "peak": hbm_peak, "unit": "GB/s", "frac": round(tb / tts["tts_s"] / 1e9 / hbm_peak, 4),
                           "model": "per voxel: gradient 4[23 nt + 47] + 3/4 (d+2) 4 nt (checkpoint recompute), "
                                    "objective 4 (5 nt + 7), window 2 (w+2) d 4 per iteration",
                           "peak_kind": kind}

    v_sol = v.clone()  # the GA-NGMRES solution (with --no-tts: the last timed iterate)

    # ---- deformation diagnostics of the solution: det grad y statistics, as reported with the results ----
    deformation = None
    if tts is not None:
        u_def = torch.empty_like(v)
        j_def = torch.empty(shape, dtype=v.dtype, device="cuda")
        P.deformation(v, u_def, j_def)  # first use loads the kernels of this path
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.deformation(v, u_def, j_def)
        torch.cuda.synchronize()
        def_ms = (time.perf_counter() - t0) * 1e3
        jd = j_def.double()
        deformation = {"det_min": float(jd.min()), "det_mean": float(jd.mean()), "det_max": float(jd.max()),
                       "det_std": float(jd.std()), "max_displacement_cells": float(u_def.abs().max()),
                       "ms": def_ms}
        del u_def, j_def, jd

    # ---- the same solve device-driven: one CUDA graph launch, decisions on the device (graphs = 2) ----
    tts_dev = None
    if tts is not None and not args.no_device_tts:
        Pd = ga.Problem(m0, m1, prec="mixed", graphs="device", **SETTINGS)
        vd = torch.zeros_like(v)
        t0 = time.perf_counter()
        try:
            Pd.solve(vd)  # the first call records and instantiates the graph
            torch.cuda.synchronize()
            first_s = time.perf_counter() - t0
            vd.zero_()
            barrier()
            t0 = time.perf_counter()
            sd, _ = Pd.solve(vd)
            err = None
        except ga.GaError as e:
            first_s, err = None, str(e)
            sd = Pd.stats()
        torch.cuda.synchronize()
        tts_dev = {"tts_s": time.perf_counter() - t0, "iters": sd.iters, "converged": bool(sd.converged),
                   "rel_grad_inf": sd.rel_grad_inf, "grad_evals": sd.grad_evals, "obj_evals": sd.obj_evals,
                   "first_call_s": first_s, "identical_to_host_driven": bool(torch.equal(vd, v_sol)),
                   "error": err}
        Pd.close()
        del Pd, vd
        torch.cuda.empty_cache()

    # ---- the same solve on the FP64 GPU path, and the error of the mixed path against it ----
    fp64 = None
    if not args.no_fp64_tts:
        d64 = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
        P64 = ga.Problem(d64(w["m0"]), d64(w["m1"]), prec="fp64", **SETTINGS)
        v64 = torch.zeros((3,) + shape, dtype=torch.float64, device="cuda")
        barrier()
        t0 = time.perf_counter()
        try:
            s64, _ = P64.solve(v64)
            err = None
        except ga.GaError as e:
            err = str(e)
            s64 = P64.stats()
        torch.cuda.synchronize()
        fp64 = {"tts_s": time.perf_counter() - t0, "iters": s64.iters, "converged": bool(s64.converged),
                "rel_grad_inf": s64.rel_grad_inf, "grad_evals": s64.grad_evals, "obj_evals": s64.obj_evals,
                "mismatch": s64.mismatch, "obj": s64.obj,
                "t_grad_ms_per_eval": s64.t_grad_ms / max(s64.grad_evals, 1), "error": err}
        if tts is not None:
            fp64["mixed_tts_speedup"] = fp64["tts_s"] / tts["tts_s"]
            # error of the mixed path per result: objective and gradient at the mixed solution, against
            # the FP64 GPU path at the same velocity (the FP64 path matches the oracle to 1e-10)
            gm = torch.empty_like(v_sol)
            g64 = torch.empty_like(v64)
            vs64 = v_sol.double()
            obj_m = P.gradient(v_sol, gm)
            obj_64 = P64.gradient(vs64, g64)
            ref_n = float(torch.linalg.vector_norm(g64))
            fp64["mixed_vs_fp64_at_mixed_solution"] = {
                "rel_l2_grad": float(torch.linalg.vector_norm(gm.double() - g64)) / ref_n,
                "rel_err_obj": abs(obj_m - obj_64) / abs(obj_64),
                "obj_mixed": obj_m, "obj_fp64": obj_64,
                "rel_inf_grad": float((gm.double() - g64).abs().max() / g64.abs().max()),
                "note": "g and obj of the mixed (FP32 fields, FP64 reductions) path and of the FP64 path, "
                        "both on the GPU, at the mixed GA-NGMRES solution v (cast to FP64)"}
            del gm, g64, vs64
        P64.close()
        del P64, v64
        torch.cuda.empty_cache()

    # ---- the same solve with the other methods of the paper's comparison (optional) ----
    methods = None
    if args.compare_methods:
        methods = {}
        for meth in ("ga-aa", "rpgd"):
            P.close()
            torch.cuda.empty_cache()
            Pm = ga.Problem(m0, m1, prec="mixed", method=meth, **SETTINGS)
            vm = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
            barrier()
            t0 = time.perf_counter()
            try:
                sm, _ = Pm.solve(vm)
                err = None
            except ga.GaError as e:
                err = str(e)
                sm = ga.Stats()
                ga.lib().ga_get_stats(Pm.ctx, sm)
            torch.cuda.synchronize()
            methods[meth] = {"tts_s": time.perf_counter() - t0, "iters": sm.iters, "converged": bool(sm.converged),
                             "rel_grad_inf": sm.rel_grad_inf, "grad_evals": sm.grad_evals,
                             "obj_evals": sm.obj_evals, "error": err}
            Pm.close()
            del Pm, vm
            torch.cuda.empty_cache()
            P = ga.Problem(m0, m1, prec="mixed", **SETTINGS)
        v.zero_()

    # ---- pure gradient throughput (ga_gradient only), at the solution of the timed solve ----
    g = torch.empty_like(v)
    P.gradient(v_sol, g)
    torch.cuda.synchronize()
    e0.record()
    reps = 5
    for _ in range(reps):
        P.gradient(v_sol, g)
    e1.record()
    torch.cuda.synchronize()
    grad_only = reps / (e0.elapsed_time(e1) / 1e3)

    # ---- discretise-then-optimise gradient (optional): advection transport of the same data ----
    dto_res = None
    if args.dto:
        sa = dict(SETTINGS, model="advection")
        Pa = ga.Problem(m0, m1, prec="mixed", **sa)
        va = torch.from_numpy(np.ascontiguousarray(0.5 * w["v_true"], dtype=np.float32)).cuda()
        go, gd = torch.empty_like(v), torch.empty_like(v)
        Pa.gradient(va, go)
        Pa.gradient_dto(va, gd)
        torch.cuda.synchronize()
        rates = {}
        for name, fn, out in (("otd", Pa.gradient, go), ("dto", Pa.gradient_dto, gd)):
            e0.record()
            for _ in range(3):
                fn(va, out)
            e1.record()
            torch.cuda.synchronize()
            rates[name] = 3 / (e0.elapsed_time(e1) / 1e3)
        rel = float(torch.linalg.vector_norm((gd - go).double()) / torch.linalg.vector_norm(go.double()))
        dto_res = {"model": "advection transport of the same data and settings, v = v_true / 2",
                   "dto_grad_evals_per_s": rates["dto"], "otd_grad_evals_per_s": rates["otd"],
                   "rel_l2_dto_vs_otd": rel}
        Pa.close()
        del Pa, va, go, gd
        torch.cuda.empty_cache()

    # ---- end to end through host buffers: setup from host m0/m1, K steps with a host v ----
    e2e = None
    if not args.no_e2e:
        P.close()
        del P
        torch.cuda.empty_cache()
        hm0 = torch.from_numpy(np.ascontiguousarray(w["m0"], dtype=np.float32)).pin_memory()
        hm1 = torch.from_numpy(np.ascontiguousarray(w["m1"], dtype=np.float32)).pin_memory()
        hv = torch.zeros((3,) + shape, dtype=torch.float32).pin_memory()
        barrier()
        t0 = time.perf_counter()
        Q = ga.Problem(hm0, hm1, prec="mixed", **SETTINGS)
        for _ in range(args.steps):
            sq = Q.step(hv)
        Q.close()
        torch.cuda.synchronize()
        dt, e2e_evals = aggregate_over_ranks(time.perf_counter() - t0, sq.grad_evals)
        e2e = {"value": e2e_evals / dt, "unit": UNIT,
               "h2d_bytes_per_step": int((2 * nv + 3 * nv) * 4 / args.steps),
               "d2h_bytes_per_step": int(3 * nv * 4),
               "note": "timed: ga_setup from pinned host m0/m1 + K ga_step calls with a pinned host v "
                       "(v^(0) uploaded once, v^(k+1) read back every step) + ga_destroy; "
                       "h2d bytes are the job's uploads divided by K"}
    # ---- the batched form (32 uneven advection problems): both forms, seeded per rank ----
    batch = None
    if not args.no_batch:
        probs = batch_inputs(32, seed=rank)
        batch = {"workload": BATCH_NAME}
        for mode in ("off", "device"):
            res, dt = measure_batch(probs, mode, 2, 1, barrier)
            key = "host_workers" if mode == "off" else "one_graph_launch"
            batch[key] = res
        del probs
        torch.cuda.empty_cache()

    cb = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()
        if tts is not None and cb.get("s_per_obj_1core_256"):
            cb["tts_estimate_256_s"] = (tts["grad_evals"] * cb["s_per_grad_1core_256"] +
                                        tts["obj_evals"] * cb["s_per_obj_1core_256"])
            cb["tts_estimate_note"] = ("ESTIMATED oracle time to rel-grad 1e-2 at 256^3 on one core: seconds per "
                                       "gradient and per objective (sample scaled by voxel count) x the GPU "
                                       "solve's evaluation counts")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD_NAME, "grid": list(shape), "nt": NT, "precision":
                           "FP32 fields/transport/FFT, FP64 compensated reductions, Gram and least squares",
                           "step": "one GA-NGMRES iteration (ga_step) of a solve from v=0",
                           "l2": "inputs larger than L2: each 256^3 field is 64 MiB and a step touches GBs",
                           "parallelism": "replicas (one independent problem per GPU)" if ws > 1 else "1 GPU"},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": int(launches),
                "deriv_tiles_zyx": deriv_tiles, "sl_brick_depth_state_adjoint": list(sl_depth),
                "clocks": clocks, "tts": tts, "tts_device": tts_dev, "fp64_tts": fp64, "batch": batch,
                "methods_tts": methods, "deformation": deformation, "dto": dto_res, "grad_only_evals_per_s": grad_only,
                "grad_evals_in_timed_steps": grad_evals, "last_step": {k: step_stats[k] for k in
                                                                       ("iters", "obj_evals", "rel_grad_inf", "obj",
                                                                        "rho_mem")}}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
