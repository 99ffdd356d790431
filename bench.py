#!/usr/bin/env python3
"""Benchmark of the GD-PG lambda path on the 128 x 128 x 600 Gaussian GLAM workload.

One step = one warm-started 50-lambda path fit (glam_fit_path: lambda_max, inner FISTA loop,
Armijo line search, FP64 KKT test to 1e-6 at every lambda) on the synthetic workload with
cubic B-spline bases p = (20, 20, 60), FP32 mode products.  The headline value is prox-grad
(inner PG) iterations per second over the timed steps; the line also carries the H-transform
GB/s of glam_predict, the whole path on an FP64 plan and on TF32 and BF16 plans, the roofline of
the dominant kernel, an end-to-end figure with host buffers, and at N = 1 the FP64 CPU oracle
baseline, the masked Poisson 96 x 96 x 365 path in four precisions, and the batched form: 64
independent fits of uneven shapes through glam_fit_path_batched against the plain FP32 path
fitting them one after another, and on TF32 plans against the FP32 batch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torchrun) every rank fits its own replica of the workload on its
own GPU (independent fits: no collective on the data path) and value is the sum of iterations
over all ranks divided by the slowest rank's time (weak scaling).
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
sys.path.insert(0, ROOT)

METRIC = "prox-grad iters/s & H-transform GB/s on 128x128x600 grid vs FP64 GPU path at KKT 1e-6"
UNIT = "iters/s"
WORKLOAD = "gauss-128x128x600 p=(20,20,60) 50-lambda path, ratio 1e-3, KKT 1e-6"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """Samples nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"glam_clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        self.f = open(self.path, "w")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            self.f.close()
            os.remove(self.path)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# oracle (CPU) legs: the cpu_baseline of our line, and the whole --impl reference arm
# ------------------------------------------------------------------------------------------

def _oracle_setup():
    import gen
    import oracle as O
    pr = gen.make_workload(1)
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    # the quadratic model of the first outer iteration at theta = 0 (W = 1: V = a, Z = Y)
    w = O.irls_weight(d.family, np.zeros_like(d.Y), d.a)
    z = O.working_response(d.family, np.zeros_like(d.Y), d.Y, d.a)
    Lhat = O.lipschitz_bound(d.Xs, w)
    return O, d, lmax, w, z, Lhat


def _oracle_iters(O, d, lmax, w, z, Lhat, iters):
    """`iters` inner PG iterations of the oracle (Sec. 3.2) at lambda = 0.1 lambda_max."""
    t0 = time.perf_counter()
    res = O.inner_pg(d, w, z, np.zeros(d.pshape), 1.0 / Lhat, 0.1 * lmax, tol=0.0, max_iter=iters)
    return res.iters, time.perf_counter() - t0


def cpu_baseline(budget_s=12.0):
    O, d, lmax, w, z, Lhat = _oracle_setup()
    n_it, t = _oracle_iters(O, d, lmax, w, z, Lhat, 1)
    per = max(t, 1e-3)
    k = int(max(2, min(200, budget_s / per)))
    n_it, t = _oracle_iters(O, d, lmax, w, z, Lhat, k)
    out = {"value": n_it / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{n_it} inner PG iterations (FP64 numpy, paper's mode order) of the "
                     f"128x128x600 Gaussian model at lambda = 0.1 lambda_max; {t:.1f} s"}
    out["single_core"] = _oracle_single_core(20)
    out["paths"] = _oracle_paths()
    return out


def _oracle_single_core(iters):
    """The same oracle iterations on one host core: a child process with every BLAS / OpenMP pool
    limited to one thread (the pools are sized when numpy loads, so it cannot be done in-process)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-rate", str(iters)],
                       capture_output=True, text=True, env=env, timeout=600)
    try:
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return {"error": (r.stderr or r.stdout)[-300:]}
    d.update({"cores": 1, "sample": f"{d['iters']} inner PG iterations of the same model, one thread"})
    return d


def _oracle_paths():
    """Whole lambda paths of the oracle on the host cores: the 20x20x20 Gaussian workload (10
    lambdas to KKT 1e-6, complete) and, as a bounded sample of the 96x96x365 Poisson workload, its
    first lambda below lambda_max (one GD-PG solve to KKT 1e-6, at most 3 outer iterations)."""
    import gen
    import oracle as O
    out = {}
    pr = gen.make_workload(0)
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    t0 = time.perf_counter()
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=pr.nlambda, ratio=pr.lambda_min_ratio, tol=1e-6)
    out["gauss_20x20x20_10_lambda_path_s"] = time.perf_counter() - t0
    pr = gen.make_workload(2)
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    lam = float(O.lambda_sequence(lmax, pr.nlambda, pr.lambda_min_ratio)[1])
    t0 = time.perf_counter()
    _, st = O.gdpg(d, lam, np.zeros(d.pshape), lmax, tol=1e-6, max_outer=3)
    out["poisson_96x96x365_second_lambda_s"] = time.perf_counter() - t0
    out["poisson_96x96x365_second_lambda_note"] = ("one GD-PG solve (at most 3 outer iterations) at "
                                                  "the path's second lambda from zero; KKT %.2e" % st.kkt)
    out["cores"] = os.cpu_count()
    return out


def run_reference(args):
    world, rank, _ = _dist()
    if world > 1 and rank != 0:
        return 0
    O, d, lmax, w, z, Lhat = _oracle_setup()
    per_step = 2
    for _ in range(args.warmup):
        _oracle_iters(O, d, lmax, w, z, Lhat, per_step)
    tot_it, tot_t = 0, 0.0
    for _ in range(args.steps):
        it, t = _oracle_iters(O, d, lmax, w, z, Lhat, per_step)
        tot_it += it
        tot_t += t
    v = tot_it / tot_t
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD + " (oracle: inner PG iterations of the same model)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{per_step} inner PG iterations per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def job_totals(dist, t_rank, iters, device):
    """Whole-job figures of independent replicas: the slowest rank's time and the iterations of
    every rank (dist None: this process alone)."""
    if dist is None:
        return t_rank, float(iters)
    import torch
    tt = torch.tensor([t_rank, float(iters)], dtype=torch.float64, device=device)
    tmax = tt.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return tmax[0].item(), tt[1].item()


def run_ours(args):
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import gen
    import paper_1510_03298_gb300 as g
    from paper_1510_03298_gb300 import build as gb
    if not os.path.exists(g.library_path()):
        gb.build()
    g.load_library()

    pr = gen.make_workload(1)
    dev = torch.device("cuda", local)
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    f64 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    X = [f32(x) for x in pr.XT]
    Y, W = f32(pr.Y), f32(pr.W)
    pen = f64(pr.pen_w)
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP32)
    opts = g.glam_opts_default(tol=1e-6, lambda_min_ratio=1e-3)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step():
        flush.fill_(1.0)  # evict L2 between steps
        return g.glam_fit_path(plan, X, Y, W, pen, nlambda=pr.nlambda, opts=opts)

    for _ in range(args.warmup):
        r = step()
    if r.status != g.GLAM_OK:
        raise SystemExit(f"fit failed: {r.message}")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    clocks = Clocks(local)
    launches0 = g.glam_launch_count()
    clocks.start()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record()
    results = [step() for _ in range(args.steps)]
    ev1.record()
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    launches = g.glam_launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    iters = sum(sum(s["inner_iters"] for s in r.stats) for r in results)
    ok = all(r.status == g.GLAM_OK for r in results)
    kkt_max = max(max(s["kkt"] for s in r.stats) for r in results)
    t_job, iters_job = job_totals(dist, ms / 1e3, iters, dev)
    value = iters_job / t_job

    extra = {}
    if rank == 0:
        extra = measure_details(g, torch, pr, plan, X, Y, W, pen, opts, dev, flush, results[-1])
        extra["e2e"] = measure_e2e(g, torch, pr, plan, opts, dev, args.steps)
        # the single-GPU side measurements run at N = 1 only: at N > 1 the other ranks would wait
        # for them in the closing barrier
        if not args.no_config3 and world == 1:
            extra["poisson_96x96x365_paths"] = measure_config3(g, torch, flush)
        if args.batched > 0 and world == 1:
            extra["batched"] = measure_batched(g, torch, args.batched, args.batched_baseline)
        if world == 1 and not args.no_cpu:
            extra["cpu_baseline"] = cpu_baseline()
    if dist is not None:
        dist.barrier()
    if rank == 0:
        st = results[-1].stats
        # time per 50-lambda path to KKT 1e-6 leads (the inner-iteration rate rewards more iterations);
        # the FP64 GPU path, the comparison point of the metric, sits beside it
        fp64 = extra.get("fp64_gpu_path", {})
        lead = {"s_per_path_to_kkt_1e-6": ms / args.steps / 1e3,
                "fp64_gpu_s_per_path_to_kkt_1e-6": fp64.get("ms_per_path", float("nan")) / 1e3,
                "speedup_vs_fp64_gpu_path": fp64.get("ms_per_path", float("nan")) / (ms / args.steps)}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "headline": lead, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": [128, 128, 600], "basis": [20, 20, 60],
                           "nlambda": pr.nlambda,
                           "precision": "fp32-accurate mode products (inner-loop product as 3xTF32 on the tcgen05 tensor cores), fp64 refinement",
                           "l2": "256 MB buffer written between steps",
                           "parallelism": f"replicas x{world}"},
                "gpu_launches": int(launches),
                "clocks": clk,
                "path": {"converged": ok, "max_kkt": kkt_max, "inner_iters_per_step": iters / args.steps,
                         "outer_iters": sum(s["outer_iters"] for s in st),
                         "fp64_passes": sum(s["fp64_passes"] for s in st),
                         "wall_s_per_step": wall / args.steps}}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# dram__bytes_read.sum + dram__bytes_write.sum of one launch of each fused slab kernel on this
# workload, from an ncu capture (cold cache) of the current kernels (None: not captured since the
# kernel last changed)
NCU_TRAFFIC_BYTES = {"3xtf32": 39764736, "tf32": 39698432, "bf16": 20022272}


def measure_details(g, torch, pr, plan, X, Y, W, pen, opts, dev, flush, last):
    peaks, src = _peaks()
    out = {}
    n1, n2, n3 = pr.n
    p1, p2, p3 = pr.p
    n, p = n1 * n2 * n3, p1 * p2 * p3
    # H-transform (glam_predict) throughput: algorithmic bytes = read Theta and X_j, write eta.
    # A timed region is a stream of K calls writing K distinct eta arrays (K x 39.3 MB, more than
    # the 129 MB L2, so the eta writes reach HBM); L2 is flushed before each region.
    theta = last.path[-1].float().contiguous()
    K = 8
    etas = [torch.empty((n3, n2, n1), dtype=torch.float32, device=dev) for _ in range(K)]
    times, cold = [], []
    for r in range(14):
        flush.fill_(1.0)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        # keep the GPU busy while the host enqueues the calls, so that the events bracket the
        # kernels and not the host-side latency of the binding
        torch.cuda._sleep(400_000)
        a.record()
        g.glam_predict(plan, X, theta, etas[0])
        c.record()
        for k in range(1, K):
            g.glam_predict(plan, X, theta, etas[k])
        b.record()
        torch.cuda.synchronize()
        if r >= 4:
            times.append(a.elapsed_time(b) / K)
            cold.append(a.elapsed_time(c))
    t_h = statistics.median(times) / 1e3
    h_bytes = 4 * (n + p + sum(a * b for a, b in zip(pr.n, pr.p)))
    h_flops = 2 * (n3 * p3 * p2 * p1 + n3 * p2 * p1 * n1 + n3 * n2 * p2 * n1)
    out["h_transform"] = {"GB/s": h_bytes / t_h / 1e9, "ms": t_h * 1e3, "bytes": h_bytes,
                          "frac_hbm": h_bytes / t_h / 1e9 / peaks["hbm_gbs"], "peak_src": src,
                          "tflops": h_flops / t_h / 1e12, "calls_per_region": K,
                          "first_call_after_flush_ms": statistics.median(cold),
                          "kernels": "predict_umma_kernel (tcgen05: FP32 first H stage and MMA0, 3xTF32 MMA1)"}
    del etas
    # dominant kernel of the inner iteration: the fused slab kernel G(V (.) H(.)), which a GLAM_FP32
    # plan runs on the tensor cores in the 3xTF32 form (FP32-level accuracy)
    q = g.glam_quad_build(plan, X, theta, Y, W)
    ms = g.glam_time_inner_kernels(plan, X, q, reps=100)
    per_iter = sum(ms)
    # algorithmic FLOPs: the first H stage (X_3 d) and, per slab, T_b = T_a X_1^T, eta = X_2 T_b,
    # r = V (.) eta, S = X_2^T r, S_b = S X_1
    slab = 2 * p2 * p1 * n1 + 4 * n2 * n1 * p2 + n2 * n1 + 2 * p2 * n1 * p1
    fl = slab * n3 + 2 * n3 * p3 * p2 * p1
    # read V, the correction d and X_3 (the kernel forms T_a = X_3 d), X_1 and X_2; write S_b
    by = 4 * n + 4 * n3 * p2 * p1 + 4 * (p + n3 * p3) + 4 * (n1 * p1 + n2 * p2)
    t_f = ms[0] / 1e3
    tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25  # dense TF32 = measured BF16 x nominal ratio
    out["roofline"] = {"bound": "hbm", "kernel": "fused_slab_umma_kernel<3,float> (3xTF32 tcgen05, TMEM accumulators, G(V(.)H) per slab)",
                       "achieved": by / t_f / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": by / t_f / 1e9 / peaks["hbm_gbs"], "traffic": NCU_TRAFFIC_BYTES["3xtf32"],
                       "bytes_per_launch": by, "ms_per_launch": ms[0], "peak_src": src,
                       "bound_note": "intensity %.0f FLOP/B is below the TF32 tensor ridge %.0f FLOP/B"
                                     % (fl / by, tf32_peak * 1e3 / peaks["hbm_gbs"]),
                       "flop_view": {"flops_per_launch": fl, "TFLOP/s": fl / t_f / 1e12,
                                     "tf32_tensor_peak": tf32_peak,
                                     "frac_of_tf32_peak": fl / t_f / 1e12 / tf32_peak}}
    # ms[2] is the mode-3 adjoint, fused with the prox step where the path does so (ms[3] = 0)
    out["inner_iteration_ms"] = {"fused_slab": ms[0], "mode3": ms[1], "mode3_adjoint": ms[2],
                                 "prox": ms[3], "sum": per_iter}
    # the metric's comparison point: the whole 50-lambda path to KKT 1e-6 with a GLAM_FP64 plan
    out["fp64_gpu_path"] = measure_path_precision(g, torch, pr, X, Y, W, pen, opts, flush, last, g.GLAM_FP64)
    out["h_transform_fp64"] = measure_h(g, torch, pr, X, theta, flush, peaks, src, fp64=True)
    out["kron_path"] = measure_kron(g, torch, pr, X, Y, W, pen, opts, flush, last)
    out["banded_fp64_passes"] = measure_banded(g, torch, pr, X, Y, W, pen, opts, flush, last)
    out["tf32_path"] = measure_tf32(g, torch, pr, X, Y, W, pen, opts, flush, last, theta, by, peaks, src)
    out["bf16_path"] = measure_path_precision(g, torch, pr, X, Y, W, pen, opts, flush, last, g.GLAM_BF16,
                                              kernel_bytes=by - 2 * n, peaks=peaks, src=src, theta=theta)
    return out


def measure_h(g, torch, pr, X, theta, flush, peaks, src, fp64=False):
    """H-transform (glam_predict) throughput of an FP64 plan: a stream of 8 calls writing 8 distinct
    eta arrays (more than L2), L2 flushed first; algorithmic bytes 8 (n + p + sum n_j p_j)."""
    n1, n2, n3 = pr.n
    n = n1 * n2 * n3
    p = int(np.prod(pr.p))
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP64)
    Xd = [x.double() for x in X]
    th = theta.double()
    K = 8
    etas = [torch.empty((n3, n2, n1), dtype=torch.float64, device=th.device) for _ in range(K)]
    times = []
    for r in range(8):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(400_000)
        a.record()
        for k in range(K):
            g.glam_predict(plan, Xd, th, etas[k])
        b.record()
        torch.cuda.synchronize()
        if r >= 2:
            times.append(a.elapsed_time(b) / K)
    t = statistics.median(times) / 1e3
    by = 8 * (n + p + sum(a * b for a, b in zip(pr.n, pr.p)))
    plan.close()
    return {"GB/s": by / t / 1e9, "ms": t * 1e3, "bytes": by, "frac_hbm": by / t / 1e9 / peaks["hbm_gbs"],
            "peak_src": src, "kernels": "FP64 SIMT mode products (gemm_kernel<double>)"}


def measure_path_precision(g, torch, pr, X, Y, W, pen, opts, flush, last, precision, kernel_bytes=None,
                           peaks=None, src=None, theta=None):
    """The same 50-lambda path to KKT 1e-6 with another plan precision (GLAM_FP64: the metric's
    comparison point; GLAM_BF16: BF16 inner products with the FP64 polish of every outer
    iteration), timed like a bench step after one warm-up path, against the FP32 path."""
    fp64 = precision == g.GLAM_FP64
    plan = g.Plan(pr.n, pr.p, pr.family, precision)
    cast = (lambda t: t.double()) if fp64 else (lambda t: t)
    Xp, Yp, Wp = [cast(x) for x in X], cast(Y), cast(W)
    g.glam_fit_path(plan, Xp, Yp, Wp, pen, lambdas=last.lambdas[:3], opts=opts)  # warm-up (graph capture)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    res = g.glam_fit_path(plan, Xp, Yp, Wp, pen, nlambda=pr.nlambda, opts=opts)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    iters = sum(s["inner_iters"] for s in res.stats)
    ms32 = sum(s["time_ms"] for s in last.stats)
    F32 = [s["objective"] for s in last.stats]
    Fp = [s["objective"] for s in res.stats]
    out = {"ms_per_path": ms, "iters_per_s": iters / (ms / 1e3), "inner_iters": iters,
           "outer_iters": sum(s["outer_iters"] for s in res.stats),
           "fp64_passes": sum(s["fp64_passes"] for s in res.stats),
           "converged": res.status == g.GLAM_OK, "max_kkt": max(s["kkt"] for s in res.stats),
           "fp32_ms_per_path": ms32, "max_rel_objective_diff_vs_fp32": max(abs(x - y) / abs(y) for x, y in zip(Fp, F32))}
    if fp64:
        out["path_speedup_fp32_over_fp64"] = ms / ms32
    else:
        out["speedup_vs_fp32_path"] = ms32 / ms
    if kernel_bytes is not None and theta is not None:
        q = g.glam_quad_build(plan, X, theta, Y, W)
        k = g.glam_time_inner_kernels(plan, X, q, reps=100)
        t_f = k[0] / 1e3
        out["inner_iteration_ms"] = {"fused_slab": k[0], "mode3_adjoint": k[2], "prox": k[3], "sum": sum(k)}
        out["roofline"] = {"bound": "hbm", "kernel": "fused_slab_umma_kernel<16,bf16> (tcgen05 kind::f16, V in BF16)",
                           "achieved": kernel_bytes / t_f / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": kernel_bytes / t_f / 1e9 / peaks["hbm_gbs"], "traffic": NCU_TRAFFIC_BYTES["bf16"],
                           "bytes_per_launch": kernel_bytes, "ms_per_launch": k[0], "peak_src": src}
    plan.close()
    return out


def measure_config3(g, torch, flush):
    """The 96x96x365 Poisson workload (log-rate in [-2, 4], 10% of cells masked, p = (30, 30, 40)),
    its 30-lambda path to KKT 1e-6 with each plan precision, timed after a warm-up path."""
    import gen
    pr = gen.make_workload(2)
    f = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    pen = f(pr.pen_w, torch.float64)
    opts = g.glam_opts_default(tol=1e-6, lambda_min_ratio=pr.lambda_min_ratio)
    out = {"workload": "poisson-96x96x365 p=(30,30,40) 10% masked, 30-lambda path, ratio 1e-3, KKT 1e-6"}
    ref = None
    for name, prec in (("fp64", g.GLAM_FP64), ("fp32", g.GLAM_FP32), ("tf32", g.GLAM_TF32), ("bf16", g.GLAM_BF16)):
        dt = torch.float64 if prec == g.GLAM_FP64 else torch.float32
        X = [f(x, dt) for x in pr.XT]
        Y, W = f(pr.Y, dt), f(pr.W, dt)
        plan = g.Plan(pr.n, pr.p, pr.family, prec)
        r = g.glam_fit_path(plan, X, Y, W, pen, nlambda=pr.nlambda, opts=opts)  # warm-up
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = g.glam_fit_path(plan, X, Y, W, pen, nlambda=pr.nlambda, opts=opts)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        Fs = [s["objective"] for s in r.stats]
        if ref is None:
            ref = Fs
        out[name] = {"ms_per_path": ms, "inner_iters": sum(s["inner_iters"] for s in r.stats),
                     "outer_iters": sum(s["outer_iters"] for s in r.stats),
                     "converged": r.status == g.GLAM_OK, "max_kkt": max(s["kkt"] for s in r.stats),
                     "max_rel_objective_diff_vs_fp64": max(abs(x - y) / abs(y) for x, y in zip(Fs, ref))}
        plan.close()
    for name in ("fp32", "tf32", "bf16"):
        out[name]["speedup_vs_fp64_path"] = out["fp64"]["ms_per_path"] / out[name]["ms_per_path"]
    return out


def measure_tf32(g, torch, pr, X, Y, W, pen, opts, flush, last, theta, by, peaks, src):
    """The mixed-precision form: the same 50-lambda path with a GLAM_TF32 plan (the bottleneck
    product on the tensor cores), timed like a bench step, against the FP32 path at the same KKT
    tolerance; plus the HBM roofline of the tensor-core kernel."""
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_TF32)
    r = g.glam_fit_path(plan, X, Y, W, pen, nlambda=pr.nlambda, opts=opts)  # warm-up
    times, res = [], None
    for _ in range(2):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = g.glam_fit_path(plan, X, Y, W, pen, nlambda=pr.nlambda, opts=opts)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ms = min(times)
    iters = sum(s["inner_iters"] for s in res.stats)
    ms32 = sum(s["time_ms"] for s in last.stats)
    q = g.glam_quad_build(plan, X, theta, Y, W)
    k = g.glam_time_inner_kernels(plan, X, q, reps=100)
    t_f = k[0] / 1e3
    F32 = [s["objective"] for s in last.stats]
    Ftf = [s["objective"] for s in res.stats]
    out = {"iters_per_s": iters / (ms / 1e3), "ms_per_path": ms, "inner_iters": iters,
           "fp32_ms_per_path": ms32, "speedup_vs_fp32_path": ms32 / ms,
           "converged": res.status == g.GLAM_OK, "max_kkt": max(s["kkt"] for s in res.stats),
           "max_rel_objective_diff_vs_fp32": max(abs(a - b) / abs(b) for a, b in zip(Ftf, F32)),
           "outer_iters": sum(s["outer_iters"] for s in res.stats),
           "inner_iteration_ms": {"fused_slab_tc": k[0], "mode3_adjoint": k[2], "prox": k[3],
                                  "sum": sum(k)},
           "roofline": {"bound": "hbm", "kernel": "fused_slab_umma_kernel<1,float> (TF32 tcgen05)",
                        "achieved": by / t_f / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": by / t_f / 1e9 / peaks["hbm_gbs"], "traffic": NCU_TRAFFIC_BYTES["tf32"],
                        "bytes_per_launch": by, "ms_per_launch": k[0], "peak_src": src}}
    plan.close()
    return out


def measure_kron(g, torch, pr, X, Y, W, pen, opts, flush, last):
    """The tensor-product-weight form of the inner loop (iwls kron, Sec. 6.2): W = 1 here, so
    X^T W X = (x)_j X_j^T X_j exactly and every inner iteration works on p-sized arrays.  The
    same 50-lambda path with an FP32 plan, timed like a bench step, against the exact-weight FP32
    path at the same KKT tolerance."""
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP32)
    ko = g.GlamOpts.from_buffer_copy(opts)
    ko.iwls = g.GLAM_IWLS_KRON
    g.glam_fit_path(plan, X, Y, W, pen, nlambda=pr.nlambda, opts=ko)  # warm-up
    times, res = [], None
    for _ in range(2):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = g.glam_fit_path(plan, X, Y, W, pen, nlambda=pr.nlambda, opts=ko)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ms = min(times)
    iters = sum(s["inner_iters"] for s in res.stats)
    ms32 = sum(s["time_ms"] for s in last.stats)
    F32 = [s["objective"] for s in last.stats]
    Fk = [s["objective"] for s in res.stats]
    out = {"ms_per_path": ms, "inner_iters": iters, "inner_iters_per_s": iters / (ms / 1e3),
           "exact_fp32_ms_per_path": ms32, "speedup_vs_exact_path": ms32 / ms,
           "converged": res.status == g.GLAM_OK, "max_kkt": max(s["kkt"] for s in res.stats),
           "max_rel_objective_diff_vs_exact": max(abs(a - b) / abs(b) for a, b in zip(Fk, F32)),
           "outer_iters": sum(s["outer_iters"] for s in res.stats),
           "fp64_passes": sum(s["fp64_passes"] for s in res.stats),
           "form": "inner product H(<X_j^T X_j>, d) on p-sized arrays; FP64 gradient and KKT per outer iteration"}
    plan.close()
    return out


def measure_banded(g, torch, pr, X, Y, W, pen, opts, flush, last):
    """The banded specialisation of the FP64 gradient passes (glam_opts.exploit_bands: the cubic
    B-spline designs have 4 consecutive nonzeros per row; not the paper's general method, so it
    is reported beside the headline, not in it): the same 50-lambda FP32 path, timed like a bench
    step, against the dense-pass path."""
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP32)
    bo = g.GlamOpts.from_buffer_copy(opts)
    bo.exploit_bands = 1
    g.glam_fit_path(plan, X, Y, W, pen, nlambda=pr.nlambda, opts=bo)  # warm-up
    times, res = [], None
    for _ in range(2):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = g.glam_fit_path(plan, X, Y, W, pen, nlambda=pr.nlambda, opts=bo)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ms = min(times)
    ms32 = sum(s["time_ms"] for s in last.stats)
    F32 = [s["objective"] for s in last.stats]
    Fb = [s["objective"] for s in res.stats]
    out = {"ms_per_path": ms, "dense_pass_ms_per_path": ms32, "speedup_vs_dense_passes": ms32 / ms,
           "inner_iters": sum(s["inner_iters"] for s in res.stats),
           "fp64_passes": sum(s["fp64_passes"] for s in res.stats),
           "converged": res.status == g.GLAM_OK, "max_kkt": max(s["kkt"] for s in res.stats),
           "max_rel_objective_diff_vs_dense": max(abs(a - b) / abs(b) for a, b in zip(Fb, F32)),
           "form": "FP64 H and G of every outer iteration as banded mode products (4 terms per output)"}
    plan.close()
    return out


def measure_e2e(g, torch, pr, plan, opts, dev, steps):
    """The same metric through the public API with pinned host buffers: every step copies
    X, Y, W and the penalty weights to the device and the path back to the host."""
    hX = [torch.tensor(x, dtype=torch.float32).pin_memory() for x in pr.XT]
    hY = torch.tensor(pr.Y, dtype=torch.float32).pin_memory()
    hW = torch.tensor(pr.W, dtype=torch.float32).pin_memory()
    hP = torch.tensor(pr.pen_w, dtype=torch.float64).pin_memory()
    hout = torch.empty((pr.nlambda,) + tuple(pr.pen_w.shape), dtype=torch.float64).pin_memory()
    dX = [torch.empty_like(x, device=dev) for x in hX]
    dY, dW, dP = torch.empty_like(hY, device=dev), torch.empty_like(hW, device=dev), torch.empty_like(hP, device=dev)
    h2d = sum(x.numel() * 4 for x in hX) + hY.numel() * 4 + hW.numel() * 4 + hP.numel() * 8
    d2h = hout.numel() * 8
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters = 0
    for _ in range(steps):
        for a, b in zip(dX, hX):
            a.copy_(b, non_blocking=True)
        dY.copy_(hY, non_blocking=True)
        dW.copy_(hW, non_blocking=True)
        dP.copy_(hP, non_blocking=True)
        r = g.glam_fit_path(plan, dX, dY, dW, dP, nlambda=pr.nlambda, opts=opts)
        hout.copy_(r.path, non_blocking=True)
        torch.cuda.synchronize()
        iters += sum(s["inner_iters"] for s in r.stats)
    t = time.perf_counter() - t0
    return {"value": iters / t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


def measure_batched(g, torch, nfit, nbase):
    """The 64-fit workload (grid sides U{32..96}, p_j U{8..24}, Gaussian or Poisson, 20-lambda
    paths to KKT 1e-6, FP32 plans) through glam_fit_path_batched, against the plain FP32 path fitting
    the first nbase of the same problems one after another.  Throughput in fits/s and in inner PG
    iterations/s (the sequential leg covers a subset, so the speedup is taken on iterations/s).
    The mixed-precision leg fits the same 64 problems on TF32 plans to the same KKT tolerance and
    reports its wall time against the FP32 batch."""
    import gen
    probs = gen.make_workload(4, nfit=nfit)
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    bps = [g.BatchProblem(g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP32), [f32(x) for x in pr.XT], f32(pr.Y),
                          f32(pr.W), torch.tensor(pr.pen_w, dtype=torch.float64, device="cuda"),
                          nlambda=pr.nlambda) for pr in probs]
    opts = g.glam_opts_default(tol=1e-6, lambda_min_ratio=1e-3)

    def run(items, threads):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = g.glam_fit_path_batched(items, opts=opts, max_threads=threads)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        its = sum(sum(st["inner_iters"] for st in r.stats) for r in res)
        kkt = max(max(st["kkt"] for st in r.stats) for r in res)
        ok = all(r.status == g.GLAM_OK for r in res)
        return dt, its, kkt, ok

    dt_b, it_b, kkt_b, ok_b = run(bps, 16)
    nb = max(1, min(nbase, nfit))
    dt_s, it_s, kkt_s, ok_s = run(bps[:nb], 1)
    # the mixed-precision batch: the same fits with TF32 plans (TF32 inner products, FP64 gradient
    # and KKT test), at the same KKT tolerance
    bpt = [g.BatchProblem(g.Plan(pr.n, pr.p, pr.family, g.GLAM_TF32), bp.X, bp.Y, bp.W, bp.pen_w,
                          nlambda=pr.nlambda) for pr, bp in zip(probs, bps)]
    dt_t, it_t, kkt_t, ok_t = run(bpt, 16)
    for bp in bpt + bps:
        bp.plan.close()
    return {"fits": nfit, "nlambda": probs[0].nlambda, "threads": 16, "wall_s": dt_b,
            "fits_per_s": nfit / dt_b, "inner_iters": it_b, "inner_iters_per_s": it_b / dt_b,
            "max_kkt": kkt_b, "converged": ok_b,
            "sequential_fp32_path": {"fits": nb, "wall_s": dt_s, "fits_per_s": nb / dt_s,
                                     "inner_iters_per_s": it_s / dt_s, "max_kkt": kkt_s, "converged": ok_s},
            "speedup_iters_per_s": (it_b / dt_b) / (it_s / dt_s),
            "mixed_precision_tf32_batch": {"fits": nfit, "wall_s": dt_t, "fits_per_s": nfit / dt_t,
                                           "inner_iters": it_t, "max_kkt": kkt_t, "converged": ok_t,
                                           "speedup_vs_fp32_batch_at_equal_kkt": dt_b / dt_t,
                                           "note": "no fit of this workload meets the tensor-core kernels' "
                                                   "shape rules (n1 a multiple of 4 up to 128, n2 a multiple "
                                                   "of 32, p1, p2 <= 32), so TF32 plans run the same FP32 "
                                                   "CUDA-core kernels as FP32 plans here"},
            "form": "each fit on its own plan and stream, 16 native host worker threads"}


def run_kernels(reps, precision="fp32"):
    """Diagnostic mode for profilers: build the 128x128x600 plan and launch the four kernels of
    one inner iteration 2 + reps times each (glam_time_inner_kernels); prints their mean times.
    It produces no bench line."""
    import torch
    import gen
    import paper_1510_03298_gb300 as g
    from paper_1510_03298_gb300 import build as gb
    if not os.path.exists(g.library_path()):
        gb.build()
    pr = gen.make_workload(1)
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    plan = g.Plan(pr.n, pr.p, pr.family, {"tf32": g.GLAM_TF32, "bf16": g.GLAM_BF16}.get(precision, g.GLAM_FP32))
    X = [f32(x) for x in pr.XT]
    theta = f32(0.01 * np.random.default_rng(0).standard_normal((pr.p[2], pr.p[1], pr.p[0])))
    q = g.glam_quad_build(plan, X, theta, f32(pr.Y), f32(pr.W))
    ms = g.glam_time_inner_kernels(plan, X, q, reps=reps)
    torch.cuda.synchronize()
    print(json.dumps({"kernels_ms": dict(zip(["fused_slab", "mode3", "mode3_adjoint", "prox"], ms))}))
    return 0


def run_predict(reps):
    """Diagnostic mode for profilers: glam_predict (the H-transform) on the 128x128x600 workload
    with an FP32 plan, reps times; prints the mean time per call.  It produces no bench line."""
    import torch
    import gen
    import paper_1510_03298_gb300 as g
    from paper_1510_03298_gb300 import build as gb
    if not os.path.exists(g.library_path()):
        gb.build()
    pr = gen.make_workload(1)
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP32)
    X = [f32(x) for x in pr.XT]
    theta = f32(np.random.default_rng(0).standard_normal((pr.p[2], pr.p[1], pr.p[0])))
    eta = torch.empty((pr.n[2], pr.n[1], pr.n[0]), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        g.glam_predict(plan, X, theta, eta)
    torch.cuda.synchronize()
    print(json.dumps({"predict_ms_per_call": (time.perf_counter() - t0) * 1e3 / reps}))
    return 0


def run_oracle_rate(iters):
    """Helper of the single-core CPU baseline (run in a child process with one BLAS thread)."""
    O, d, lmax, w, z, Lhat = _oracle_setup()
    n_it, t = _oracle_iters(O, d, lmax, w, z, Lhat, iters)
    print(json.dumps({"value": n_it / t, "unit": UNIT, "iters": n_it, "seconds": t}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline leg")
    ap.add_argument("--batched", type=int, default=64, metavar="NFIT",
                    help="fits of the batched-path measurement (0: skip it)")
    ap.add_argument("--batched-baseline", type=int, default=8, metavar="NFIT",
                    help="fits of its sequential plain-FP32-path baseline")
    ap.add_argument("--kernels", type=int, default=0, metavar="REPS",
                    help="diagnostic: launch the inner-iteration kernels REPS times for a profiler")
    ap.add_argument("--kernels-precision", choices=["fp32", "tf32", "bf16"], default="fp32",
                    help="plan precision of the --kernels diagnostic")
    ap.add_argument("--predict", type=int, default=0, metavar="REPS",
                    help="diagnostic: run glam_predict REPS times for a profiler")
    ap.add_argument("--oracle-rate", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--no-config3", action="store_true", help="skip the 96x96x365 Poisson paths")
    args = ap.parse_args()
    if args.oracle_rate > 0:
        return run_oracle_rate(args.oracle_rate)
    if args.predict > 0:
        return run_predict(args.predict)
    if args.kernels > 0:
        return run_kernels(args.kernels, args.kernels_precision)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
