"""Benchmark: Nystrom-preconditioned matrix-free NGD steps/s on one GB300 (or N replicas).

Workload: the 5-D Poisson PINN (MLP 5-64-64-64-1, p = 8769, 4000 interior + 1000 boundary
points, FP32 activations and Jacobian, FP64 CG reductions, ell = 500, mu = 1e-7, PCG rtol 1e-6),
synthetic Monte-Carlo points drawn from a fixed seed.  One step = one ngd_step: gradient and
Jacobian, Gaussian test matrix, sketch, Nystrom factor, preconditioned CG, Armijo, update.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--sketch f64|df|f32|tf32|bf16]

--sketch f64 (default) forms the sketch in FP64-accurate arithmetic on the tensor cores (exact
sums of BF16 digit-plane products of the FP32 Jacobian) and the Nystrom factor in double-float;
df forms the same FP64-accurate sketch in double-float on the FP32 pipes; f32/tf32/bf16 are the
lower-precision variants of the precision study (larger shift nu, more PCG iterations).

N > 1 runs under torchrun: every rank steps an independent replica (its own seed), with no
data-path collective; the barrier and the max-over-ranks timing use the process group.
--impl reference times the FP64 CPU oracle on the host cores for the same workload.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "poisson5d"
METRIC = "NGD steps/s at PCG rtol 1e-6"


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (read only)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# the source files each profiled kernel is compiled from (its translation unit and the headers it
# includes from the package): a committed ncu summary counts only while these are unchanged
KERNEL_SOURCES = {"k_pcg_fused": ["pcg_fused.cu", "df.cuh"]}


def kernel_source_sha(kernel: str = "k_pcg_fused"):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2505_11638_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(profile: str, kernel: str, field: str = "traffic_bytes_per_launch"):
    """DRAM bytes (per launch, or per the unit `field` names) of `kernel` from the committed ncu
    summary profiles/<profile>.md, if that summary was taken on the kernel's current sources."""
    path = os.path.join(ROOT, "profiles", f"{profile}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(field + r":\s*([0-9.eE+]+)", text)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_source_sha(kernel):
        return None
    return float(m.group(1))


# ------------------------------------------------------------------ ranks (N > 1: independent replicas)
def replica_seed(rank: int) -> int:
    """Seed offset of rank's replica: the same workload shape with its own points and theta0."""
    return rank * 1000


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest x over the ranks of the process group (x itself without one): a run's time is
    its slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_problem(seed_offset: int = 0):
    from paper_2505_11638_gb300 import inputs
    wl, thetas = inputs.make_workload(WORKLOAD, seed=seed_offset)
    return wl, wl.problems[0], thetas[0]


# ------------------------------------------------------------------ reference arm (CPU oracle)
def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


def oracle_steps(pr, theta, wl, k_max, budget_s):
    """Time up to k_max oracle NGD steps (stopping once budget_s is spent). Returns (times, infos)."""
    from oracle import solve
    times, infos = [], []
    th = theta.copy()
    for k in range(k_max):
        t0 = time.perf_counter()
        th, info = solve.ngd_step(pr, th, ell=wl.ell, mu=wl.mu, rtol=wl.rtol, maxit=1000, seed=0, step=k,
                                  mant_bits=52)
        times.append(time.perf_counter() - t0)
        infos.append(info)
        if sum(times) > budget_s:
            break
    return times, infos


def oracle_cost_model(pr, theta, wl, pcg_iters=40):
    """The FP64 oracle's cost of one NGD step on the full workload, split into the part outside
    pCG (gradient and Jacobian, test matrix, sketch, Nystrom factor, Armijo) and the cost of one
    pCG iteration (matvec with the explicit G, preconditioner apply, vector updates).
    Returns (t_fixed_s, t_iter_s, pcg_iters)."""
    from oracle import gramian, nystrom, solve
    t0 = time.perf_counter()
    _, _, parts = solve.ngd_step(pr, theta, ell=wl.ell, mu=wl.mu, rtol=0.0, maxit=1, seed=0, step=0,
                                 mant_bits=52, return_parts=True)
    t_step1 = time.perf_counter() - t0
    J, U, lam, g = parts["J"], parts["U"], parts["lam"], parts["g"]
    mu = wl.mu
    t0 = time.perf_counter()
    solve.pcg(lambda v: gramian.gramian_mv(J, pr.w, v, mu), g, lambda v: nystrom.precond_apply(U, lam, mu, v),
              0.0, pcg_iters)
    t_iter = (time.perf_counter() - t0) / pcg_iters
    return max(t_step1 - t_iter, 0.0), t_iter, pcg_iters


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    wl, pr, theta = make_problem()
    budget = float(os.environ.get("NGD_REF_BUDGET_S", "150"))
    _, _ = oracle_steps(pr, theta, wl, 0, budget)          # imports outside the timed loop
    times, infos = oracle_steps(pr, theta, wl, args.steps, budget)
    t = float(np.mean(times))
    value = 1.0 / t
    sample = (f"{len(times)} of the requested {args.steps} FP64 oracle NGD steps on the full workload "
              f"(time budget {budget:.0f} s); mean PCG iterations {np.mean([i.pcg_iters for i in infos]):.1f}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": len(times), "warmup": 0, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": pr.n, "p": pr.p, "ell": wl.ell, "mu": wl.mu, "rtol": wl.rtol},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2505_11638_gb300 import build, ngd

    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    build.build()
    ngd.lib()
    wl, pr, theta0 = make_problem(seed_offset=replica_seed(rank))
    ctx = ngd.Context(pr, dtype=wl.dtype)
    opts = dict(ell=wl.ell, mu=wl.mu, rtol=wl.rtol, maxit=1000, sketch=args.sketch, seed=rank)
    theta = torch.tensor(theta0, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    # warm-up (also builds every lazily sized workspace)
    for k in range(args.warmup):
        ctx.step(theta, step=k, **opts)
    theta.copy_(torch.tensor(theta0, device="cuda"))

    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    l0 = ngd.ngd_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    torch.cuda.nvtx.range_push("timed")     # lets a profiler select the timed steps
    e0.record(stream)
    for k in range(args.steps):
        infos.append(ctx.step(theta, step=k, **opts))
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = ngd.ngd_kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, dist)
    ms_per_step = ms_max / args.steps
    value = world * 1e3 / ms_per_step

    # end to end through the public API with host buffers, over the same K steps from the same
    # theta0: every step copies theta in from pinned host memory and theta and the loss back out
    h_theta = torch.tensor(theta0).pin_memory()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = args.steps
    for k in range(e2e_steps):
        theta.copy_(h_theta, non_blocking=True)
        info = ctx.step(theta, step=k, **opts)
        h_theta.copy_(theta, non_blocking=True)
        torch.cuda.synchronize()
        _ = info["loss_after"]
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist)
    barrier()

    # The Gramian matvec alone (ngd_gramian_mv: k_pcg_fused in matvec mode), timed on the context stream
    v = torch.randn(pr.p, dtype=torch.float64, device="cuda")
    ctx.gramian_mv(theta, v, wl.mu)
    y = torch.empty_like(v)
    reps = 200
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(5):
        ngd.ngd_gramian_mv(ctx.handle, None, v, wl.mu, y)
    torch.cuda.nvtx.range_push("gramian_mv")   # lets a profiler select these launches
    ev0.record(stream)
    for _ in range(reps):
        ngd.ngd_gramian_mv(ctx.handle, None, v, wl.mu, y)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    gv_ms = ev0.elapsed_time(ev1) / reps
    ldJ = (pr.p + 31) // 32 * 32
    j_bytes = float(pr.n * ldJ * (4 if wl.dtype == "f32" else 8))

    # Roofline of the dominant kernel, k_pcg_fused (the whole preconditioned CG in one launch), per
    # CG iteration: PCG at the final theta with a fresh Nystrom factor, rtol 0 and two fixed
    # iteration counts; the difference cancels the per-solve setup.  Algorithmic DRAM bytes per
    # iteration: one read of J plus ~12 p-vectors of float64 (U, 2 p l 8 bytes, is read from L2).
    g_fin, _, _ = ctx.gradient(theta)
    Om_f, Y_f = ctx.nystrom_sketch(None, wl.ell, seed=rank, step=10 ** 6, prec=args.sketch)
    U_f, lam_f, _ = ctx.nystrom_factor(wl.ell, Om_f, Y_f, args.sketch)

    def pcg_ms(k):
        ctx.pcg_solve(None, g_fin, wl.mu, U_f, lam_f, wl.ell, rtol=0.0, maxit=k)
        torch.cuda.synchronize()
        ev0.record(stream)
        _, it, _ = ctx.pcg_solve(None, g_fin, wl.mu, U_f, lam_f, wl.ell, rtol=0.0, maxit=k)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), it

    t_lo, k_lo = pcg_ms(20)
    t_hi, k_hi = pcg_ms(220)
    us_it = (t_hi - t_lo) / max(k_hi - k_lo, 1) * 1e3
    bytes_it = j_bytes + 12.0 * pr.p * 8
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak = hbm if hbm else 6800.0
    achieved = bytes_it / (us_it * 1e-6) / 1e9
    roofline = {"kernel": "k_pcg_fused (whole PCG, one launch); unit: one CG iteration", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs, burst)" if hbm else "fallback 6.8 TB/s",
                "traffic": profiled_traffic("k_pcg_fused_poisson5d", "k_pcg_fused", "traffic_bytes_per_iteration"),
                "bytes_per_iteration": bytes_it,
                "us_per_iteration": us_it,
                "matvec": {"kernel": "k_pcg_fused, matvec mode (ngd_gramian_mv)", "us": gv_ms * 1e3,
                           "bytes": j_bytes, "GB/s": j_bytes / (gv_ms * 1e-3) / 1e9}}

    phases = {k: float(np.mean([i[k] for i in infos])) for k in
              ["ms_linearize", "ms_sketch", "ms_factor", "ms_pcg", "ms_linesearch"]}
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": pr.n, "p": pr.p, "ell": wl.ell, "mu": wl.mu, "rtol": wl.rtol,
                       "sketch": args.sketch, "maxit": 1000,
                       "l2": "inputs larger than L2: the FP32 Jacobian streamed by every matvec is 176 MB"},
            "gramian_mv_per_s": 1e3 / gv_ms * world,
            "pcg_iters_mean": float(np.mean([i["pcg_iters"] for i in infos])),
            "shift_retries_total": int(sum(i["shift_retries"] for i in infos)),
            "loss_first_last": [infos[0]["loss_before"], infos[-1]["loss_after"]],
            "phases_ms": phases,
            "e2e": {"value": world / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": pr.p * 8,
                    "d2h_bytes_per_step": pr.p * 8 + 8},
            "gpu_launches": int(launches), "roofline": roofline, "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's cost per step outside pCG plus its cost per pCG iteration, evaluated at the
        # pCG iteration count of the steps timed above (the same trajectory on both sides)
        t_fixed, t_iter, k_meas = oracle_cost_model(pr, theta0, wl)
        iters = line["pcg_iters_mean"]
        t_step = t_fixed + iters * t_iter
        line["cpu_baseline"] = {"value": 1.0 / t_step, "unit": "steps/s", "cores": cpu_threads(), "kind": "oracle",
                                "sample": f"FP64 oracle on the full workload at theta0: {t_fixed:.3f} s per step "
                                          f"outside pCG (one step timed) + {1e3 * t_iter:.2f} ms per pCG iteration "
                                          f"({k_meas} iterations timed), evaluated at {iters:.1f} pCG iterations "
                                          f"per step (this run's timed steps)",
                                "s_per_step_outside_pcg": t_fixed, "s_per_pcg_iteration": t_iter}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch(args, rank, world, local_rank):
    """The batching form: every step is one ngd_batch_step over the 64 problems of batch64."""
    import torch
    from paper_2505_11638_gb300 import build, inputs, ngd

    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    build.build()
    wl, thetas0 = inputs.make_workload("batch64", seed=replica_seed(rank))
    batch = ngd.Batch(wl.problems, dtype=wl.dtype)
    opts = dict(ell=wl.ell, mu=None, rtol=wl.rtol, maxit=1000, sketch=args.sketch, seed=rank)
    thetas = [torch.tensor(th, device="cuda") for th in thetas0]
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    if args.packing is not None:
        batch.set_packing(args.packing)
    for k in range(args.warmup):             # the first step also tunes the packing of the solves
        batch.step(thetas, step=k, **opts)
    for th, th0 in zip(thetas, thetas0):
        th.copy_(torch.tensor(th0, device="cuda"))
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    l0 = ngd.ngd_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for k in range(args.steps):
        infos.append(batch.step(thetas, step=k, **opts))
    e1.record(stream)
    barrier()
    launches = ngd.ngd_kernel_launches() - l0
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    n_prob = len(wl.problems)
    value = world * args.steps * n_prob / (ms * 1e-3)
    iters = [i["pcg_iters"] for step in infos for i in step]
    line = {"metric": "NGD problem-steps/s at PCG rtol 1e-6 (batching form)", "value": value,
            "unit": "problem-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64", "problems": n_prob, "N_total": int(sum(pr.n for pr in wl.problems)),
                       "p_each": wl.problems[0].p, "ell": wl.ell, "mu": "rule", "rtol": wl.rtol,
                       "sketch": args.sketch},
            "pcg_iters_mean": float(np.mean(iters)), "pcg_iters_max": int(np.max(iters)),
            "solves_per_launch": batch.packing, "solve_launches_per_step": batch.solve_launches,
            "shift_retries_total": int(sum(i["shift_retries"] for step in infos for i in step)),
            "gpu_launches": int(launches), "gpu_launches_per_step": int(launches) / args.steps, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_precision_study(args, rank):
    """Precision form (10-D Poisson, p = 51073, N = 20480, ell = 1000): the same NGD steps from the
    same theta0 with the sketch in FP64 (FP64 context), FP64-accurate on the tensor cores (digit
    planes of the FP32 Jacobian), FP64-accurate double-float (FP32 pipes), TF32 and BF16 (tcgen05,
    rounded operands, FP32 accumulation).  Damping of Sec. 5, mu = max(gamma eps lambda_1,
    1e-4 L^2), so that every form can reach the common PCG tolerance rtol = 1e-6 (maxit 3000).
    Reported per form: time per step and per phase, PCG iterations and final residuals, loss,
    relative L2 error of u_theta on 4096 independent points, and the sketch product Y = G V alone
    (ngd_gramian_mm on a fixed V at the final theta, CUDA events): its time and rate."""
    import torch
    from paper_2505_11638_gb300 import build, inputs, ngd

    if rank != 0:
        return 0
    build.build()
    wl, thetas = inputs.make_workload("poisson10d", seed=0)
    pr = wl.problems[0]
    xe = inputs.eval_points(pr, 4096, seed=0)
    ue = inputs.u_star(pr, xe)
    ev = inputs.Problem(name="eval", pde=pr.pde, widths=pr.widths, X=xe, w=np.full(len(xe), 1.0 / len(xe)),
                        target=ue, n_int=0, n_bnd=len(xe), freq=pr.freq)
    peaks = measured_peaks()
    bf16_peak = peaks.get("bf16_tflops", 1881.0)
    prod_flop = 4.0 * pr.n * pr.p * wl.ell           # the two products of the sketch, as FP64-accurate work
    forms = [("fp64", "f64", "f64"), ("fp64-accurate tensor cores", "f32", "f64"), ("double-float", "f32", "df"),
             ("tf32", "f32", "tf32"), ("bf16", "f32", "bf16")]
    stream = torch.cuda.current_stream()
    out = {}
    for name, dtype, sketch in forms:
        ctx = ngd.Context(pr, dtype=dtype)
        ectx = ngd.Context(ev, dtype="f64")
        theta = torch.tensor(thetas[0], device="cuda")
        infos = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(args.steps):
            infos.append(ctx.step(theta, ell=wl.ell, mu=None, mu_loss_coef=1e-4, rtol=1e-6, maxit=3000, seed=0,
                                  step=k, sketch=sketch))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        r, _ = ectx.residual(theta)
        l2 = float(torch.linalg.norm(r).item() / np.linalg.norm(ue))
        # the sketch product alone on a fixed V
        wd = torch.float64 if dtype == "f64" else torch.float32
        V = torch.randn(wl.ell, pr.p, generator=torch.Generator(device="cuda").manual_seed(5), device="cuda",
                        dtype=torch.float64).to(wd)
        ctx.gramian_mm(theta, V, sketch)               # linearize; digit planes of J made
        reps = 1 if dtype == "f64" else 3
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            ctx.gramian_mm(None, V, sketch)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_prod = e0.elapsed_time(e1) / reps
        entry = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "pcg_iters": [i["pcg_iters"] for i in infos],
                 "relres": [i["relres"] for i in infos], "shift_retries": [i["shift_retries"] for i in infos],
                 "mu": [i["mu"] for i in infos], "loss": infos[-1]["loss_after"], "rel_l2_error": l2,
                 "ms_sketch": float(np.mean([i["ms_sketch"] for i in infos])),
                 "ms_factor": float(np.mean([i["ms_factor"] for i in infos])),
                 "ms_pcg": float(np.mean([i["ms_pcg"] for i in infos])),
                 "ms_product": ms_prod, "product_tflops": prod_flop / (ms_prod * 1e-3) / 1e12}
        if sketch in ("tf32", "bf16"):
            peak = bf16_peak * (0.5 if sketch == "tf32" else 1.0)
            entry["product_roofline"] = {"bound": "tensor", "achieved": entry["product_tflops"], "peak": peak,
                                         "unit": "TFLOP/s", "frac": entry["product_tflops"] / peak,
                                         "peak_source": "measured BF16 (x 1/2 for TF32, nominal ratio)",
                                         "note": "includes the operand copies (transpose, BF16 rounding)"}
        out[name] = entry
        ctx.close()
        ectx.close()
        del theta, V
        torch.cuda.empty_cache()
    line = {"metric": "precision form: NGD steps/s, PCG iterations and L2 error per sketch precision",
            "config": {"workload": "poisson10d", "N": pr.n, "p": pr.p, "ell": wl.ell,
                       "mu": "max(10 eps lambda_1, 1e-4 L^2) (Sec. 5)", "rtol": 1e-6, "maxit": 3000,
                       "steps": args.steps}, "data": "synthetic", "forms": out}
    print(json.dumps(line), flush=True)
    return 0


def run_sketch_product(args, rank):
    """The sketch product Y = G V (ngd_gramian_mm) alone on the 5-D Poisson workload (N = 5000,
    p = 8769, ell = 500, FP32 Jacobian) in the precision --sketch: --warmup products, then --steps
    timed with CUDA events.  Rates: FP64-accurate work 4 N p ell flop per product, and for the
    digit-plane form the BF16 tensor-core flops it issues (the kept digit-plane pairs of both
    GEMMs on the padded tiles)."""
    import torch
    from paper_2505_11638_gb300 import build, ngd

    if rank != 0:
        return 0
    build.build()
    wl, pr, theta0 = make_problem()
    ctx = ngd.Context(pr, dtype="f32")
    theta = torch.tensor(theta0, device="cuda")
    V = torch.randn(wl.ell, pr.p, generator=torch.Generator(device="cuda").manual_seed(5), device="cuda",
                    dtype=torch.float32)
    ctx.gramian_mm(theta, V, args.sketch)
    for _ in range(args.warmup):
        ctx.gramian_mm(None, V, args.sketch)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ctx.gramian_mm(None, V, args.sketch)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    flop = 4.0 * pr.n * pr.p * wl.ell
    line = {"metric": "sketch product Y = G V per second", "value": 1e3 / ms, "unit": "products/s", "ms": ms,
            "sketch": args.sketch, "fp64_accurate_tflops": flop / (ms * 1e-3) / 1e12,
            "config": {"workload": WORKLOAD, "N": pr.n, "p": pr.p, "ell": wl.ell}}
    if args.sketch == "f64":
        ldj = (pr.p + 31) // 32 * 32
        pairs1, pairs2 = 19, 20                          # kept digit-plane pairs of Z = J V and Y = J^T Z
        m1, n1, k1 = -(-pr.n // 128) * 128, -(-wl.ell // 96) * 96, -(-ldj // 256) * 256
        m2, k2 = -(-pr.p // 128) * 128, -(-(-(-pr.n // 32) * 32) // 256) * 256
        issued = 2.0 * (pairs1 * m1 * n1 * k1 + pairs2 * m2 * n1 * k2)
        line["tensor_tflops_issued"] = issued / (ms * 1e-3) / 1e12
        line["tensor_peak_tflops"] = measured_peaks().get("bf16_tflops", 1881.0)
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_matvec_study(args, rank):
    """Gramian matvecs/s: (G + mu I) v through ngd_gramian_mv at the current linearization, in FP32
    contexts on the 5-D Poisson (p = 8769), 10-D Poisson (p = 51073) and 4-D heat (p = 133121)
    workloads, with J stored (one fused pass over J when p <= 9216, else a row pass and a column
    pass) or matrix-free (J v by forward tangents, then J^T (w .* J v) from Jacobian row blocks of
    about 64 MB recomputed and reduced while they sit in L2).  CUDA events around --steps products
    after --warmup; the stored form is reported against the measured HBM copy bandwidth with its
    algorithmic bytes (the passes over the N x ldJ FP32 Jacobian)."""
    import torch
    from paper_2505_11638_gb300 import build, inputs, ngd

    if rank != 0:
        return 0
    build.build()
    hbm = measured_peaks().get("hbm_gbs")
    cases = [("poisson5d", "stored"), ("poisson10d", "stored"), ("poisson10d", "matrix_free"),
             ("heat4d", "stored"), ("heat4d", "matrix_free")]
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    clocks.start()
    out = []
    for name, mode in cases:
        wl, thetas = inputs.make_workload(name, seed=0)
        pr = wl.problems[0]
        mu = float(wl.mu) if isinstance(wl.mu, float) else 1e-6
        ctx = ngd.Context(pr, dtype="f32", gv_mode=mode)
        theta = torch.tensor(thetas[0], device="cuda")
        v = torch.tensor(np.random.default_rng(0).standard_normal(pr.p), device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.gramian_mv(theta, v, mu)                       # linearize (J formed, or the tape)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_linearize = e0.elapsed_time(e1)
        for _ in range(args.warmup):
            ctx.gramian_mv(None, v, mu)
        torch.cuda.synchronize()
        l0 = ngd.ngd_kernel_launches()
        e0.record(stream)
        for _ in range(args.steps):
            ctx.gramian_mv(None, v, mu)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        ldj = (pr.p + 31) // 32 * 32
        jbytes = pr.n * ldj * 4
        entry = {"workload": name, "mode": mode, "N": pr.n, "p": pr.p, "ms_per_gv": ms, "gv_per_s": 1e3 / ms,
                 "ms_first_gv_with_linearization": ms_linearize,
                 "launches_per_gv": (ngd.ngd_kernel_launches() - l0) / args.steps,
                 "jacobian_fp32_bytes": jbytes}
        if mode == "stored":
            passes = 1 if pr.p <= 9216 else 2
            gbs = passes * jbytes / (ms * 1e-3) / 1e9
            entry["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                 "frac": gbs / hbm if hbm else None, "passes_over_J": passes}
        out.append(entry)
        ctx.close()
        del theta, v
        torch.cuda.empty_cache()
    clk = clocks.stop()
    line = {"metric": "Gramian matvecs/s ((G + mu I) v, FP32 Jacobian, FP64-accurate accumulation)",
            "unit": "Gv/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "cases": out, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_train(args, rank):
    """NystromNGD training run on the paper's 3-D Poisson PINN (poisson3d: MLP 3-64-64-64-1,
    p = 8641, 10000 + 1000 points): Alg. 1 with Alg. 3 and Alg. 4, adaptive rank from 20 up to
    500 in steps of 20, damping max(gamma eps lambda_hat_1, 1e-4 L^2), pCG capped at 20
    iterations (the paper's settings for its NGD runs); --test-matrix picks the Gaussian or the
    sampling test matrix.  Reports NGD steps/s over the run (CUDA
    events around every step), the rank trajectory, and the relative L2 and H1 errors of u_theta
    against u* on 10x the training points (independent, interior), every 10 steps."""
    import torch
    from paper_2505_11638_gb300 import build, inputs, ngd

    if rank != 0:
        return 0
    build.build()
    wl, thetas = inputs.make_workload("poisson3d", seed=0)
    pr = wl.problems[0]
    ctx = ngd.Context(pr, dtype=wl.dtype)
    xe = inputs.eval_points(pr, 10 * pr.n, seed=0)
    ue, ge = inputs.u_star(pr, xe), inputs.grad_u_star(pr, xe)
    ev = inputs.Problem(name="eval", pde=pr.pde, widths=pr.widths, X=xe, w=np.full(len(xe), 1.0 / len(xe)),
                        target=ue, n_int=0, n_bnd=len(xe), freq=pr.freq)
    ectx = ngd.Context(ev, dtype="f64", gv_mode="matrix_free", mem_budget=1)
    ue_t, ge_t = torch.tensor(ue, device="cuda"), torch.tensor(ge, device="cuda")
    norm_l2 = float(torch.linalg.norm(ue_t))
    norm_h1 = float(torch.sqrt((ue_t ** 2).sum() + (ge_t ** 2).sum()))

    def errors(theta):
        out = ectx.eval(theta)
        du, dg = out[:, 0] - ue_t, out[:, 1:1 + pr.d] - ge_t
        return (float(torch.linalg.norm(du)) / norm_l2,
                float(torch.sqrt((du ** 2).sum() + (dg ** 2).sum())) / norm_h1)

    theta = torch.tensor(thetas[0], device="cuda")
    if args.precond == "full":
        # Alg. 2: the direction by Cholesky of the explicit G + mu I (no preconditioner, no pCG)
        opts = dict(mu=None, mu_loss_coef=1e-4, precond="full", sketch=args.sketch, seed=0)
    elif args.precond == "rpchol":
        # Alg. 5: rank found by block RPCholesky (20 pivots per round, at most 500), no rank rule
        opts = dict(mu=None, mu_loss_coef=1e-4, precond="rpchol", rpchol_block=20, rtol=wl.rtol, maxit=20,
                    sketch=args.sketch, seed=0)
    else:
        opts = dict(mu=None, mu_loss_coef=1e-4, ell_max=500, ell_delta=20, rtol=wl.rtol, maxit=20,
                    sketch=args.sketch, seed=0, test_matrix=args.test_matrix)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    ell, total_ms, log, ells = (500 if args.precond == "rpchol" else 1 if args.precond == "full" else wl.ell), 0.0, [], []
    l2, h1 = errors(theta)
    log.append({"step": 0, "seconds": 0.0, "ell": ell, "loss": None, "rel_l2": l2, "rel_h1": h1})
    for k in range(args.train_steps):
        e0.record(stream)
        info = ctx.step(theta, ell=ell, step=k, **opts)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        ells.append(info["ell_next"] if args.precond == "rpchol" else 0 if args.precond == "full" else ell)
        if args.precond == "nystrom":
            ell = info["ell_next"]
        if (k + 1) % 10 == 0 or k + 1 == args.train_steps:
            l2, h1 = errors(theta)
            log.append({"step": k + 1, "seconds": total_ms / 1e3, "ell": ells[-1], "loss": info["loss_after"],
                        "mu": info["mu"], "pcg_iters": info["pcg_iters"], "rel_l2": l2, "rel_h1": h1})
    line = {"metric": "NystromNGD training run: NGD steps/s, rank trajectory and relative errors",
            "value": args.train_steps / (total_ms / 1e3), "unit": "steps/s", "n_gpus": 1,
            "steps": args.train_steps, "ms_per_step": total_ms / args.train_steps, "data": "synthetic",
            "config": {"workload": "poisson3d", "N": pr.n, "p": pr.p, "ell0": wl.ell, "ell_max": 500,
                       "ell_delta": 20, "mu": "max(10 eps lambda_1, 1e-4 L^2)", "pcg_maxit": 20,
                       "sketch": args.sketch, "test_matrix": args.test_matrix, "precond": args.precond,
                       "eval_points": len(xe)},
            "final": log[-1], "ell_trajectory": ells, "log": log}
    print(json.dumps(line), flush=True)
    ctx.close()
    ectx.close()
    return 0


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sketch", default="f64", choices=["f64", "df", "f32", "tf32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--packing", type=int, default=None,
                    help="batch64: pCG solves per cooperative launch (default: tuned by the first step)")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "batch64"],
                    help="batch64: the batching form, 64 problems of uneven size per step (ngd_batch_step)")
    ap.add_argument("--train", action="store_true",
                    help="a NystromNGD training run (adaptive rank and damping) on the 3-D Poisson PINN, "
                         "--train-steps NGD steps, with L2/H1 errors every 10 steps")
    ap.add_argument("--train-steps", type=int, default=200)
    ap.add_argument("--precond", default="nystrom", choices=["nystrom", "rpchol", "full"],
                    help="direction method in --train: NystromNGD (Alg. 4), RPCholNGD (Alg. 5; the rank is the one "
                         "block RPCholesky finds, at most 500) or NGD full (Alg. 2: Cholesky of the explicit Gramian)")
    ap.add_argument("--test-matrix", default="gaussian", choices=["gaussian", "sampling"],
                    help="test matrix of the Nystrom sketch in --train (sampling: columns drawn proportionally "
                         "to diag G)")
    ap.add_argument("--sketch-product", action="store_true",
                    help="time the sketch product Y = G V alone on the bench workload (--sketch precision)")
    ap.add_argument("--matvec-study", action="store_true",
                    help="Gramian matvecs/s on the 5-D Poisson, 10-D Poisson and 4-D heat workloads, J stored "
                         "or matrix-free, --steps products each")
    ap.add_argument("--precision-study", action="store_true",
                    help="the precision form on poisson10d: all-FP64 GPU path vs FP64-accurate (double-float) "
                         "vs TF32 / BF16 tensor-core sketches, --steps NGD steps each")
    return ap


def main():
    args = build_parser().parse_args()
    rank, world, local_rank = _env_rank()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.precision_study:
        return run_precision_study(args, rank)
    if args.matvec_study:
        return run_matvec_study(args, rank)
    if args.sketch_product:
        return run_sketch_product(args, rank)
    if args.train:
        return run_train(args, rank)
    if args.workload == "batch64":
        return run_batch(args, rank, world, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
