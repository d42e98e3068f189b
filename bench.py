#!/usr/bin/env python
"""Benchmark of the IBSN hot path on the 16384-bin grid workload.

One step = one full solve (Alg. 2) from gamma = 0 to a certified relative
duality gap <= 1e-8, on 128 x 128 grid histograms (smoothed random fields,
squared grid distance / max rebuilt on the fly from bin coordinates).
value = seconds per solve (CUDA events on the solve's stream, inputs resident
in HBM).  The anchored exponent matrix (1 GiB float32 / 2 GiB float64) is
larger than L2, so no flush is needed between steps.

Also reported: the plain float64 GPU path on the same problem (speedup
denominator) with the mixed result's difference from it, one solve at the
paper's image eta = 1e-3, the plan-pass bandwidth, the roofline of the
dominant step (HBM and, for the persistent CG, latency), an end-to-end time
through the public API with host buffers, and the CPU oracle timed on real
work on this host's cores (a reported baseline only).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload grid|batch64|warmstart|eot|ablation|sphere|points]
Under torchrun each rank solves the same problem on its own GPU (replicas).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the CPU oracle baseline runs on one host core: keep numpy's BLAS single-threaded
# (set before numpy is first imported; the GPU path does not use it)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "s to rel. gap 1e-8 at m=n=16384; plan-pass HBM GB/s; speedup vs plain FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=128, help="grid side h (m = n = h*h)")
    ap.add_argument("--eta", type=float, default=1e-4)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain float64 comparison solve")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cost", default="grid", choices=["grid", "dense32"],
                    help="grid: cost rebuilt from bin coordinates; dense32: the same cost stored as a float32 matrix")
    ap.add_argument("--recompute", action="store_true",
                    help="grid: passes rebuild the anchored exponent from the cost (no stored m x n matrix)")
    ap.add_argument("--no-eta3", dest="eta3", action="store_false",
                    help="skip the extra mixed solve of the grid workload at eta = 1e-3")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--oracle-job", default="", help=argparse.SUPPRESS)
    ap.add_argument("--max-cg", type=int, default=0, help="CG iteration cap per Newton direction (0: library default)")
    ap.add_argument("--max-outer", type=int, default=0,
                    help="outer iteration cap (0: library default); a small cap gives a short profiling case")
    ap.add_argument("--nnz-cap", type=int, default=0,
                    help="nonzeros reserved for the sparsified Hessian (0: library default)")
    ap.add_argument("--ws-train", type=int, default=64, help="warmstart: training solves")
    ap.add_argument("--ws-train-n", type=int, default=256, help="warmstart: points per cloud in training")
    ap.add_argument("--ws-eval-n", type=int, default=1024, help="warmstart: points per cloud in evaluation")
    ap.add_argument("--ws-adam-steps", type=int, default=600, help="warmstart: Adam steps")
    ap.add_argument("--workload", default="grid", choices=["grid", "batch64", "warmstart", "eot", "ablation", "sphere", "points"],
                    help="grid: the 16384-bin headline; batch64: 64 uneven point-cloud problems "
                         "(m, n ~ U{500..5000}) solved by one ibsn_solve_batch call; eot: (E)IBSN on the "
                         "paper's Square EOT setting; ablation: IBSN against IBN (dense Hessian)")
    ap.add_argument("--sizes", default="", help="eot/ablation: comma-separated m = n values")
    ap.add_argument("--batch-threads", type=int, default=8)
    ap.add_argument("--sequential", action="store_true", help="batch64: also time the problems one by one")
    ap.add_argument("--verbose", type=int, default=0, help="per-outer log lines of the solver on stderr")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(",") for r in self.file.read().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus: int):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Largest x over the ranks (the slowest replica sets the step time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_line_fields(per_rank_seconds: float, world: int) -> dict:
    """Fields of the JSON line for N replicas of the same solve.  The metric is
    time per solve; every rank solves its own copy of the problem (weak
    scaling: fixed work per GPU), so the job's value is the slowest rank's
    time, and the solves completed per second are world / that time."""
    t = max_over_ranks(per_rank_seconds, world)
    return {"value": t, "n_gpus": world, "scaling": "weak", "solves_per_s": world / t if t > 0 else None}


def host_cores() -> int:
    """Cores this process may run on (the CPU baseline's all-core thread count)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def blas_threads() -> int:
    """Threads this process's oracle work may use: numpy's elementwise passes
    run on one thread, its BLAS calls on at most OPENBLAS_NUM_THREADS."""
    try:
        return max(1, int(os.environ.get("OPENBLAS_NUM_THREADS", "1")))
    except ValueError:
        return 1


def oracle_job(name: str, h: int, eta: float) -> dict:
    """Real oracle work timed on the host (runs in a child process whose BLAS
    thread count is set by its environment).

    c0:        the oracle's full solve (Alg. 2) of the 256^2 uniform-points
               workload (eta = 1e-4) to a relative gap of 1e-8.
    c2_newton: the oracle's Sinkhorn warm-up and first Newton iteration (Alg. 1
               sparsification, dense H_rho, shifted Newton system by PCG,
               Armijo on L directly, update and next plan pass) on the full
               h^2 x h^2 grid workload from gamma = 0 at k = 0; the cost matrix
               and log X^0 are built before the clock starts.
    """
    import numpy as np

    from oracle import ibsn as O
    from workloads import grid_marginals, grid_sq_cost, workload

    if name == "c0":
        p = workload("c0")
        t0 = time.perf_counter()
        r = O.ibsn(p.C, p.a, p.b, O.IBSNParams(eta=p.eta))
        return {"s": time.perf_counter() - t0, "outer": r.outer_iters, "newton": r.newton_iters,
                "cg": r.cg_iters, "rel_gap": r.rel_gap, "converged": bool(r.converged)}
    a, b, scale = grid_marginals(h, h, seed=2)
    C = grid_sq_cost(h, h) * scale
    m, n = C.shape
    prm = O.IBSNParams(eta=eta)
    logX = O.initial_log_plan(a, b)
    mu = O.mu_k(0, prm)
    parts = {}
    t_all = time.perf_counter()
    t0 = time.perf_counter()
    gamma, sk_it, _ = O.sinkhorn_warmup(logX, C, a, b, eta, np.zeros(n), prm.sinkhorn_tol, prm.max_sinkhorn)
    gamma = gamma - gamma.mean()
    parts["sinkhorn"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    P = O.plan(logX, C, eta, gamma)
    g = O.gradient(P, a, b)
    gnorm = float(np.linalg.norm(g))
    parts["plan"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Q = O.sparsify_plan(P, a, O.sparsification_threshold(eta, m, n, gnorm))
    del P
    parts["sparsify"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    H = O.sparsified_hessian(Q, a, eta)
    del Q
    parts["hessian"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    delta, cg_it = O.newton_direction(H, g, prm.cg_rtol, prm.max_cg, mu)
    del H
    parts["cg"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    t, trials, _ = O.armijo(logX, C, a, b, eta, gamma, delta, g, prm.sigma, prm.beta, prm.max_armijo)
    parts["armijo"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    gamma = gamma + t * delta
    gn_next = float(np.linalg.norm(O.gradient(np.exp(O.log_plan(logX, C, eta, gamma)), a, b)))
    parts["update"] = time.perf_counter() - t0
    return {"s": time.perf_counter() - t_all, "parts": parts, "sinkhorn_iters": sk_it, "cg_iters": cg_it,
            "armijo_trials": trials, "grad_norm": [gnorm, gn_next]}


def run_oracle_job(name: str, threads: int, h: int, eta: float, timeout: float = 1200.0) -> dict | None:
    """oracle_job in a child process with `threads` BLAS / OpenMP threads."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-job", name, "--grid", str(h), "--eta", repr(eta)]
    try:
        res = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=timeout)
        out = json.loads(res.stdout.strip().splitlines()[-1])
        out["threads"] = threads
        return out
    except Exception as e:  # the baseline is reported, never required
        return {"error": f"{type(e).__name__}: {str(e)[:200]}", "threads": threads}


def cpu_baseline(args, newton_iters: int) -> dict:
    """The oracle as it stands, timed on this host's cores: one real Newton
    iteration on the full benchmark workload with all cores, scaled by the
    Newton iterations of the GPU solve to the metric's unit (seconds per
    solve), plus the full 256^2 solve on one core and on all cores."""
    cores = host_cores()
    c2 = run_oracle_job("c2_newton", cores, args.grid, args.eta)
    c0_1 = run_oracle_job("c0", 1, args.grid, args.eta)
    c0_n = run_oracle_job("c0", cores, args.grid, args.eta) if cores > 1 else c0_1
    per_newton = c2.get("s") if c2 else None
    value = per_newton * newton_iters if per_newton else None
    m = args.grid * args.grid
    return {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": f"one real oracle Newton iteration (Sinkhorn warm-up, Alg. 1 sparsification, dense H_rho, "
                      f"PCG, Armijo, update; numpy float64, {cores} cores) on the full {m}x{m} workload, "
                      f"{per_newton if per_newton is None else round(per_newton, 2)} s, times the "
                      f"{newton_iters} Newton iterations of the GPU solve (an estimate: the oracle cannot finish "
                      f"this solve inside a benchmark run)",
            "c2_newton_iteration": c2, "c0_full_solve": {"one_core": c0_1, "all_cores": c0_n}}


def grid_config(args, world: int) -> dict:
    """The `config` of the grid workload's line (both arms)."""
    h = args.grid
    m = h * h
    return {"workload": f"grid{h}x{h} smoothed random fields ({m} bins), eta={args.eta}, "
                        + ("C = squared grid distance / max stored as a dense float32 matrix"
                           if getattr(args, "cost", "grid") == "dense32" else
                           "C = squared grid distance / max rebuilt on the fly")
                        + (", anchored exponent rebuilt in every pass (no stored matrix)" if args.recompute else ""),
            "m": m, "n": m, "eta": args.eta, "precision": args.precision, "gap_tol": 1e-8,
            "l2": "inputs larger than L2 (anchored matrix 1 GiB f32 / 2 GiB f64), no flush",
            "parallelism": f"replicas x{world}"}


TRAJECTORY = os.path.join(ROOT, "profiles", "grid_trajectory.json")


def oracle_pass_count(rec: dict) -> int:
    """Dense m x n passes the oracle's Alg. 2 makes along a solve with these
    iteration counts: per outer step the c-transform certificate, the outer
    update and the first plan pass (3), per Sinkhorn iteration a zeta- and a
    gamma-step (2), per Newton step the plan pass, L at gamma, and the plan at
    the accepted point (3), and one L evaluation per Armijo trial."""
    return 3 * rec["outer_iters"] + 2 * rec["sinkhorn_iters"] + 3 * rec["newton_iters"] + rec["armijo_trials"]


def oracle_plan_pass(a, b, C, eta) -> float:
    """One real oracle plan-and-gradient pass (Eqs. 6-7) over the full matrix; seconds."""
    import numpy as np

    from oracle import ibsn as O

    logX = O.initial_log_plan(a, b)
    t0 = time.perf_counter()
    P = O.plan(logX, C, eta, np.zeros(len(b)))
    _ = O.gradient(P, a, b)
    return time.perf_counter() - t0


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on this host's cores.  Each
    step is one real oracle plan pass (Eqs. 6-7) over the full workload; the
    value scales the mean step time by the oracle's dense passes for the
    solve's iteration counts (recorded from a GPU solve of this workload in
    profiles/grid_trajectory.json).  It leaves out the oracle's dense Hessian
    and CG work, so it understates the oracle's solve time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from workloads import grid_marginals, grid_sq_cost

    h = args.grid
    a, b, scale = grid_marginals(h, h, seed=2)
    C = grid_sq_cost(h, h) * scale
    try:
        rec = json.load(open(TRAJECTORY))[f"{h}:{args.eta:g}"]
    except Exception as e:
        print(json.dumps({"impl": "reference", "unavailable": f"no recorded trajectory for grid {h}, eta "
                                                              f"{args.eta:g} ({type(e).__name__})"}), flush=True)
        return
    passes = oracle_pass_count(rec)
    for _ in range(max(args.warmup, 0)):
        oracle_plan_pass(a, b, C, args.eta)
    steps = [oracle_plan_pass(a, b, C, args.eta) for _ in range(args.steps)]
    per_pass = statistics.mean(steps)
    v = per_pass * passes
    sample = (f"each step one real oracle plan pass (Eqs. 6-7, numpy float64) over the full {h * h}x{h * h} "
              f"workload ({per_pass:.2f} s); value = that time x {passes} dense passes of the oracle's Alg. 2 "
              f"for the recorded iteration counts ({rec['outer_iters']} outer, {rec['newton_iters']} Newton, "
              f"{rec['armijo_trials']} Armijo trials, {rec['sinkhorn_iters']} Sinkhorn); leaves out the dense "
              f"Hessian and CG work")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_pass * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": grid_config(args, 1), "value_basis": "estimate scaled from the timed steps",
            "cpu_baseline": {"value": v, "unit": "s", "cores": blas_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """64 independent uneven problems (2-D uniform points, squared Euclidean
    cost / max rebuilt on the fly from the points, eta = 1e-4),
    mixed precision with polish, one ibsn_solve_batch call per step; also the
    same 64 solved one after another on one stream for comparison."""
    import numpy as np
    import torch

    import paper_2603_07156_gb300 as G
    from workloads import batched_points

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    probs = []
    for (m, n, x, y, a, b, eta) in batched_points(count=64):
        xd = torch.tensor(x, device=dev).contiguous()
        yd = torch.tensor(y, device=dev).contiguous()
        # squared-Euclidean cost / max rebuilt on the fly from the points; the
        # max of ||x_i - y_j||^2 is taken once here (float64, on the device)
        cmax = float(((xd[:, None, :] - yd[None, :, :]) ** 2).sum(-1).max())
        probs.append(G.Problem(a=torch.tensor(a, device=dev), b=torch.tensor(b, device=dev), eta=eta, x=xd, y=yd,
                               cost_scale=1.0 / cmax))
    extra = {"nnz_cap": args.nnz_cap} if args.nnz_cap > 0 else {}
    prm = G.params(precision="mixed", **extra)
    wss = [G.alloc_workspace(p, prm) for p in probs]
    entries = sum(int(p.a.numel()) * int(p.b.numel()) for p in probs)
    for _ in range(max(args.warmup, 1)):  # warm-up on the 8 smallest problems
        small = sorted(range(len(probs)), key=lambda q: probs[q].a.numel() * probs[q].b.numel())[:8]
        G.solve_batch([probs[q] for q in small], prm, threads=args.batch_threads, workspaces=[wss[q] for q in small])
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index if dev.index is not None else 0) if rank == 0 else None
    if clocks:
        clocks.start()
    times, out = [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = G.solve_batch(probs, prm, threads=args.batch_threads, workspaces=wss)
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t0)
    barrier(world)
    clk = clocks.stop() if clocks else None
    rep = replica_line_fields(statistics.mean(times), world)
    t_seq = None
    if args.sequential:  # the same problems one after another on one stream, for comparison
        t0 = time.perf_counter()
        for p, w in zip(probs, wss):
            G.solve(p, prm, workspace=w)
        torch.cuda.synchronize(dev)
        t_seq = time.perf_counter() - t0
    if rank != 0:
        return
    gaps = [r["rel_gap"] for r in out]
    line = {
        "metric": "s for 64 uneven OT problems to rel. gap 1e-8 (batched)", "value": rep["value"], "unit": "s",
        "n_gpus": rep["n_gpus"], "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": rep["value"] * 1e3, "higher_is_better": False, "scaling": rep["scaling"],
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "64 problems, m, n ~ U{500..5000}, 2-D uniform points, squared Euclidean / max "
                               "(rebuilt on the fly from the points), random marginals, seeds 100..163, eta=1e-4",
                   "entries": entries, "threads": args.batch_threads, "precision": "mixed",
                   "l2": "64 problems' data far larger than L2, no flush", "parallelism": f"replicas x{world}"},
        "sequential_s": t_seq, "batch_speedup": t_seq / rep["value"] if t_seq else None,
        "outer_iters": {"mean": statistics.mean(r["outer_iters"] for r in out),
                        "max": max(r["outer_iters"] for r in out)},
        "solve_s": {"mean": statistics.mean(r["seconds"] for r in out), "max": max(r["seconds"] for r in out)},
        "converged": sum(1 for r in out if r["converged"]), "max_rel_gap": max(gaps),
        "timing": "host wall clock around the call (the call ends with every stream synchronised)",
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_warmstart(args):
    """Learned warm start: solve --ws-train problems (2-D 4-component Gaussian
    mixtures, m = n = --ws-train-n, eta = 1e-4, mixed precision), train the
    network on their potentials with the library's kernels (minibatches of
    16), then time solves of fresh problems at m = n = --ws-eval-n from the
    zero start and from the judged warm start (prediction + judge + solve).
    One step = one evaluation problem solved both ways."""
    import numpy as np
    import torch

    import paper_2603_07156_gb300 as G
    from workloads import warmstart_gmm_problem, warmstart_init_params

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    prm = G.params(precision="mixed")

    from types import SimpleNamespace

    def gpu(p):  # squared-Euclidean cost rebuilt on the fly from the points
        t = lambda v: torch.tensor(v, dtype=torch.float64, device=dev)  # noqa: E731
        return G.Problem(a=t(p.a), b=t(p.b), eta=p.eta, x=t(p.x).contiguous(), y=t(p.y).contiguous(),
                         cost_scale=p.cost_scale)

    def clouds(n, seed):  # the generator's points and marginals, without its cost matrix
        p = warmstart_gmm_problem(n, seed)
        return SimpleNamespace(x=p.x, y=p.y, a=p.a, b=p.b, eta=p.eta, cost_scale=p.cost_scale)

    t0 = time.perf_counter()
    train = [clouds(args.ws_train_n, 10_000 + s) for s in range(args.ws_train)]
    targets, solved = [], 0
    for k in range(0, len(train), 32):  # training solves run concurrently, 32 problems per batched call
        outs = G.solve_batch([gpu(p) for p in train[k:k + 32]], prm, threads=args.batch_threads)
        targets += [r["gamma"] for r in outs]
        solved += sum(int(r["converged"]) for r in outs)
        print(f"training solves {len(targets)}/{len(train)} converged {solved} "
              f"{time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)
    torch.cuda.synchronize(dev)
    t_solves = time.perf_counter() - t0
    batches = []
    for k in range(0, len(train) - 15, 16):
        batches.append((G.warmstart.PointBatch.from_problems(train[k:k + 16], device=dev),
                        torch.cat(targets[k:k + 16]).contiguous()))
    tr = G.warmstart.Trainer(warmstart_init_params(0), device=dev)
    t0 = time.perf_counter()
    losses = [tr.step(*batches[s % len(batches)]) for s in range(args.ws_adam_steps)]
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0

    def evaluate(seed):
        p = clouds(args.ws_eval_n, 20_000 + seed)
        gp = gpu(p)
        ws = G.alloc_workspace(gp, prm)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        plain = G.solve(gp, prm, workspace=ws)
        torch.cuda.synchronize(dev)
        t_plain = time.perf_counter() - t1
        t1 = time.perf_counter()
        pb = G.warmstart.PointBatch.from_problems([p], device=dev)
        gh = G.warmstart.predict(pb, tr.theta)
        warm = G.warmstart.solve_warm(gp, prm, gh, workspace=ws)
        torch.cuda.synchronize(dev)
        t_warm = time.perf_counter() - t1
        return plain, warm, t_plain, t_warm

    for s in range(args.warmup):
        evaluate(1000 + s)
    barrier(world)
    rows = [evaluate(s) for s in range(args.steps)]
    barrier(world)
    if rank != 0:
        return
    t_plain = statistics.mean(r[2] for r in rows)
    t_warm = statistics.mean(r[3] for r in rows)
    line = {
        "metric": f"s to rel. gap 1e-8 at m=n={args.ws_eval_n} from the judged learned warm start",
        "value": t_warm, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (t_plain + t_warm) * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (network: bf16 weights, f32)", "data": "synthetic",
        "config": {"workload": f"2-D 4-component Gaussian mixtures, m=n={args.ws_eval_n}, random marginals, "
                               f"eta=1e-4; network trained on {args.ws_train} solves at m=n={args.ws_train_n}",
                   "precision": "mixed", "parallelism": f"replicas x{world}"},
        "plain_s": t_plain, "speedup_vs_plain_start": t_plain / t_warm,
        "warm_used": sum(int(r[1]["warm_used"]) for r in rows),
        "outer": [[r[0]["outer_iters"], r[1]["outer_iters"]] for r in rows],
        "sinkhorn": [[r[0]["sinkhorn_iters"], r[1]["sinkhorn_iters"]] for r in rows],
        "converged": sum(int(r[0]["converged"]) + int(r[1]["converged"]) for r in rows),
        "training": {"solves": len(train), "converged": solved, "solve_s": t_solves, "adam_steps": len(losses),
                     "train_s": t_train, "loss_first": losses[0] if losses else None,
                     "loss_last": float(np.mean(losses[-8:])) if losses else None},
        "timing": "host wall clock with device synchronisation; warm includes prediction and judge",
    }
    print(json.dumps(line), flush=True)


def _dense_problem(G, prob, dev, dtype=None):
    import torch
    t = lambda v: torch.tensor(v, dtype=torch.float64, device=dev)  # noqa: E731
    C = t(prob.C) if dtype is None else t(prob.C).to(dtype).contiguous()
    return G.Problem(a=t(prob.a), b=t(prob.b), eta=prob.eta, C=C)


def _timed_solve(G, gp, prm, dev, stream):
    import torch
    ws = G.alloc_workspace(gp, prm)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    r = G.solve(gp, prm, workspace=ws)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    r["s"] = ev0.elapsed_time(ev1) / 1e3
    pcg = [v for k, v in r["profile"].items() if k.startswith("pcg")]
    r["cg_s"] = sum(v["ms"] for v in pcg) / 1e3
    del ws
    return r


def run_eot(args):
    """(E)IBSN on the paper's EOT setting (App. C.4, Table 2): Square cost
    C_ij = (i - j)^2 / max, U(0, 1) marginals, eta = 1e-4, one entropic
    subproblem with X = 1 1^T solved to ||g|| < 1e-9.  Each size is solved in
    float64 and in mixed precision; one step = the largest size, mixed."""
    import torch

    import paper_2603_07156_gb300 as G
    from workloads import paper_synthetic_problem

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sizes = [int(v) for v in args.sizes.split(",")] if args.sizes else [1000, 5000, 10000]
    rows = []
    for n in sizes:
        prob = paper_synthetic_problem("square", n, n, seed=0, eta=1e-4)
        gp = _dense_problem(G, prob, dev)
        for prec in ("fp64", "mixed"):
            r = _timed_solve(G, gp, G.params(precision=prec, eot=1, profile=1, max_newton=200), dev, stream)
            rows.append({"n": n, "precision": prec, "s": r["s"], "cg_s": r["cg_s"], "newton": r["newton_iters"],
                         "mean_cg": r["cg_iters"] / max(r["newton_iters"], 1), "sinkhorn": r["sinkhorn_iters"],
                         "grad_norm": r["grad_norm"], "converged": r["converged"],
                         "polish": bool(r["polish_outer"])})
        del gp
    n = sizes[-1]
    prob = paper_synthetic_problem("square", n, n, seed=0, eta=1e-4)
    gp = _dense_problem(G, prob, dev)
    prm = G.params(precision="mixed", eot=1, max_newton=200)
    for _ in range(args.warmup):
        _timed_solve(G, gp, prm, dev, stream)
    times = [_timed_solve(G, gp, prm, dev, stream)["s"] for _ in range(args.steps)]
    rep = replica_line_fields(statistics.mean(times), world)
    if rank != 0:
        return
    line = {"metric": f"s to ||g|| < 1e-9 on one EOT subproblem ((E)IBSN), Square cost m=n={n}",
            "value": rep["value"], "unit": "s", "n_gpus": rep["n_gpus"], "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rep["value"] * 1e3, "higher_is_better": False,
            "scaling": rep["scaling"], "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"Square cost (i-j)^2/max, U(0,1) marginals, seed 0, eta=1e-4, X = 1 1^T",
                       "m": n, "n": n, "precision": "mixed", "parallelism": f"replicas x{world}"},
            "table": rows,
            "paper_context": "Table 2 (Apple M2 Pro CPU): (E)IBSN MeanCG 163.6 / 290.4 / 241.2, Ite 11 / 13 / 13, "
                             "0.54 / 23.64 / 88.63 s at m=n=1000 / 5000 / 10000"}
    print(json.dumps(line), flush=True)


def run_sphere(args):
    """Unbalanced spherical transport (App. C.4, m >> n): (E)IBSN with
    C = arccos<x, y> / max on synthetic clustered demand and uniform supply
    points on S^2, eta = 1e-3, to ||g|| < 1e-9, for n in {50, 80} and growing
    m, in float64 and mixed precision.  One step = the largest m, n = 80, mixed."""
    import torch

    import paper_2603_07156_gb300 as G
    from workloads import sphere_problem

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sizes = [int(v) for v in args.sizes.split(",")] if args.sizes else [10_000, 100_000, 1_000_000]
    rows = []
    for m in sizes:
        for n in (50, 80):
            prob = sphere_problem(m, n, seed=0)
            gp = _dense_problem(G, prob, dev)
            for prec in ("fp64", "mixed"):
                r = _timed_solve(G, gp, G.params(precision=prec, eot=1, profile=1, max_newton=200), dev, stream)
                rows.append({"m": m, "n": n, "precision": prec, "s": r["s"], "cg_s": r["cg_s"],
                             "newton": r["newton_iters"], "mean_cg": r["cg_iters"] / max(r["newton_iters"], 1),
                             "sinkhorn": r["sinkhorn_iters"], "grad_norm": r["grad_norm"],
                             "converged": r["converged"]})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            del gp
    m, n = sizes[-1], 80
    prob = sphere_problem(m, n, seed=0)
    gp = _dense_problem(G, prob, dev)
    prm = G.params(precision="mixed", eot=1, max_newton=200)
    for _ in range(args.warmup):
        _timed_solve(G, gp, prm, dev, stream)
    times = [_timed_solve(G, gp, prm, dev, stream)["s"] for _ in range(args.steps)]
    rep = replica_line_fields(statistics.mean(times), world)
    if rank != 0:
        return
    line = {"metric": f"s to ||g|| < 1e-9 on one EOT subproblem ((E)IBSN), spherical cost m={m}, n={n}",
            "value": rep["value"], "unit": "s", "n_gpus": rep["n_gpus"], "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rep["value"] * 1e3, "higher_is_better": False,
            "scaling": rep["scaling"], "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "clustered demand / uniform supply points on S^2, C = arccos<x,y>/max, "
                                   "U(0,1) marginals, seed 0, eta=1e-3, X = 1 1^T", "m": m, "n": n,
                       "precision": "mixed", "parallelism": f"replicas x{world}"},
            "table": rows}
    print(json.dumps(line), flush=True)


def run_points(args):
    """The point-cloud workloads: 256^2 uniform points in 2-D (eta = 1e-4) and
    4096^2 points from two 8-component Gaussian mixtures in R^10 (eta = 1e-4),
    each solved to a relative gap of 1e-8 in float64 and in mixed precision,
    with the squared-Euclidean cost rebuilt on the fly from the points and
    with the cost passed as a dense float64 matrix.  One step = the 4096^2
    problem, mixed precision, cost from the points."""
    import torch

    import paper_2603_07156_gb300 as G
    from workloads import workload

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    t = lambda v: torch.tensor(v, dtype=torch.float64, device=dev)  # noqa: E731

    def pts(prob):
        return G.Problem(a=t(prob.a), b=t(prob.b), eta=prob.eta, x=t(prob.x).contiguous(), y=t(prob.y).contiguous(),
                         cost_scale=prob.cost_scale)

    rows = []
    for name in ("c0", "c1"):
        prob = workload(name)
        for cost in ("points", "dense_f64"):
            gp = pts(prob) if cost == "points" else _dense_problem(G, prob, dev)
            for prec in ("fp64", "mixed"):
                r = _timed_solve(G, gp, G.params(precision=prec, profile=1), dev, stream)
                rows.append({"workload": name, "m": prob.m, "n": prob.n, "cost": cost, "precision": prec,
                             "s": r["s"], "cg_s": r["cg_s"], "outer": r["outer_iters"], "newton": r["newton_iters"],
                             "rel_gap": r["rel_gap"], "primal": r["primal"], "converged": r["converged"]})
            del gp
    for q in rows:  # accuracy of each result against the float64 path with the same cost
        ref = next(r for r in rows if r["workload"] == q["workload"] and r["cost"] == q["cost"]
                   and r["precision"] == "fp64")
        q["primal_rel_diff_vs_fp64"] = abs(q["primal"] - ref["primal"]) / abs(ref["primal"])
    prob = workload("c1")
    gp = pts(prob)
    prm = G.params(precision="mixed")
    for _ in range(args.warmup):
        _timed_solve(G, gp, prm, dev, stream)
    times = [_timed_solve(G, gp, prm, dev, stream)["s"] for _ in range(args.steps)]
    rep = replica_line_fields(statistics.mean(times), world)
    if rank != 0:
        return
    line = {"metric": "s to rel. gap 1e-8 at m=n=4096 (R^10 Gaussian mixtures, cost from the points)",
            "value": rep["value"], "unit": "s", "n_gpus": rep["n_gpus"], "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rep["value"] * 1e3, "higher_is_better": False,
            "scaling": rep["scaling"], "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "two 8-component Gaussian mixtures in R^10 (means U[-3,3]^10, unit covariance), "
                                   "4096 points each, C = squared Euclidean / max rebuilt on the fly, "
                                   "U(0.1,1) marginals, seed 1, eta=1e-4", "m": 4096, "n": 4096,
                       "precision": "mixed", "parallelism": f"replicas x{world}"},
            "table": rows}
    print(json.dumps(line), flush=True)


def run_ablation(args):
    """IBSN against IBN (no Hessian sparsification) on the paper's synthetic
    Uniform and Square settings (App. C.3, Table 1): eta = 1e-4, at most 300
    outer steps, stop at a relative duality gap of 1e-8.  Reports Newton
    iterations, time in the Newton-direction solves and total time for both,
    in float64 and in mixed precision.  One step = IBSN, Uniform, largest size,
    mixed."""
    import torch

    import paper_2603_07156_gb300 as G
    from workloads import paper_synthetic_problem

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sizes = [int(v) for v in args.sizes.split(",")] if args.sizes else [1000, 2000]
    rows = []
    # the Square cost hits the outer cap (as in the paper); its dense-Hessian
    # (IBN) solves are run at the smallest size only
    cases = [(n, "uniform") for n in sizes] + [(sizes[0], "square")]
    for n, kind in cases:
        prob = paper_synthetic_problem(kind, n, n, seed=0, eta=1e-4)
        gp = _dense_problem(G, prob, dev)
        for prec in ("fp64", "mixed"):
            for sp in (1, 0):
                prm = G.params(precision=prec, sparsify=sp, profile=1, max_outer=300)
                r = _timed_solve(G, gp, prm, dev, stream)
                rows.append({"n": n, "cost": kind, "precision": prec, "alg": "IBSN" if sp else "IBN",
                             "newton": r["newton_iters"], "cg_iters": r["cg_iters"], "cg_s": r["cg_s"],
                             "s": r["s"], "outer": r["outer_iters"], "rel_gap": r["rel_gap"],
                             "primal": r["primal"], "max_nnz": r["max_nnz"], "converged": r["converged"]})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del gp
    n = sizes[-1]
    prob = paper_synthetic_problem("uniform", n, n, seed=0, eta=1e-4)
    gp = _dense_problem(G, prob, dev)
    prm = G.params(precision="mixed", max_outer=300)
    for _ in range(args.warmup):
        _timed_solve(G, gp, prm, dev, stream)
    times = [_timed_solve(G, gp, prm, dev, stream)["s"] for _ in range(args.steps)]
    rep = replica_line_fields(statistics.mean(times), world)
    if rank != 0:
        return
    line = {"metric": f"s to rel. gap 1e-8 (IBSN), Uniform cost m=n={n}; IBN/IBSN Newton-direction time",
            "value": rep["value"], "unit": "s", "n_gpus": rep["n_gpus"], "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rep["value"] * 1e3, "higher_is_better": False,
            "scaling": rep["scaling"], "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "Uniform C ~ U(0,1)/max and Square (i-j)^2/max, U(0,1) marginals, seed 0, "
                                   "eta=1e-4, at most 300 outer steps", "m": n, "n": n, "precision": "mixed",
                       "parallelism": f"replicas x{world}"},
            "table": rows,
            "paper_context": "Table 1 (Apple M2 Pro CPU): CG time IBN/IBSN 28.38/3.86 s (Uniform 1000), "
                             "497.19/9.69 s (Uniform 5000), 61.55/11.13 s (Square 1000), 803.53/74.37 s (Square 5000)"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_job:
        print(json.dumps(oracle_job(args.oracle_job, args.grid, args.eta)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch64":
        run_batch(args)
        return
    if args.workload == "warmstart":
        run_warmstart(args)
        return
    if args.workload == "eot":
        run_eot(args)
        return
    if args.workload == "ablation":
        run_ablation(args)
        return
    if args.workload == "sphere":
        run_sphere(args)
        return
    if args.workload == "points":
        run_points(args)
        return
    import numpy as np
    import torch

    import paper_2603_07156_gb300 as G

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    h = args.grid
    m = n = h * h
    from workloads import grid_marginals

    a_np, b_np, scale = grid_marginals(h, h, seed=2)
    a = torch.tensor(a_np, dtype=torch.float64, device=dev)
    b = torch.tensor(b_np, dtype=torch.float64, device=dev)
    if args.cost == "dense32":
        # the grid cost materialised as a dense float32 matrix (1 GiB at 16384^2), built in row chunks
        idx = torch.arange(n, device=dev)
        Cd = torch.empty((m, n), dtype=torch.float32, device=dev)
        for r0 in range(0, m, 1024):
            rows = idx[r0:r0 + 1024]
            q = (rows[:, None] // h - idx[None, :] // h) ** 2 + (rows[:, None] % h - idx[None, :] % h) ** 2
            Cd[r0:r0 + 1024] = (q.to(torch.float64) * scale).to(torch.float32)
        prob = G.Problem(a=a, b=b, eta=args.eta, C=Cd)
    else:
        prob = G.Problem(a=a, b=b, eta=args.eta, grid=(h, h), cost_scale=scale)
    extra = {"max_cg": args.max_cg} if args.max_cg > 0 else {}
    if args.max_outer > 0:
        extra["max_outer"] = args.max_outer
    if args.nnz_cap > 0:
        extra["nnz_cap"] = args.nnz_cap
    if args.recompute:
        extra["recompute"] = 1
    prm = G.params(precision=args.precision, profile=1, verbose=args.verbose, **extra)
    ws = G.alloc_workspace(prob, prm)
    stream = torch.cuda.current_stream(dev)

    def one(prm_):
        return G.solve(prob, prm_, workspace=ws, want_plan=False)

    for _ in range(args.warmup):
        one(prm)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index if dev.index is not None else 0) if rank == 0 else None
    if clocks:
        clocks.start()
    results = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(args.steps):
        ev0.record(stream)
        r = one(prm)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(ev0.elapsed_time(ev1) / 1e3)
        results.append(r)
    barrier(world)
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks else None
    rep = replica_line_fields(statistics.mean(times), world)
    t_mean = rep["value"]

    # end to end through the public API: host (pinned) marginals in, potentials out
    e2e = None
    if not args.no_e2e:
        a_h = torch.tensor(a_np, dtype=torch.float64).pin_memory()
        b_h = torch.tensor(b_np, dtype=torch.float64).pin_memory()
        g_h = torch.empty(n, dtype=torch.float64).pin_memory()
        e_times = []
        for _ in range(min(args.steps, 5)):
            torch.cuda.synchronize(dev)
            ev0.record(stream)
            a_d = a_h.to(dev, non_blocking=True)
            b_d = b_h.to(dev, non_blocking=True)
            pe = G.Problem(a=a_d, b=b_d, eta=args.eta, C=prob.C) if args.cost == "dense32" else \
                G.Problem(a=a_d, b=b_d, eta=args.eta, grid=(h, h), cost_scale=scale)
            r = G.solve(pe, prm, workspace=ws)
            g_h.copy_(r["gamma"], non_blocking=True)
            p_h = float(r["primal"])
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            e_times.append(ev0.elapsed_time(ev1) / 1e3)
            assert np.isfinite(p_h)
        e2e = {"value": max_over_ranks(statistics.mean(e_times), world), "unit": "s",
               "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8 + 8}

    # plain float64 GPU path on the same problem (speedup denominator), once
    fp64 = None
    if not args.no_fp64 and args.precision == "mixed" and rank == 0:
        prm64 = G.params(precision="fp64", profile=1, **extra)
        ev0.record(stream)
        r64 = one(prm64)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        t64 = ev0.elapsed_time(ev1) / 1e3
        r_mx = results[-1]
        fp64 = {"s": t64, "rel_gap": r64["rel_gap"], "outer_iters": r64["outer_iters"],
                "converged": r64["converged"], "primal": r64["primal"], "speedup": t64 / t_mean,
                # accuracy of the mixed result against the float64 path (both certified)
                "mixed_primal_rel_diff": abs(r_mx["primal"] - r64["primal"]) / abs(r64["primal"]),
                "mixed_dual_rel_diff": abs(r_mx["dual"] - r64["dual"]) / abs(r64["dual"])}

    # the image-setting eta = 1e-3 of the paper (Sec. 5.2) on the same workload: one mixed solve
    eta3 = None
    if args.eta3 and rank == 0 and args.precision == "mixed":
        prob3 = G.Problem(a=a, b=b, eta=1e-3, C=prob.C) if args.cost == "dense32" else \
            G.Problem(a=a, b=b, eta=1e-3, grid=(h, h), cost_scale=scale)
        ev0.record(stream)
        r3 = G.solve(prob3, G.params(precision="mixed", **extra), workspace=ws)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        eta3 = {"eta": 1e-3, "s": ev0.elapsed_time(ev1) / 1e3, "rel_gap": r3["rel_gap"],
                "outer_iters": r3["outer_iters"], "newton_iters": r3["newton_iters"], "cg_iters": r3["cg_iters"],
                "primal": r3["primal"], "converged": r3["converged"]}
        try:
            rec = json.load(open(TRAJECTORY)).get(f"{h}:0.001", {})
            if "fp64_s" in rec:
                eta3["fp64_plain_recorded_s"] = rec["fp64_s"]
                eta3["speedup_vs_recorded_fp64"] = rec["fp64_s"] / eta3["s"]
        except Exception:
            pass

    if rank != 0:
        return
    # roofline of the dominant step from the live CUDA-event profile of the timed steps
    prof = {}
    launches = 0
    for r in results:
        launches += r["kernel_launches"]
        for k, v in r["profile"].items():
            q = prof.setdefault(k, dict(ms=0.0, calls=0, bytes=0.0))
            q["ms"] += v["ms"]
            q["calls"] += v["calls"]
            q["bytes"] += v["bytes"]
    hbm, hbm_src = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, dv = dom
    d_avg_ms = dv["ms"] / max(dv["calls"], 1)
    d_bytes = dv["bytes"] / max(dv["calls"], 1)
    d_gbs = d_bytes / (d_avg_ms * 1e-3) / 1e9 if d_avg_ms > 0 else 0.0
    roof = {"kernel": dname, "bound": "hbm", "achieved": d_gbs, "peak": hbm, "unit": "GB/s",
            "frac": d_gbs / hbm, "traffic": None, "peak_source": hbm_src,
            "bytes_per_launch": d_bytes, "avg_launch_ms": d_avg_ms}
    try:  # DRAM bytes per launch of the dominant kernel from an ncu capture (profiles/)
        tr = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        if dname in tr:
            roof["traffic"] = tr[dname]
            roof["traffic_source"] = ("ncu DRAM counters of the grid-wide k_pcg32 launches of the early outer "
                                      "steps (profiles/pcg_grid16384.md); the cluster kernel of the later "
                                      "steps reads DRAM only to stage its entries")
    except Exception:
        pass
    if dname.startswith("pcg"):
        # the persistent CG is bound by its synchronisation latency: time per
        # iteration against a floor of two cluster barriers per iteration
        # (0.7 us each, measured on the cluster kernel)
        cg_total = sum(r["cg_iters"] for r in results)
        us = dv["ms"] * 1e3 / max(cg_total, 1)
        roof["latency"] = {"us_per_cg_iter": us, "floor_us": 1.4, "frac": 1.4 / us if us > 0 else None,
                           "cg_iters_per_direction": cg_total / max(sum(r["newton_iters"] for r in results), 1)}
    plan = prof.get("plan_f32") or prof.get("plan_f64")
    plan_pass = None
    if plan:
        pg = plan["bytes"] / (plan["ms"] * 1e-3) / 1e9
        plan_pass = {"gbs": pg, "frac_of_measured": pg / hbm, "frac_of_8tbs": pg / 8000.0,
                     "avg_ms": plan["ms"] / plan["calls"], "calls": plan["calls"]}
    r0 = results[-1]
    # CPU oracle baseline: real oracle work on this host's cores
    cpu = None if args.no_cpu else cpu_baseline(args, int(r0["newton_iters"]))
    line = {
        "metric": METRIC, "value": t_mean, "unit": "s", "n_gpus": rep["n_gpus"], "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_mean * 1e3, "higher_is_better": False, "scaling": rep["scaling"],
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": grid_config(args, world),
        "roofline": roof, "plan_pass": plan_pass, "fp64_plain": fp64, "eta_1e-3": eta3,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        "solve": {k: r0[k] for k in ("rel_gap", "primal", "dual", "outer_iters", "newton_iters", "cg_iters",
                                     "sinkhorn_iters", "polish_outer", "max_nnz", "dense_passes",
                                     "marg_viol", "converged")},
        "profile_ms": {k: round(v["ms"] / len(results), 2) for k, v in sorted(prof.items())},
        "profile_calls": {k: v["calls"] // len(results) for k, v in sorted(prof.items())},
        "profile_gbs": {k: round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) for k, v in sorted(prof.items())
                        if v["ms"] > 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
