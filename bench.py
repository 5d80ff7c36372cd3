#!/usr/bin/env python3
"""Benchmark of the PDD Monte Carlo nodal stage on GB300.

Workload (one "step"): the 2D interfacial problem with 256 nodes (2x2
subdomains, 4 interfaces x 64 nodes), 10^5 Euler-Maruyama paths per node at
dt = 1e-4 (Gobet-Menozzi exit test), run four times per step: the plain
estimator and the pathwise control variate built from three synthetic
previous iterates v = u + eps sin(3 pi x) sin(2 pi y) on a 129^2 grid,
eps in {1e-1, 1e-2, 1e-3}.  Inputs are resident in HBM; L2 is flushed
between timed steps.

Prints one JSON line: value = path-steps/s of the whole step (device-resident
inputs), e2e = the same metric through the C ABI with host buffers, the
roofline of the dominant (control-variate) kernel, the FP64 CPU oracle timed
on the host cores as cpu_baseline, nodes/s at a fixed RMSE for every mode,
and the SM clocks sampled during the timed region.

``--impl reference`` times the oracle (the only other implementation of the
method) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("path-steps/s and interfacial nodes/s at fixed RMSE; controlled vs plain; "
          "p50/p99")
UNIT = "path-steps/s"
N_PATHS = 100_000
DT = 1e-4
GRID_N = 129
EPS = [1e-1, 1e-2, 1e-3]
SEED = 1234
TARGET_RMSE = 1e-3
# Thread-instructions per path-step of the 2D kernels (Philox share,
# Box-Muller, coefficients, updates, exit test, and for the control variate
# the cell record, bilinear gradient and xi update), as executed: ncu's
# smsp__thread_inst_executed.sum over the path-steps of the full-size launches
# of this benchmark (a one-pass capture of the 4-steps-per-iteration kernels;
# the planning estimates were 110 and 150).
ALGO_INSTR = {"plain": 93.7, "cv": 126.4}
# DRAM bytes (read + write) per launch of the dominant kernel (the eps = 1e-2
# pass) from the same full-size capture; None whenever the kernel has changed
# since that capture.
NCU_TRAFFIC_BYTES = 1364224
# Thread-instructions per path-step of the 3D control-variate kernel over the
# full-size cascade launch of --workload c2 (ncu smsp__thread_inst_executed.sum
# over its path-steps, a one-pass capture; the planning estimate was 190), for
# the short (4 steps per iteration) and the long (8) iteration the autotuner
# may pick.
INSTR_3D = {"short": 222.7, "long": 217.0}
WORKLOAD = ("2D CFG0 (b=(sin y/2, cos x/2), c=1+x^2+y^2, u=e^{x+y}cos(x-y)), 2x2 subdomains, "
            "256 interfacial nodes x 1e5 paths, dt=1e-4, Gobet-Menozzi; plain + control "
            "variate on 129^2 grids eps in {1e-1,1e-2,1e-3}")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-nodes", type=int, default=64)
    ap.add_argument("--cpu-paths", type=int, default=1000)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch shape")
    ap.add_argument("--small", action="store_true",
                    help="profiling case: the 256 nodes x 1e4 paths (same kernels, launch "
                         "shape and passes as the default step)")
    ap.add_argument("--workload", choices=["c0", "c1", "c2", "c3", "c4", "fit", "mlmc", "paper",
                                           "peaks", "cascade", "cascade3d"],
                    default="c1",
                    help="c1 (default): 2D, 256 nodes, plain + 3 control grids; c0: 24 nodes, "
                         "plain, dt 1e-3; fit: Algorithm 3 on the 24 nodes; c2: 3D "
                         "three-level cascade in one launch (CUDA graph); c3: serving with "
                         "Poisson arrivals; c4: anisotropic 2D, FP32 vs FP64 paths; mlmc: "
                         "multilevel driver at a fixed RMSE vs the single level; paper: the "
                         "paper's example PDE on 18 nodes; cascade / cascade3d: Algorithms 3-5 "
                         "on the 2D / 3D nodes")
    ap.add_argument("--a0", type=float, default=1e-3, help="cascade: nodal target tolerance")
    ap.add_argument("--window", type=float, default=10.0, help="c3: arrival window (s)")
    ap.add_argument("--rate", type=float, default=200.0, help="c3: arrivals per second")
    ap.add_argument("--iteration", choices=["tuned", "auto", "short", "long"], default="tuned",
                    help="c2: steps per iteration (default: the autotuner's choice)")
    ap.add_argument("--deadline", type=float, default=10.0,
                    help="c3: admission deadline (s) of the server at the offered rate")
    return ap.parse_args()


# ---------------------------------------------------------------- CPU oracle --
def _oracle_task(task):
    """One (pass, node) of the oracle on the host (spawned worker)."""
    import numpy as np
    import oracle
    from paper_1512_02818_gb300 import workloads as W
    eps, node, n_paths, tag = task
    grad, cv, gn = None, oracle.CV_NONE, 0
    if eps is not None:
        grad = oracle.build_gradient(2, W.control_grid(0, GRID_N, eps))
        cv, gn = oracle.CV_GRID, GRID_N
    r = oracle.estimate_nodes(0, np.asarray(node, dtype=np.float32)[None], n_paths, DT, seed=SEED,
                              tag=tag, cv=cv, grad=grad, grid_n=gn, per_path=False)
    return float(r["mean_steps"][0]) * n_paths


_GRADS = {}


def _oracle_task_any(task):
    """One node of the oracle for any workload (spawned worker):
    task = (kind, eps, grid_n, node, n_paths, h, tag); eps None = plain."""
    import numpy as np
    import oracle
    from paper_1512_02818_gb300 import workloads as W
    kind, eps, gn, node, n_paths, h, tag = task
    dim = 3 if kind == W.CUBE_3D else 2
    grad, cv = None, oracle.CV_NONE
    if eps is not None:
        key = (kind, gn, eps)
        if key not in _GRADS:
            _GRADS[key] = oracle.build_gradient(dim, W.control_grid(kind, gn, eps))
        grad = _GRADS[key]
        cv = oracle.CV_GRID_CELLS16 if dim == 3 else oracle.CV_GRID
    r = oracle.estimate_nodes(kind, np.asarray(node, dtype=np.float32)[None], n_paths, h,
                              seed=SEED, tag=tag, cv=cv, grad=grad, grid_n=gn if grad is not None
                              else 0, per_path=False)
    return float(r["mean_steps"][0]) * n_paths


def oracle_pool_time(tasks, cores, fn=_oracle_task):
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(fn, tasks[:cores])  # warm the workers (imports, table builds)
        t0 = time.perf_counter()
        steps = pool.map(fn, tasks)
        dt = time.perf_counter() - t0
    return sum(steps), dt


def cpu_baseline_of(kind, eps, grid_n, nodes, n_paths, h, tag, sample):
    """The oracle, as it stands, on all host cores over a bounded sample
    (one task per node); returns the bench line's cpu_baseline object."""
    cores = cpu_cores()
    tasks = [(kind, eps, grid_n, tuple(float(c) for c in nd), n_paths, h, tag) for nd in nodes]
    steps, secs = oracle_pool_time(tasks, cores, _oracle_task_any)
    return {"value": steps / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sample} ({steps:.3g} path-steps, {secs:.2f} s wall, FP64, one process "
                      "per core)"}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ clocks ----
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id: str | None):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, power, reasons = [], [], [], set()
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.file.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ helpers ---
def smi_id(local: int) -> str:
    """nvidia-smi -i selector of the CUDA device `local` (its UUID)."""
    import torch
    uuid = getattr(torch.cuda.get_device_properties(local), "uuid", None)
    if uuid is None:
        return str(local)
    u = str(uuid)
    return u if u.startswith("GPU-") else "GPU-" + u


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def stream_tag(rank: int, pass_idx: int) -> int:
    """Independent Philox streams per rank (replicas of the same workload)."""
    return 16 * rank + pass_idx


# ---------------------------------------------------------------- our arm -----
def fixed_rmse_runs(torch, pdd, prob, dev, nodes_np, res_np, passes, rank, target):
    """Measured nodes/s at a fixed RMSE `target` for every mode of the step.

    For node i and mode m, N_i = ceil(V_i / (target^2 / 2)) paths, V_i being
    the mode's per-node variance from the timed step (plain: V[phi], control
    variate: V[phi + xi]), so that the statistical error of every node is at
    most target / sqrt(2) (the balanced choice of eq. F:N_y_h; the rest of the
    budget is the bias).  The nodes are sorted by N_i and split into up to 128
    groups, each run as one level of a single pdd_estimate_levels call with
    the group's largest N_i and a stream of its own, the groups with the
    longest expected paths (exit indices of the timed step) first.  The call (device-resident
    inputs and outputs, synchronous) is timed on the host clock, after a
    1-path-per-node call of the same levels loaded the kernel.  The achieved
    RMSE is against the exact solution over all nodes, bias included."""
    import numpy as np
    from paper_1512_02818_gb300 import workloads as W
    n = nodes_np.shape[0]
    u = W.exact_u(0, nodes_np.astype(np.float64))
    out = {"target_rmse": target, "measured": True}
    for pi, (name, gid) in enumerate(passes):
        r = res_np[pi]
        var = r["var_phi"] if gid == pdd.PDD_CV_NONE else r["var_cv"]
        need = np.maximum(2, np.ceil(var / (target * target / 2.0))).astype(np.int64)
        groups = [g for g in np.array_split(np.argsort(need, kind="stable"), min(128, n))
                  if g.size]
        # launch order: the groups with the longest expected paths first (their
        # segments' paths start in the launch's first wave instead of joining a
        # late wave and lengthening its tail); each group keeps its own stream
        order = sorted(range(len(groups)), key=lambda gi: -float(r["mean_steps"][groups[gi]].max()))
        levels = []
        for gi in order:
            idx = groups[gi]
            cols = [torch.from_numpy(np.ascontiguousarray(nodes_np[idx, j])).to(dev)
                    for j in range(2)]
            levels.append((idx, cols, int(need[idx].max()),
                           1_000_000 + 4096 * rank + 512 * pi + gi))

        def prep(n_paths_of):
            pr = [prob._prepare(cols, n_paths_of(np_), DT, gid, SEED, tag, 1.0, False, True,
                                False, False) for (_, cols, np_, tag) in levels]
            return [p[0] for p in pr], [p[1] for p in pr], [p[2] for p in pr]

        wa, wo, _ = prep(lambda _: 1)
        st = pdd.pdd_estimate_levels(prob.handle, wa, wo, 0)
        la, lo, lres = prep(lambda np_: np_)
        torch.cuda.synchronize()
        prob.ctx.set_timing(True)
        prob.ctx.kernel_time()
        t0 = time.perf_counter()
        st = pdd.pdd_estimate_levels(prob.handle, la, lo, 0)
        wall = time.perf_counter() - t0
        kernel_ms, _, _ = prob.ctx.kernel_time()
        prob.ctx.set_timing(False)
        est = np.zeros(n)
        path_steps = 0.0
        key = "mean_phi" if gid == pdd.PDD_CV_NONE else "mean_cv"
        for (idx, _, np_, _), rr in zip(levels, lres):
            est[idx] = rr[key].cpu().numpy()
            path_steps += float((rr["mean_steps"].cpu().numpy() * np_).sum())
        out[name] = {"nodes_per_s": n / wall, "wall_s": wall, "status": int(st),
                     "path_kernel_s": kernel_ms / 1e3, "segments": len(levels),
                     "paths": int(sum(np_ * len(idx) for (idx, _, np_, _) in levels)),
                     "path_steps": path_steps, "path_steps_per_s": path_steps / wall,
                     "achieved_rmse": float(np.sqrt(np.mean((est - u) ** 2))),
                     "median_paths_per_node": float(np.median(need)),
                     "median_var": float(np.median(var))}
    for name, _ in passes[1:]:
        out[name]["speedup_vs_plain"] = out[name]["nodes_per_s"] / out["plain"]["nodes_per_s"]
    return out


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_1512_02818_gb300 import pdd
    from paper_1512_02818_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    gpu_id = smi_id(local)

    # CPU baseline pool first (spawned workers, rank 0 at N=1 only)
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nodes_all = W.workload_nodes("c1")
        stride = max(1, len(nodes_all) // args.cpu_nodes)
        sample = nodes_all[::stride][: args.cpu_nodes]
        tasks = [(1e-2, tuple(map(float, x)), args.cpu_paths, 2) for x in sample]
        cores = cpu_cores()
        steps, secs = oracle_pool_time(tasks, cores)
        cpu_baseline = {"value": steps / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
                        "sample": (f"{len(tasks)} nodes x {args.cpu_paths} paths of the eps=1e-2 "
                                   f"control-variate pass ({steps:.3g} path-steps, "
                                   f"{secs:.1f} s wall, FP64, one process per core)")}

    ctx = pdd.Context(local)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    for slot, eps in enumerate(EPS):
        prob.set_control_grid(slot, W.control_grid(0, GRID_N, eps))
    nodes_np = W.workload_nodes("c1")
    n_paths = N_PATHS
    if args.small:
        n_paths = 10_000
    n_nodes = nodes_np.shape[0]
    cols_dev = [torch.from_numpy(np.ascontiguousarray(nodes_np[:, j])).to(dev) for j in range(2)]
    cols_host = [torch.from_numpy(np.ascontiguousarray(nodes_np[:, j])).pin_memory()
                 for j in range(2)]
    passes = [("plain", pdd.PDD_CV_NONE)] + [(f"eps{e:g}", i) for i, e in enumerate(EPS)]

    def step(host=False):
        out = []
        for pi, (_, gid) in enumerate(passes):
            out.append(prob.estimate(cols_host if host else cols_dev, n_paths, DT, grid_id=gid,
                                     seed=SEED, stream_tag=stream_tag(rank, pi),
                                     async_=not host, device_out=not host, host_inputs=host,
                                     pin_host=host))
        return out

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.set_stream(ctx.stream)  # events, flushes and kernels on one stream
    # launch shape and iteration from the library's autotuner, on one full
    # control-variate pass
    tuned = (0, 0, None)
    if not args.no_autotune:
        tuned = prob.autotune(cols_dev, n_paths, DT, grid_id=1)
    launch_iter = ctx.get_launch()[2]
    launch_claim = ctx.get_claim()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ctx.kernel_time()  # drop warm-up events
    launches0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_id)
    results = None
    for s in range(args.steps):
        flush.zero_()  # L2 flush (256 MB > 126 MB L2), outside the timed events
        ev[s][0].record()
        results = step()
        ev[s][1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    launches = ctx.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    _, n_timed, per_launch = ctx.kernel_time()
    ctx.set_timing(False)

    # work of one step, from the results (deterministic, identical every step)
    res_np = [{k: v.cpu().numpy() for k, v in r.items() if torch.is_tensor(v)} for r in results]
    pass_steps = [float((r["mean_steps"] * r["n_paths"]).sum()) for r in res_np]
    steps_per_step = sum(pass_steps)
    total_ms = max(1e-9, sum(step_ms))
    total_ms_max = reduce_max(total_ms, world)
    total_work = reduce_sum(steps_per_step * args.steps, world)
    value = total_work / (total_ms_max / 1e3)

    # per-pass kernel durations (launch order: plain, eps1, eps2, eps3 per step)
    P = len(passes)
    dur = {name: [per_launch[s * P + i] for s in range(args.steps)]
           for i, (name, _) in enumerate(passes)}
    rate = {name: pass_steps[i] / (statistics.mean(dur[name]) / 1e3)
            for i, (name, _) in enumerate(passes)}
    kappa = {name: rate["plain"] / rate[name] for name, _ in passes[1:]}

    # roofline of the dominant kernel: the control-variate path kernel (eps 1e-2)
    dom = "eps0.01"
    avg_ms = statistics.mean(dur[dom])
    instr = ALGO_INSTR["cv"] * pass_steps[2]
    achieved = instr / (avg_ms / 1e3) / 1e12
    peak = sms * 4 * 32 * 2.070e9 / 1e12  # one warp instruction per SMSP per cycle at max clock
    plain_ms = statistics.mean(dur["plain"])
    plain_frac = ALGO_INSTR["plain"] * pass_steps[0] / (plain_ms / 1e3) / 1e12 / peak
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "T thread-instr/s", "frac": achieved / peak, "traffic": NCU_TRAFFIC_BYTES,
                "kernel": "paths_2d<Cfg0,float,grid-CV>",
                "algorithmic": f"{ALGO_INSTR['cv']:.1f} thread-instr per path-step (ncu, "
                               f"executed) x {pass_steps[2]:.4g} path-steps per launch",
                "peak_basis": f"{sms} SMs x 4 schedulers x 32 lanes x 2070 MHz "
                              "(derived issue peak)",
                "plain_kernel_frac": plain_frac}

    # nodes/s at a fixed RMSE, measured: per node N_i = ceil(V_i / (a^2/2))
    # paths (the balanced choice of eq. F:N_y_h) with V_i from the timed step,
    # then every mode run at those N through the library and timed
    fixed = fixed_rmse_runs(torch, pdd, prob, dev, nodes_np, res_np, passes, rank,
                            TARGET_RMSE if not args.small else 4 * TARGET_RMSE)
    for i, (name, _) in enumerate(passes):
        if i == 0:
            continue
        r = res_np[i]
        pred = r["var_phi"] / (kappa[name] * r["var_cv"])
        fixed[name]["predicted_speedup_median"] = float(np.median(pred))
        fixed[name]["kappa"] = kappa[name]
        # the paper's cost unit (eq. F:VR_Pointwise_cost): path-steps, the
        # controlled ones weighted by kappa -- the speedup the prediction is about
        fixed[name]["work_speedup_vs_plain"] = (
            fixed["plain"]["path_steps"] / (kappa[name] * fixed[name]["path_steps"]))

    # end to end through the C ABI with host buffers (pinned), copies included
    torch.cuda.synchronize()
    e2e_s = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(host=True)
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = reduce_max(sum(e2e_s), world)
    e2e_value = reduce_sum(steps_per_step * len(e2e_s), world) / e2e_total
    h2d = len(passes) * 2 * n_nodes * 4
    d2h = len(passes) * (len(pdd.STAT_FIELDS) + len(pdd.COUNT_FIELDS)) * n_nodes * 8

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.small else "profiling case: " + WORKLOAD,
                   "n_nodes": n_nodes, "n_paths": n_paths, "dt": DT,
                   "grid": GRID_N, "eps": EPS, "passes_per_step": len(passes),
                   "path_steps_per_step": steps_per_step, "l2": "flushed between steps (256 MB)",
                   "parallelism": f"replicas x{world} (independent Philox streams per rank)"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "cpu_baseline": cpu_baseline,
        "fixed_rmse": fixed,
        "pass_rate_path_steps_per_s": rate,
        "clocks": clk,
        "timed_kernel_launches": n_timed,
        "launch_shape": {"block_threads": tuned[0] or (512 if n_nodes <= 512 else 128),
                         "max_blocks": tuned[1],
                         "iteration": ["auto", "short", "long"][launch_iter],
                         "paths_per_lane_claim": launch_claim or "auto",
                         "chosen_by": "pdd_autotune on the eps=1e-2 pass" if tuned[2]
                         else "library default"},
    }
    prob.close()
    ctx.close()
    return line


# ---------------------------------------------------------- reference arm -----
def run_reference(args):
    import numpy as np
    from paper_1512_02818_gb300 import workloads as W
    nodes_all = W.workload_nodes("c1")
    sample = nodes_all[::8][:32]
    paths = 400
    eps_list = [None] + EPS
    tasks = [(e, tuple(map(float, x)), paths, pi) for pi, e in enumerate(eps_list)
             for x in sample]
    cores = cpu_cores()
    for _ in range(args.warmup):
        pass  # the pool warm-up inside oracle_pool_time covers imports
    times, work = [], []
    for _ in range(args.steps):
        steps, secs = oracle_pool_time(tasks, cores)
        times.append(secs)
        work.append(steps)
    value = sum(work) / sum(times)
    sample_desc = (f"{len(sample)} of 256 nodes x {paths} paths x 4 passes per step "
                   f"(plain + 3 control-variate grids), FP64, one process per core")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_nodes": 256, "n_paths": N_PATHS, "dt": DT,
                   "grid": GRID_N, "eps": EPS, "sample": sample_desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ----------------------------------------------------------- other workloads ---
def _timed_steps(torch, stream, steps, fn, flush):
    """CUDA-event times (ms) of `steps` calls of fn() on `stream`, L2 flushed between."""
    out = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def run_c2(args):
    """3D cube, 4^3 subdomains, 9,216 nodes; three levels (1e3/1e4/1e5 paths at
    dt 1e-2/1e-3/1e-4 with eps 1e-1/1e-2/1e-3 grids on 65^3) plus a plain pass
    at the coarsest level, all in one persistent launch replayed from a CUDA
    graph."""
    import numpy as np
    import torch

    from paper_1512_02818_gb300 import pdd
    from paper_1512_02818_gb300 import workloads as W
    # oracle pool first: spawned workers, before this process touches the GPU
    cpu = None if args.no_cpu_baseline else cpu_baseline_of(
        W.CUBE_3D, 1e-3, 65, W.workload_nodes("c2")[::576], 1000, 1e-4, 3,
        "level 3: 16 of the 9,216 nodes x 1e3 paths at h = 1e-4, eps = 1e-3 grid 65^3")
    dev = torch.device("cuda", 0)
    ctx = pdd.Context(0)
    torch.cuda.set_stream(ctx.stream)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CUBE_3D)
    levels_cfg = W.WORKLOADS["c2"]["levels"]
    for slot, lv in enumerate(levels_cfg):
        prob.set_control_grid(slot, W.control_grid(2, 65, lv["eps"]))
    nodes = W.workload_nodes("c2")
    div = 1
    if args.small:  # profiling case: 1/16 of the nodes, 1/10 of the paths
        nodes, div = nodes[::16].copy(), 10
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).to(dev) for j in range(3)]
    lv = [dict(nodes=cols, n_paths=c["n_paths"] // div, dt=c["dt"], grid_id=i, stream_tag=1 + i)
          for i, c in enumerate(levels_cfg)]
    lv.append(dict(nodes=cols, n_paths=levels_cfg[0]["n_paths"] // div, dt=levels_cfg[0]["dt"],
                   grid_id=pdd.PDD_CV_NONE, stream_tag=1))
    prepared = [prob._prepare(l["nodes"], l["n_paths"], l["dt"], l["grid_id"], SEED,
                              l["stream_tag"], 1.0, False, True, False, False) for l in lv]
    largs, louts = [p[0] for p in prepared], [p[1] for p in prepared]
    # launch shape from the autotuner on an eighth of the finest level (the
    # level that holds 99 % of the cascade's path-steps)
    tuned = (0, 0, None)
    if not args.no_autotune:
        sub = [torch.from_numpy(np.ascontiguousarray(nodes[::8, j])).to(dev) for j in range(3)]
        tuned = prob.autotune(sub, levels_cfg[2]["n_paths"] // (10 * div), levels_cfg[2]["dt"],
                              grid_id=2, stream_tag=77)
    if args.iteration != "tuned":
        ctx.set_iteration({"auto": pdd.PDD_ITER_AUTO, "short": pdd.PDD_ITER_SHORT,
                           "long": pdd.PDD_ITER_LONG}[args.iteration])
    # the cascade's auto rule takes the long iteration (its short-path level
    # holds 0.02 % of the path-steps)
    iter_run = {0: "long", 1: "short", 2: "long"}[ctx.get_launch()[2]]
    instr_3d = INSTR_3D[iter_run]

    def step():
        pdd.pdd_estimate_levels(prob.handle, largs, louts, pdd.PDD_FLAG_GRAPH | pdd.PDD_FLAG_ASYNC)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    clocks = ClockSampler(smi_id(0))
    ms = _timed_steps(torch, ctx.stream, args.steps, step, flush)
    clk = clocks.stop()
    launches = ctx.launch_count() - launches0
    res = [{k: v.cpu().numpy() for k, v in p[2].items() if torch.is_tensor(v)} for p in prepared]
    u = W.exact_u(2, nodes.astype(np.float64))
    per_level = []
    work = 0.0
    for i, r in enumerate(res):
        steps_l = float((r["mean_steps"] * r["n_paths"]).sum())
        work += steps_l
        mean = r["mean_cv"] if i < 3 else r["mean_phi"]
        per_level.append({"n_paths": lv[i]["n_paths"], "dt": lv[i]["dt"],
                          "cv": "grid eps %g" % levels_cfg[i]["eps"] if i < 3 else "plain",
                          "path_steps": steps_l,
                          "rmse": float(np.sqrt(np.mean((mean - u) ** 2))),
                          "median_vr": float(np.nanmedian(r["vr"])) if i < 3 else 1.0,
                          "mean_steps": float(np.mean(r["mean_steps"]))})
    total_ms = sum(ms)
    value = work * args.steps / (total_ms / 1e3)
    line = {"workload": "c2", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "3D cube b=0 c=1 u=e^x sin y cos z + xyz, 4^3 subdomains, "
                                   "9216 nodes, levels (1e3,1e-2,eps 1e-1) (1e4,1e-3,eps 1e-2) "
                                   "(1e5,1e-4,eps 1e-3) on 65^3 grids + plain level-1 pass, one "
                                   "persistent launch replayed from a CUDA graph",
                       "l2": "flushed between steps (256 MB)"},
            "nodes_per_s": len(nodes) * args.steps / (total_ms / 1e3),
            "launch_shape": {"block_threads": tuned[0] or 128, "max_blocks": tuned[1],
                             "iteration": ["auto", "short", "long"][ctx.get_launch()[2]],
                             "paths_per_lane_claim": ctx.get_claim() or "auto",
                             "chosen_by": "pdd_autotune on 1/8 of the finest level" if tuned[2]
                             else "library default"},
            "levels": per_level, "graph_captures": ctx.graph_count(),
            "gpu_launches": int(launches), "clocks": clk, "cpu_baseline": cpu,
            "roofline": {"bound": "alu", "unit": "T thread-instr/s",
                         "achieved": instr_3d * value / 1e12 if instr_3d else None,
                         "peak": torch.cuda.get_device_properties(0).multi_processor_count
                         * 4 * 32 * 2.070e9 / 1e12,
                         "algorithmic": f"{instr_3d} thread-instr per 3D control-variate "
                                        f"path-step ({iter_run} iteration; ncu, executed, "
                                        "full-size cascade launch)",
                         "second_limit": "L1 data pipe: 78 % of its peak in the ncu capture of "
                                         "the profiling case (two 256-bit cell-record gathers "
                                         "per step), issue 75 %"}}
    line["roofline"]["frac"] = (line["roofline"]["achieved"] / line["roofline"]["peak"]
                                if instr_3d else None)
    prob.close()
    ctx.close()
    return line


def run_c3(args):
    """Serving: Poisson arrivals of requests over the 2D problem (1-4,096 nodes
    log-uniform, 1e3-1e6 paths log-uniform, dt in {1e-2,1e-3,1e-4}, eps in
    {none, 1e-1, 1e-2}); continuous batching with admission by predicted work
    against a deadline; p50/p99 latency of completed requests and goodput
    (completed over executed path-steps).  Runs the offered rate, then an
    arrival rate whose offered path-steps/s are 0.7x the served rate of one
    large request."""
    import numpy as np
    import torch

    from paper_1512_02818_gb300 import pdd
    from paper_1512_02818_gb300 import workloads as W
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, GRID_N, 1e-1))
    prob.set_control_grid(1, W.control_grid(0, GRID_N, 1e-2))
    gid = {None: pdd.PDD_CV_NONE, 1e-1: 0, 1e-2: 1}

    def serve(rate, window, drain_s, seed, policy=pdd.PDD_SERVE_FAIR, deadline=0.0,
              steps_of=None):
        reqs = W.serving_requests(seed, rate, window)
        srv = pdd.Server(ctx, max_active=32, max_queue=64, device_arena_bytes=1 << 30,
                         policy=policy, deadline_s=deadline)
        t0 = time.perf_counter()
        outstanding, lat, done_steps, done_nodes = {}, [], 0.0, 0
        refused = {"busy": 0, "deadline": 0, "nomem": 0, "other": 0}
        i = 0

        def poll_all():
            nonlocal done_steps, done_nodes
            for t in list(outstanding):
                r = outstanding[t]
                st, res = srv.poll(t, r["n_nodes"], 0)
                if st == pdd.PDD_ERR_NOT_READY:
                    continue
                del outstanding[t]
                if st == pdd.PDD_OK:
                    lat.append(time.perf_counter() - t0 - r["arrival"])
                    done_steps += float((res["mean_steps"] * res["n_paths"]).sum())
                    done_nodes += r["n_nodes"]

        names = {pdd.PDD_ERR_BUSY: "busy", pdd.PDD_ERR_DEADLINE: "deadline",
                 pdd.PDD_ERR_NOMEM: "nomem"}
        while i < len(reqs) or (outstanding and time.perf_counter() - t0 < window + drain_s):
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i]["arrival"] <= now:
                r = reqs[i]
                i += 1
                try:
                    t = srv.submit(prob, r["nodes"], r["n_paths"], r["dt"], grid_id=gid[r["eps"]],
                                   seed=SEED, stream_tag=r["tag"])
                    outstanding[t] = r
                except pdd.PddError as e:
                    refused[names.get(e.status, "other")] += 1
            poll_all()
            time.sleep(0.001)
        elapsed = time.perf_counter() - t0
        unfinished = len(outstanding)
        for t in list(outstanding):
            srv.cancel(t)
        stats = srv.stats()
        srv.close()
        offered = sum(float(r["n_nodes"]) * r["n_paths"] * steps_of(r["dt"]) for r in reqs)
        return {"rate_per_s": rate, "window_s": window, "deadline_s": deadline,
                "policy": {pdd.PDD_SERVE_SHORTEST: "shortest_first", pdd.PDD_SERVE_FAIR: "fair",
                           pdd.PDD_SERVE_EARLIEST_DEADLINE: "earliest_deadline"}[policy],
                "offered_requests": len(reqs), "offered_path_steps_per_s": offered / window,
                "completed": len(lat), "refused": refused,
                "cancelled_at_end": unfinished, "launches": stats["launches"],
                "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat else None,
                "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat else None,
                "completed_path_steps_per_s": done_steps / elapsed,
                "completed_nodes_per_s": done_nodes / elapsed, "elapsed_s": elapsed,
                # every path-step the retired launches ran, including the slices of
                # requests still running (or cancelled) when the window closed
                "executed_path_steps_per_s": stats["path_steps"] / elapsed,
                "goodput": (stats["completed_path_steps"] / stats["path_steps"]
                            if stats["path_steps"] else None),
                "server_rate_estimate": stats["rate_path_steps_per_s"]}

    clocks = ClockSampler(smi_id(0))
    # capacity: one large request (256 nodes x 1e5 paths, dt 1e-4, eps 1e-2) alone
    # through the server gives its sustained path-steps/s
    srv = pdd.Server(ctx, max_active=32, max_queue=64, device_arena_bytes=1 << 30)
    cal_nodes = W.workload_nodes("c1")
    tc = time.perf_counter()
    t = srv.submit(prob, cal_nodes, N_PATHS, DT, grid_id=1, seed=SEED, stream_tag=999)
    st, res = srv.poll(t, len(cal_nodes), int(600e6))
    cal_s = time.perf_counter() - tc
    srv.close()
    cal_rate = float((res["mean_steps"] * res["n_paths"]).sum()) / cal_s
    # expected exit time on the interfaces (tau = k dt), for the offered work
    e_tau = float(np.mean(res["mean_steps"])) * DT

    def steps_of(dt):
        return e_tau / dt

    # served form at a fixed RMSE: N per request from the pilot variances
    # (balanced choice, stat^2 <= a^2/2 at every node), plain vs eps = 1e-2 CV
    a_t = 2e-3
    u = W.exact_u(0, cal_nodes.astype(np.float64))
    fixed = {}
    for name, grid, var in (("plain", pdd.PDD_CV_NONE, res["var_phi"]),
                            ("cv_eps1e-2", 1, res["var_cv"])):
        n_req = int(np.ceil(np.max(var) / (a_t**2 / 2.0)))
        srv = pdd.Server(ctx, max_active=32, max_queue=64, device_arena_bytes=1 << 30)
        tc = time.perf_counter()
        t = srv.submit(prob, cal_nodes, n_req, DT, grid_id=grid, seed=SEED, stream_tag=77)
        st, rr = srv.poll(t, len(cal_nodes), 2**31 - 1)
        if st != pdd.PDD_OK:
            raise RuntimeError(f"served fixed-RMSE request failed: status {st}")
        secs = time.perf_counter() - tc
        srv.close()
        mean = rr["mean_phi"] if grid == pdd.PDD_CV_NONE else rr["mean_cv"]
        fixed[name] = {"n_paths": n_req, "seconds": secs, "nodes_per_s": len(cal_nodes) / secs,
                       "rmse_vs_exact": float(np.sqrt(np.mean((mean - u) ** 2)))}
    fixed["cv_speedup_nodes_per_s"] = fixed["cv_eps1e-2"]["nodes_per_s"] / fixed["plain"]["nodes_per_s"]
    deadline = args.deadline
    sat = serve(args.rate, args.window, 30.0, 11, pdd.PDD_SERVE_EARLIEST_DEADLINE,
                deadline=deadline, steps_of=steps_of)
    sat_fair = serve(args.rate, args.window, 30.0, 11, deadline=deadline, steps_of=steps_of)
    sat_short = serve(args.rate, args.window, 30.0, 11, pdd.PDD_SERVE_SHORTEST, deadline=deadline,
                      steps_of=steps_of)
    # steady state: arrivals whose offered path-steps/s are 0.7x the served rate
    probe = W.serving_requests(12, 100.0, 100.0)
    mean_req = float(np.mean([r["n_nodes"] * r["n_paths"] * steps_of(r["dt"]) for r in probe]))
    steady_rate = 0.7 * cal_rate / mean_req
    steady = serve(steady_rate, max(30.0, args.window), 90.0, 12, steps_of=steps_of)
    clk = clocks.stop()
    prob.close()
    ctx.close()
    return {"workload": "c3", "metric": METRIC, "value": sat["completed_path_steps_per_s"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serving, Poisson arrivals over the 2D CFG0 problem; "
                                   "1-4096 nodes, 1e3-1e6 paths (log-uniform), dt in "
                                   "{1e-2,1e-3,1e-4}, eps in {none,1e-1,1e-2}; max_active 32, "
                                   "max_queue 64, quantum 8e9 path-steps, admission deadline "
                                   f"{deadline:g} s at the offered rate (earliest-deadline "
                                   "policy; fair shares and shortest-first beside it)"},
            "saturation": sat, "saturation_fair_shares": sat_fair,
            "saturation_shortest_first": sat_short,
            "at_0.7x_served_rate": steady,
            "served_rate_one_request_path_steps_per_s": cal_rate,
            "expected_exit_time": e_tau,
            "fixed_rmse_served": {"target_rmse": a_t, **fixed},
            "mean_request_path_steps": mean_req, "clocks": clk}


def run_c4(args):
    """Anisotropic 2D, 32x32 subdomains, 31,744 nodes x 1e4 paths, dt = 1e-4,
    eps = 1e-2 grid on 513^2: FP32 paths at full size; FP32 and FP64 paths on a
    256-node subsample, compared path by path (first 32 paths of every node) and
    node by node.  Their comparison with the FP64 oracle on the same subsample
    is a GPU test (tests/test_gpu_precision.py)."""
    import numpy as np
    import torch

    from paper_1512_02818_gb300 import pdd
    from paper_1512_02818_gb300 import workloads as W
    # oracle pool first: spawned workers, before this process touches the GPU
    cpu = None if args.no_cpu_baseline else cpu_baseline_of(
        W.ANISO_2D, 1e-2, 513, W.workload_nodes("c4")[::124][:256], 1000, 1e-4, 0,
        "256 of the 31,744 nodes x 1e3 paths, eps = 1e-2 grid 513^2")
    dev = torch.device("cuda", 0)
    ctx = pdd.Context(0)
    torch.cuda.set_stream(ctx.stream)
    v = W.control_grid(1, 513, 1e-2)
    p32 = pdd.Problem(ctx, pdd.PDD_PROBLEM_ANISO_2D)
    p64 = pdd.Problem(ctx, pdd.PDD_PROBLEM_ANISO_2D, precision=pdd.PDD_PATH_FP64)
    p32.set_control_grid(0, v)
    p64.set_control_grid(0, v)
    nodes = W.workload_nodes("c4")
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).to(dev) for j in range(2)]
    n_paths, h = 10_000, 1e-4
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    holder = {}

    def full():
        holder["r"] = p32.estimate(cols, n_paths, h, grid_id=0, async_=True)

    full()
    torch.cuda.synchronize()
    clocks = ClockSampler(smi_id(0))
    ms = _timed_steps(torch, ctx.stream, max(1, args.steps), full, flush)
    r = {k: t.cpu().numpy() for k, t in holder["r"].items() if torch.is_tensor(t)}
    work = float((r["mean_steps"] * r["n_paths"]).sum())
    sub = nodes[::124][:256]
    res, tms = {}, {}
    for name, prob in (("fp32", p32), ("fp64", p64)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        rr = prob.estimate(sub, n_paths, h, grid_id=0, emit_paths=True)
        e1.record(ctx.stream)
        ctx.stream.synchronize()
        tms[name] = e0.elapsed_time(e1)
        res[name] = rr
    clk = clocks.stop()
    k = 32
    ni = np.repeat(np.arange(len(sub)), k)
    pi = np.tile(np.arange(k), len(sub))
    prec = {}
    for name in ("fp32", "fp64"):
        ps = float((res[name]["mean_steps"].cpu().numpy() * n_paths).sum())
        prec[name] = {"path_steps_per_s": ps / (tms[name] / 1e3)}
    # FP32 paths against FP64 paths on the same streams (the FP64 paths' output
    # is emitted in FP32)
    out32 = {f: res["fp32"][f].cpu().numpy()[ni, pi] for f in ("phi", "xi", "steps")}
    out64 = {f: res["fp64"][f].cpu().numpy()[ni, pi] for f in ("phi", "xi", "steps")}
    same = out32["steps"] == out64["steps"]
    prec["paths_fp32_vs_fp64"] = {
        "paths_compared": int(same.size), "exit_step_flips": int((~same).sum()),
        "max_abs_diff_phi": float(np.abs(out32["phi"].astype(np.float64) - out64["phi"])[same].max()),
        "max_abs_diff_xi": float(np.abs(out32["xi"].astype(np.float64) - out64["xi"])[same].max())}
    m32 = res["fp32"]["mean_cv"].cpu().numpy()
    m64 = res["fp64"]["mean_cv"].cpu().numpy()
    se = res["fp64"]["se_cv"].cpu().numpy()
    ok = se > 0  # nodes whose paths all finish at k = 0 have SE = 0
    prec["node_mean_fp32_vs_fp64"] = {"max_abs": float(np.abs(m32 - m64).max()),
                                      "max_over_se": float((np.abs(m32 - m64)[ok] / se[ok]).max())}
    u = W.exact_u(1, nodes.astype(np.float64))
    out = {"workload": "c4", "metric": METRIC, "value": work * len(ms) / (sum(ms) / 1e3),
           "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
           "data": "synthetic", "ms_per_step": sum(ms) / len(ms),
           "config": {"workload": "anisotropic 2D A=[[1,.5],[.5,1]](1+sin(2 pi x)/2), 32x32 "
                                  "subdomains, 31744 nodes x 1e4 paths, dt=1e-4, eps=1e-2 grid "
                                  "513^2; precision study on 256 nodes"},
           "rmse_fp32_full": float(np.sqrt(np.mean((r["mean_cv"] - u) ** 2))),
           "precision": prec, "clocks": clk, "cpu_baseline": cpu}
    p32.close()
    p64.close()
    ctx.close()
    return out


def run_c0(args):
    """The small 2D case: 24 nodes x 1e4 paths, dt = 1e-3, plain estimator."""
    import numpy as np
    import torch

    from paper_1512_02818_gb300 import pdd
    from paper_1512_02818_gb300 import workloads as W
    nodes = W.workload_nodes("c0")
    # oracle pool first: spawned workers, before this process touches the GPU
    cpu = None if args.no_cpu_baseline else cpu_baseline_of(
        W.CFG0_2D, None, 0, nodes, 10_000, 1e-3, 0, "the whole workload: 24 nodes x 1e4 paths")
    ctx = pdd.Context(0)
    torch.cuda.set_stream(ctx.stream)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).cuda() for j in range(2)]
    holder = {}

    def step():
        holder["r"] = prob.estimate(cols, 10_000, 1e-3, async_=True)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        step()
    ms = _timed_steps(torch, ctx.stream, args.steps, step, flush)
    r = {k: v.cpu().numpy() for k, v in holder["r"].items() if torch.is_tensor(v)}
    work = float((r["mean_steps"] * r["n_paths"]).sum())
    u = W.exact_u(0, nodes.astype(np.float64))
    out = {"workload": "c0", "metric": METRIC, "value": work * len(ms) / (sum(ms) / 1e3),
           "unit": UNIT, "ms_per_step": sum(ms) / len(ms), "dtype": "f32", "data": "synthetic",
           "config": {"workload": "2D CFG0, 2x2 subdomains, 24 nodes x 1e4 paths, dt=1e-3, plain"},
           "nodes_per_s": len(nodes) * len(ms) / (sum(ms) / 1e3),
           "rmse": float(np.sqrt(np.mean((r["mean_phi"] - u) ** 2))),
           "max_err_over_se": float(np.max(np.abs(r["mean_phi"] - u) / r["se_phi"])),
           "cpu_baseline": cpu}
    prob.close()
    ctx.close()
    return out


def run_paper(args):
    """The paper's example PDE (sigma = sqrt(2) I, b = cos(x+y)(1,1)/(1.1+sin(x+y)),
    c = (x^2+y^2)/(1.1+sin(x+y)), exact u given) on the assumed domain: the
    unit square cut into 4 vertical strips, 3 interfaces x 6 nodes = 18
    nodes; 1e5 paths at dt = 1e-4, plain and with the control variate of
    v = u + 1e-2 sin(3 pi x) sin(2 pi y) on 129^2; nodes/s at RMSE 1e-3."""
    import numpy as np
    import torch

    from paper_1512_02818_gb300 import pdd
    from paper_1512_02818_gb300 import workloads as W
    ctx = pdd.Context(0)
    torch.cuda.set_stream(ctx.stream)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_PAPER_EX_2D)
    prob.set_control_grid(0, W.control_grid(W.PAPER_EX_2D, GRID_N, 1e-2))
    nodes = W.workload_nodes("paper")
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).cuda() for j in range(2)]
    u = W.exact_u(W.PAPER_EX_2D, nodes.astype(np.float64))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(smi_id(0))
    modes, total_ms, total_steps = {}, 0.0, 0.0
    for name, gid in (("plain", pdd.PDD_CV_NONE), ("cv_eps1e-2", 0)):
        holder = {}

        def step():
            holder["r"] = prob.estimate(cols, N_PATHS, DT, grid_id=gid, async_=True)

        for _ in range(args.warmup):
            step()
        ms = _timed_steps(torch, ctx.stream, args.steps, step, flush)
        r = {k: v.cpu().numpy() for k, v in holder["r"].items() if torch.is_tensor(v)}
        steps = float((r["mean_steps"] * r["n_paths"]).sum())
        mean = r["mean_phi"] if gid == pdd.PDD_CV_NONE else r["mean_cv"]
        var = r["var_phi"] if gid == pdd.PDD_CV_NONE else r["var_cv"]
        rate = steps / (np.mean(ms) / 1e3)
        # nodes/s at RMSE a: N_i = ceil(V_i / (a^2/2)) paths per node at the measured rate
        need = np.ceil(var / (TARGET_RMSE**2 / 2.0)) * r["mean_steps"]
        modes[name] = {"path_steps_per_s": rate, "ms": float(np.mean(ms)),
                       "rmse_at_1e5_paths": float(np.sqrt(np.mean((mean - u) ** 2))),
                       "median_var": float(np.median(var)),
                       "nodes_per_s_at_rmse": len(nodes) / (float(need.sum()) / rate)}
        total_ms += float(np.sum(ms))
        total_steps += steps * len(ms)
    clk = clocks.stop()
    kappa = modes["plain"]["path_steps_per_s"] / modes["cv_eps1e-2"]["path_steps_per_s"]
    sp = modes["cv_eps1e-2"]["nodes_per_s_at_rmse"] / modes["plain"]["nodes_per_s_at_rmse"]
    prob.close()
    ctx.close()
    return {"workload": "paper", "metric": METRIC, "value": total_steps / (total_ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "paper's example PDE, assumed 4-strip domain, 18 nodes x 1e5 "
                                   "paths, dt=1e-4, plain + control variate eps=1e-2 on 129^2",
                       "l2": "flushed between steps (256 MB)"},
            "modes": modes, "kappa": kappa, "cv_speedup_at_rmse": sp,
            "target_rmse": TARGET_RMSE, "clocks": clk}


def run_peaks(args):
    """Issue-rate probe: thread-operations/s of FP32 FMA, INT32 multiply-add,
    SFU exp2 and 3-input logic ops, against the derived issue peak (one warp
    instruction per scheduler per cycle at the maximum SM clock)."""
    import torch

    from paper_1512_02818_gb300 import pdd
    torch.cuda.init()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 4 * 32 * 2.07e9
    clocks = ClockSampler(smi_id(0))
    rates = {}
    for name, kind, iters in (("ffma", 0, 8192), ("imad", 1, 8192), ("sfu_ex2", 2, 2048),
                              ("lop3", 3, 8192)):
        ops, ms = pdd.pdd_debug_issue_rate(kind, iters)
        rates[name] = {"thread_ops_per_s": ops, "ms": ms, "frac_of_issue_peak": ops / peak}
    clk = clocks.stop()
    return {"workload": "peaks", "metric": "thread-operations/s per instruction class",
            "value": rates["ffma"]["thread_ops_per_s"], "unit": "thread-ops/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"issue-rate probe, {4 * sms} blocks x 512 threads, 8 "
                                   "independent chains per thread"},
            "issue_peak_derived": peak, "rates": rates, "clocks": clk}


def run_fit(args):
    """Algorithm 3 on the 24 nodes: cloud of 100 time steps in [1e-3, 1e-2],
    1,000 paths each, psi drawn alongside from w = sin(3 pi x) sin(2 pi y)."""
    import numpy as np
    import torch

    from paper_1512_02818_gb300 import pdd
    from paper_1512_02818_gb300 import workloads as W
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, GRID_N, 1.0) - W.control_grid(0, GRID_N, 0.0))
    nodes = W.workload_nodes("c0")
    prob.fit_constants(nodes, 1000, 1e-3, 1e-2, 100, grid_id=0)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = prob.fit_constants(nodes, 1000, 1e-3, 1e-2, 100, grid_id=0)
    secs = time.perf_counter() - t0
    cloud = r["cloud"]
    work = float((cloud[:, :, 3] / cloud[:, :, 0]).sum() * 1000)  # E[tau_h]/h x paths
    u = W.exact_u(0, nodes.astype(np.float64))
    # Algorithm 4 on the fitted constants: kappa from the per-step time of the
    # control-variate and plain kernels on these nodes, starting tolerance 0.05
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).cuda() for j in range(2)]
    rate = {}
    for name, gid in (("plain", pdd.PDD_CV_NONE), ("cv", 0)):
        prob.estimate(cols, 20000, 1e-3, grid_id=gid)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rr = prob.estimate(cols, 20000, 1e-3, grid_id=gid)
        torch.cuda.synchronize()
        rate[name] = float((rr["mean_steps"].cpu().numpy() * 20000).sum()) / (time.perf_counter() - t1)
    kappa = rate["plain"] / rate["cv"]
    t1 = time.perf_counter()
    a_sched, sp_sched = pdd.pdd_schedule(r["K"], r["beta"], r["alpha"], r["V_phi"], r["V_psi"],
                                         r["rho_phi_psi"], 1.0, kappa, 0.05)
    sched_s = time.perf_counter() - t1
    out = {"workload": "fit", "metric": METRIC, "value": work / secs, "unit": UNIT,
           "seconds": secs, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "Algorithm 3, 24 nodes, 100 time steps in [1e-3, 1e-2], "
                                  "1000 paths each, psi from a synthetic w grid; Algorithm 4 "
                                  "from a0 = 0.05 on the fitted constants"},
           "schedule": {"kappa": kappa, "tolerances": [float(x) for x in a_sched],
                        "predicted_speedups": [float(x) for x in sp_sched], "seconds": sched_s},
           "E_phi_rmse_vs_exact": float(np.sqrt(np.mean((r["E_phi"] - u) ** 2))),
           "median_beta": float(np.median(r["beta"])), "median_V_phi": float(np.median(r["V_phi"])),
           "median_E_tau": float(np.median(r["E_tau"])), "median_K": float(np.median(r["K"])),
           "median_rho_phi_psi": float(np.median(r["rho_phi_psi"]))}
    prob.close()
    ctx.close()
    return out


def run_cascade(args):
    """The cascade Algorithm 4 schedules, run (Algorithm 5's nodal loop) on
    the 256 interfacial nodes of the 2D problem (--workload cascade) or on
    every 16th of the 9,216 nodes of the 3D problem (--workload cascade3d, 576
    nodes, 65^3 grids): Algorithm 3 fit (100 time steps in [1e-3, 1e-2], 10^4
    paths each, psi from w = sin 3pi x sin 2pi y [sin pi z]; nodes within the
    shrinkage layer at some h of the cloud cannot be fitted and are left out),
    kappa measured, the schedule from a0, every level's balanced (h, N) per
    node, all levels in one launch; against PlainPDD(a0) run the same way.
    The previous iterate of tolerance a is synthetic, v = u + (a/2) w."""
    import numpy as np
    import torch

    from paper_1512_02818_gb300 import cascade as C
    from paper_1512_02818_gb300 import pdd
    from paper_1512_02818_gb300 import workloads as W
    three_d = args.workload == "cascade3d"
    kind = pdd.PDD_PROBLEM_CUBE_3D if three_d else pdd.PDD_PROBLEM_CFG0_2D
    gn = 65 if three_d else GRID_N
    ctx = pdd.Context(0)
    torch.cuda.set_stream(ctx.stream)
    prob = pdd.Problem(ctx, kind)
    w_slot = 7
    w = W.control_grid(kind, gn, 1.0) - W.control_grid(kind, gn, 0.0)
    prob.set_control_grid(w_slot, w)
    nodes = W.workload_nodes("c2")[::16] if three_d else W.workload_nodes("c1")
    dim = nodes.shape[1]
    u = W.exact_u(kind, nodes.astype(np.float64))
    n_fit = 10_000
    t0 = time.perf_counter()
    fit = prob.fit_constants(nodes, n_fit, 1e-3, 1e-2, 100, grid_id=w_slot, stream_tag_base=200)
    fit_s = time.perf_counter() - t0
    fit_steps = float((fit["cloud"][:, :, 3] / fit["cloud"][:, :, 0]).sum() * n_fit)
    # kappa: per-step time of the control-variate and plain kernels on these nodes
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).cuda() for j in range(dim)]
    rate = {}
    for name, gid in (("plain", pdd.PDD_CV_NONE), ("cv", w_slot)):
        prob.estimate(cols, 20000, 1e-3, grid_id=gid)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rr = prob.estimate(cols, 20000, 1e-3, grid_id=gid)
        torch.cuda.synchronize()
        rate[name] = float((rr["mean_steps"].cpu().numpy() * 20000).sum()) / (
            time.perf_counter() - t1)
    kappa = rate["plain"] / rate["cv"]
    a0 = args.a0
    # nodes inside the shrinkage layer at some h of the cloud cannot be fitted
    ok, fit, nodes = C.fitted_subset(fit, nodes)
    u = u[ok]
    a, sp = pdd.pdd_schedule(fit["K"], fit["beta"], fit["alpha"], fit["V_phi"], fit["V_psi"],
                             fit["rho_phi_psi"], 1.0, kappa, a0, max_levels=6)
    for j in range(len(a) - 1):  # level j reads the iterate of tolerance a[j+1]
        prob.set_control_grid(j, W.control_grid(kind, gn, a[j + 1] / 2.0))
    levels = C.plan_levels(fit, a)
    C.run_levels(prob, nodes, C.plan_levels(fit, a), n_pilot=200)  # warm-up (kernel loads)
    run = C.run_levels(prob, nodes, levels, e_tau=fit["E_tau"])
    summ = C.summary(levels, run, u, kappa, fit, a0)
    plain_lv = C.plan_levels(fit, [a0])
    C.run_levels(prob, nodes, C.plan_levels(fit, [a0]), n_pilot=200, n_max=1000)  # warm-up
    plain = C.run_levels(prob, nodes, plain_lv, e_tau=fit["E_tau"])
    plain_obs = plain["levels"][0]["path_steps"]
    where = ("576 nodes (every 16th) of the 3D problem, previous iterates v = u + (a_{j+1}/2) "
             "sin 3pi x sin 2pi y sin pi z on 65^3" if three_d else
             "256 nodes of the 2D problem, previous iterates v = u + (a_{j+1}/2) sin 3pi x "
             "sin 2pi y on 129^2")
    out = {"workload": args.workload, "metric": METRIC, "unit": UNIT, "dtype": "f32",
           "data": "synthetic",
           "value": (sum(o["path_steps"] for o in run["levels"])) / run["wall_s"],
           "config": {"workload": "Algorithm 4 schedule run as one launch (Algorithm 5 nodal "
                                  "loop), " + where + ", target a0",
                      "a0": a0, "q": 2.0, "delta": 1.0, "fit_paths_per_h": n_fit,
                      "fit_time_steps": 100, "nodes_fitted": int(ok.sum()),
                      "nodes_left_out": int((~ok).sum())},
           "fit": {"seconds": fit_s, "path_steps": fit_steps,
                   "median_beta": float(np.median(fit["beta"])),
                   "median_V_phi": float(np.median(fit["V_phi"])),
                   "median_E_tau": float(np.median(fit["E_tau"]))},
           "kappa": kappa,
           "schedule": {"tolerances": [float(x) for x in a],
                        "predicted_step_speedups": [float(x) for x in sp]},
           "levels": summ["rows"],
           "cascade": {"wall_s": run["wall_s"], "status": run["status"],
                       "pilot_wall_s": run["pilot_s"],
                       "pilot_path_steps": run["pilot_path_steps"],
                       "pred_cost": summ["pred_cost"], "obs_cost": summ["obs_cost"],
                       "pred_cumulative_speedup": summ["pred_cumulative_speedup"]},
           "plain_a0": {"wall_s": plain["wall_s"], "status": plain["status"],
                        "pred_path_steps": C.predicted_plain_steps(fit, a0),
                        "obs_path_steps": plain_obs,
                        "rmse_vs_exact": float(np.sqrt(np.mean(
                            (plain["levels"][0]["estimate"] - u) ** 2)))},
           "obs_cumulative_speedup": plain_obs / summ["obs_cost"],
           "wall_speedup": plain["wall_s"] / run["wall_s"]}
    prob.close()
    ctx.close()
    return out


def run_mlmc(args):
    """Multilevel Monte Carlo (pdd_mlmc) on the 256-node 2D workload at a fixed
    RMSE, plain and with the eps = 1e-2 control grid, against the single-level
    estimator at the multilevel run's finest step with the same node-mean
    variance budget (N = ceil(2 Vbar / a^2) from a pilot run).  Also on the
    nodes at least 0.1 from the boundary, where the weak-order-1 expansion
    that the stopping test assumes holds (near the boundary the level
    corrections of the Gobet-Menozzi scheme fall like sqrt(h))."""
    import numpy as np
    import torch

    from paper_1512_02818_gb300 import pdd
    from paper_1512_02818_gb300 import workloads as W
    ctx = pdd.Context(0)
    torch.cuda.set_stream(ctx.stream)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, GRID_N, 1e-2))
    all_nodes = W.workload_nodes("c1")
    interior = all_nodes[np.minimum(all_nodes, 1.0 - all_nodes).min(axis=1) >= 0.1]
    dev = torch.device("cuda", 0)
    a_t, dt0 = 1e-3, 1.6e-2
    clocks = ClockSampler(smi_id(0))
    modes = {}
    for name, gid, nodes in (("plain", pdd.PDD_CV_NONE, all_nodes), ("cv_eps1e-2", 0, all_nodes),
                             ("plain_interior", pdd.PDD_CV_NONE, interior),
                             ("cv_eps1e-2_interior", 0, interior)):
        cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).to(dev) for j in range(2)]
        u = W.exact_u(0, nodes.astype(np.float64))
        kw = dict(grid_id=gid, min_levels=2, max_levels=8, n_pilot=2000, stream_tag_base=300)
        prob.mlmc(nodes, dt0, a_t, **kw)  # warm-up (same work)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = prob.mlmc(nodes, dt0, a_t, **kw)
        secs = time.perf_counter() - t0
        hL = dt0 / 2 ** (r["n_levels"] - 1)
        # single level at h_L: pilot variance, then N for the same variance budget
        pilot = prob.estimate(cols, 20000, hL, grid_id=gid, stream_tag=500)
        vcol = "var_phi" if gid == pdd.PDD_CV_NONE else "var_cv"
        n_sl = int(np.ceil(2.0 * float(pilot[vcol].mean().item()) / a_t**2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sl = prob.estimate(cols, n_sl, hL, grid_id=gid, stream_tag=501)
        torch.cuda.synchronize()
        secs_sl = time.perf_counter() - t0
        mcol = "mean_phi" if gid == pdd.PDD_CV_NONE else "mean_cv"
        m_sl = sl[mcol].cpu().numpy()
        sl_steps = float((sl["mean_steps"].cpu().numpy() * n_sl).sum())
        modes[name] = {
            "nodes": int(len(nodes)),
            "status": int(r["status"]), "levels": int(r["n_levels"]), "rounds": int(r["rounds"]),
            "finest_dt": hL, "n_paths": [int(x) for x in r["n_paths"]],
            "var_mean": [float(x) for x in r["var_mean"]],
            "cost_mean": [float(x) for x in r["cost_mean"]],
            "bias_estimate": float(r["bias_estimate"]), "seconds": secs,
            "path_steps": int(r["path_steps"]), "nodes_per_s": len(nodes) / secs,
            "rmse_vs_exact": float(np.sqrt(np.mean((r["estimate"] - u) ** 2))),
            "extrapolated_rmse_vs_exact": float(np.sqrt(np.mean((r["extrapolated"] - u) ** 2))),
            "single_level": {"n_paths": n_sl, "seconds": secs_sl, "path_steps": sl_steps,
                             "nodes_per_s": len(nodes) / secs_sl,
                             "rmse_vs_exact": float(np.sqrt(np.mean((m_sl - u) ** 2)))},
            "speedup_vs_single_level": secs_sl / secs,
        }
    clk = clocks.stop()
    prob.close()
    ctx.close()
    return {"workload": "mlmc", "metric": METRIC, "value": modes["cv_eps1e-2"]["nodes_per_s"],
            "unit": "nodes/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "multilevel Monte Carlo on the 2D CFG0 problem, 256 nodes, "
                                   "target RMSE 1e-3, dt0 = 1.6e-2 halved per level (adaptive, "
                                   "2-8 levels), 2000 pilot paths, Gobet-Menozzi, alpha = 1; "
                                   "plain and eps = 1e-2 control grid 129^2; all nodes and the "
                                   "nodes >= 0.1 from the boundary"},
            "modes": modes, "clocks": clk}


def main():
    args = parse_args()
    rank, world, local = dist_info()
    if args.workload != "c1" and args.impl == "ours":
        if rank == 0:
            fn = {"c0": run_c0, "c2": run_c2, "c3": run_c3, "c4": run_c4,
                  "fit": run_fit, "mlmc": run_mlmc, "paper": run_paper,
                  "peaks": run_peaks, "cascade": run_cascade,
                  "cascade3d": run_cascade}[args.workload]
            print(json.dumps(fn(args)), flush=True)
        return
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
