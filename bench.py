#!/usr/bin/env python3
"""Benchmark of the sparse grid characteristics hot path on GB300.

One step = one pass of the whole path on the level-4 6-D attitude workload:
  Step I    sparse grid, d = 6, level 4 (1457 CGL nodes) on [-pi/4, pi/4]^6
  Step II   one characteristic BVP per node, T in {10, 20, 40} with N = 64 / 128
            / 256 Lobatto intervals, Newton to |F|_inf <= 1e-8 (mixed precision:
            FP32 Jacobian / elimination / direction; FP64 residual, boundary
            rows, line search and update)
  Step III  surpluses of u*(x) at the nodes
  on-line   u*(x) at 1e6 query states (half uniform, half N(0, 0.2^2) clipped),
            3xTF32 on the tensor cores (error against FP64 reported beside)
The headline value is converged BVP solves per second of whole-step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

Multi-GPU (torchrun): one job split over the ranks (paper_1507_04769_gb300/
sharded.py): each rank solves a contiguous node range of about equal cost, one
all-gather brings every node's result to every rank, the surpluses are built
replicated and the queries are split evenly.  Total work is fixed (strong
scaling); value = the job's converged solves / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "converged BVP solves/s at 1e-8 residual"
UNIT = "solves/s"
LEVEL, D = 4, 6
N_QUERIES = 1_000_000
E2E_EVAL_CHUNKS = 4        # e2e step: evaluation calls whose results go down while the next evaluates
TOL = 1e-8
SEG_LEN = 16   # intervals per segment of the library's segmented staircase

# dram__bytes_read.sum + dram__bytes_write.sum per unit of work from an ncu
# capture of the kernel as it stands (the 600-node solve case: the first Newton
# iteration, 88,064 intervals in one launch; profiles/
# solver_kernels_attitude6d_600nodes.md).  An entry is removed when its kernel
# changes, until it is captured again.
DRAM_BYTES_PER_UNIT = {
    "k_condense_reg_fp32": ((164.841728e6 + 417.7536e6) / 88064, "interval"),
}
WORKLOAD = ("attitude6d_L4_1457nodes_T{10,20,40}_N{64,128,256}_mixedprec"
            "+surplus+1e6queries_tf32x3")

# ALU peaks: the roofline divides by the FP32 / FP64 rates measured in the same
# run by the library's FMA-chain probe (sg_fma_probe); these derived figures
# are the fallback when no probe figure is given (unit counts x maximum SM
# clock, 2070 MHz, 152 SMs):
#   FP32: 128 FMA lanes/SM x 2 flops = 80.6 TFLOP/s
#   FP64: the nominal 1.25 TFLOP/s of GB300 (about 2 FMA/clk/SM)
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
PEAK_FP64_TFLOPS = 1.25


# ------------------------------------------------------------------ work model
def flops_condense_interval() -> float:
    """Per interval: build of the 36 x 49 system (1728 scaled Jacobian entries,
    36 residual rows of 4 FMA + 2) and Gaussian elimination of 24 columns with
    multipliers: sum_k (35-k) + 2 (35-k)(48-k), plus 24 reciprocals."""
    ge = sum((35 - k) + 2 * (35 - k) * (48 - k) for k in range(24)) + 24
    return 1728 + 36 * 10 + ge


def flops_abd_interval() -> float:
    """Per interval: elimination of 12 columns of the 18 x 25 panel, plus the
    back substitution (12 x 12 product and triangular solve)."""
    ge = sum((17 - k) + 2 * (17 - k) * (24 - k) for k in range(12)) + 12
    return ge + 2 * 144 + 144 + 12


def flops_abd_seg_interval() -> float:
    """Per interior mesh point of a segment: elimination of 12 columns of the
    24 x 37 panel [carry rows; block row] (36 - k columns updated in the
    23 - k rows left at step k, plus the multipliers)."""
    return float(sum((23 - k) + 2 * (23 - k) * (36 - k) for k in range(12)) + 12)


def flops_abd_segback_interval() -> float:
    """Per interior mesh point: two 12 x 12 products and a 12 x 12 triangular solve."""
    return 2 * 2 * 144 + 144 + 12


def flops_recover_interval() -> float:
    """Per interval: 24 x 24 product and 24 x 24 triangular solve."""
    return 2 * 576 + 576 + 24


def bytes_point(tsize: int) -> float:
    """Per collocation point: read y (12 f64), write F (12 f64) and J (144 x tsize)."""
    return 12 * 8 + 12 * 8 + 144 * tsize


def flops_eval_query(M: int, k: int) -> float:
    """Per query: the contraction (2 k flops per node) and one product per node."""
    return M * (2 * k + 1)


# ------------------------------------------------------------------ helpers
def _rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device) -> float:
    """Maximum of a per-rank scalar (seconds) over the process group; the
    identity without one. Timing only: the data path has no collective."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(n: int, device) -> int:
    """Sum of a per-rank count over the process group; the identity without
    one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(n)
    t = torch.tensor([int(n)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle worker
def _oracle_solve_node(job):
    """One oracle BVP solve (a process-pool task): returns converged flag."""
    from oracle import bvp as obvp
    from oracle import problems as oprob
    x0, T, N = job
    pr = oprob.make(synth.attitude_params(0))
    s = obvp.solve(pr, np.asarray(x0), float(T), int(N), tol=TOL, polish=False)
    return int(s.status == obvp.CONVERGED)


def stratified_sample(T, n_nodes: int, seed: int) -> np.ndarray:
    """n_nodes node indices drawn per horizon in the batch's proportions."""
    rng = np.random.default_rng(seed)
    out = []
    vals, counts = np.unique(T, return_counts=True)
    quota = np.floor(n_nodes * counts / counts.sum()).astype(int)
    quota[np.argsort(-(n_nodes * counts / counts.sum() - quota))[:n_nodes - quota.sum()]] += 1
    for v, q in zip(vals, quota):
        cand = np.flatnonzero(T == v)
        out += rng.choice(cand, min(q, cand.size), replace=False).tolist()
    return np.array(sorted(out))


def cpu_model() -> str:
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_worker(n_nodes: int, seed: int, procs: int = 1, steps: int = 1) -> dict:
    """Times the oracle on bounded samples of the workload: per step n_nodes
    BVP solves drawn from the level-4 nodes with their horizons (in the batch's
    horizon proportions), on `procs` processes (one thread each)."""
    from oracle import grid as ogrid
    lo, hi = synth.box(D)
    g = ogrid.Grid(D, LEVEL, lo, hi)
    T, N = synth.mixed_horizons(g.M, seed=2)
    pool = None
    if procs > 1:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(procs)
        pool.map(_oracle_solve_node, [(g.x[0], 1.0, 1)] * procs)   # start-up outside the timing
    per_step = []
    Ns = []
    try:
        for st in range(steps):
            idx = stratified_sample(T, n_nodes, seed + st)
            jobs = [(g.x[i], T[i], N[i]) for i in idx]
            t0 = time.perf_counter()
            if pool is None:
                conv = sum(_oracle_solve_node(j) for j in jobs)
            else:
                conv = sum(pool.map(_oracle_solve_node, jobs, chunksize=1))
            per_step.append({"converged": int(conv), "seconds": time.perf_counter() - t0})
            Ns += [int(N[i]) for i in idx]
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    conv = sum(p["converged"] for p in per_step)
    secs = sum(p["seconds"] for p in per_step)
    return {"converged": conv, "seconds": secs, "nodes": int(n_nodes) * steps, "procs": procs,
            "per_step": per_step, "N_counts": {str(k): Ns.count(k) for k in sorted(set(Ns))}}


def run_cpu_baseline(n_nodes: int, seed: int = 123, procs: int = 1, steps: int = 1) -> dict:
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    for v in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(v, None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", str(n_nodes), str(seed),
                        str(procs), str(steps)], capture_output=True, text=True, env=env, timeout=1200)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------ reference arm
def reference_arm(args):
    """The oracle timed on all host cores (one process per core, one thread
    each), each step a bounded stratified sample of the level-4 nodes."""
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    cores = host_cores()
    per_step = 8 * cores
    r = run_cpu_baseline(per_step, seed=1000, procs=cores, steps=args.warmup + args.steps)
    timed = r["per_step"][args.warmup:]
    total = sum(p["seconds"] for p in timed)
    conv = sum(p["converged"] for p in timed)
    value = conv / total
    sample = (f"{per_step} oracle BVP solves per step (level-4 nodes, horizons in the batch's proportions), "
              f"{cores} processes x 1 thread on {cpu_model()}, tol 1e-8")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def gpu_arm(args):
    import torch
    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1507_04769_gb300 import sg
    from paper_1507_04769_gb300 import sharded

    prec = {"mixed": sg.PREC_MIXED, "mixed-pair": sg.PREC_MIXED_PAIR, "fp64": sg.PREC_FP64}[args.precision]
    eval_mode = {"fp64": sg.EVAL_FP64, "df32": sg.EVAL_DF32, "tf32x3": sg.EVAL_TF32X3}[args.eval]
    lo, hi = synth.box(D)
    params = synth.attitude_params(0)
    prob = sg.problem_from(params)
    g0 = sg.Grid(D, LEVEL, lo, hi)
    M = g0.M
    T_h, N_h = synth.mixed_horizons(M, seed=2)
    # the job's split over the ranks: node ranges of about equal cost, even query ranges
    ranges = sharded.partition(sharded.node_costs(N_h), world)
    n0, n1 = ranges[rank]
    q0, q1 = sharded.even_range(N_QUERIES, rank, world)
    n_loc, q_loc = n1 - n0, q1 - q0
    xq_h = synth.mixed_queries(N_QUERIES, lo, hi, seed=1)[q0:q1]
    T_d = torch.as_tensor(T_h, device=dev)
    N_d = torch.as_tensor(N_h, dtype=torch.int32, device=dev)
    xq_d = torch.as_tensor(xq_h, device=dev)
    n_max = int(N_h.max())
    ws = torch.empty(max(sg.workspace_bytes(n_loc, n_max, prec), 1), dtype=torch.uint8, device=dev)
    u_out = torch.empty((q_loc, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # execution form of the solve: picked by the library's autotuner on this
    # batch (outside the timed region), or fixed from the command line
    x0_d = torch.empty((M, 6), dtype=torch.float64, device=dev)
    x0_d.copy_(g0.coords)
    tune_ms = None
    if args.only_steps:
        args.form = "phase"
        args.skip_cpu = args.skip_fp64 = args.skip_serving = args.skip_extensions = True
    if args.form == "auto":
        form, tune_ms = sg.autotune_solve(prob, x0_d[n0:n1], T_d[n0:n1], N_d[n0:n1], tol=TOL, precision=prec,
                                          n_max=n_max, workspace=ws)
    else:
        form = {"phase": dict(persistent=False, graph=0, blocks_per_sm=0),
                "phase-graph": dict(persistent=False, graph=1, blocks_per_sm=0),
                "phase-graph-per-mesh": dict(persistent=False, graph=2, blocks_per_sm=0),
                "persistent": dict(persistent=True, graph=1, blocks_per_sm=0)}[args.form]
    res_out = {"lambda0": torch.empty((n_loc, 6), dtype=torch.float64, device=dev),
               "u0": torch.empty((n_loc, 3), dtype=torch.float64, device=dev),
               "V": torch.empty((n_loc,), dtype=torch.float64, device=dev),
               "status": torch.empty((n_loc,), dtype=torch.int32, device=dev),
               "iters": torch.empty((n_loc,), dtype=torch.int32, device=dev)}

    def step(events=None, queries_ready=None, eval_chunks=1, after_chunk=None):
        if events:
            events[0].record(stream)
        g = sg.Grid(D, LEVEL, lo, hi)
        x0_d.copy_(g.coords)
        if events:
            events[1].record(stream)
        res = sharded.sharded_solve(prob, x0_d, T_d, N_d, ranges=ranges, tol=TOL, precision=prec, workspace=ws,
                                    n_max=n_max, out=res_out, **form)
        if events:
            events[2].record(stream)
        S = sg.Surplus(g, res["u0"])
        if events:
            events[3].record(stream)
        if queries_ready is not None:
            stream.wait_event(queries_ready)
        # the queries in eval_chunks consecutive calls (after_chunk(a, b) is
        # told of each one as it is queued)
        for c in range(eval_chunks):
            a, b = q_loc * c // eval_chunks, q_loc * (c + 1) // eval_chunks
            sg.eval_feedback(S, xq_d[a:b], mode=eval_mode, out=u_out[a:b])
            if after_chunk is not None:
                after_chunk(a, b)
        if events:
            events[4].record(stream)
        return res

    for _ in range(args.warmup):
        res = step()
        flush.zero_()
    torch.cuda.synchronize()
    status = res["status"].cpu().numpy()
    iters = res["iters"].cpu().numpy().astype(np.int64)
    conv_per_step = int(np.sum(status == sg.CONVERGED))   # the whole job's (results are gathered)

    # ---------------- timed region
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = sg.LIB.sg_kernel_launches()
    sg.LIB.sg_timing_enable(1)
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            res = step(ev[s])
            flush.zero_()
        torch.cuda.synchronize()
    sg.LIB.sg_timing_enable(0)
    launches = sg.LIB.sg_kernel_launches() - launches0
    kt = collect_kernel_times(sg)
    kt_form = "timed region"
    if form.get("graph") or form.get("persistent"):
        # inside a graph the library's per-launch events see only the graph
        # launch; a second timed region runs the same kernels one launch per
        # phase for the per-kernel durations and the executed-kernel count
        phase = dict(form, persistent=False, graph=0, blocks_per_sm=0)
        for _ in range(2):
            sharded.sharded_solve(prob, x0_d, T_d, N_d, ranges=ranges, tol=TOL, precision=prec, workspace=ws,
                                  n_max=n_max, out=res_out, **phase)
        torch.cuda.synchronize()
        la = sg.LIB.sg_kernel_launches()
        sg.LIB.sg_timing_enable(1)
        for _ in range(args.steps):
            g = sg.Grid(D, LEVEL, lo, hi)
            x0_d.copy_(g.coords)
            r2 = sharded.sharded_solve(prob, x0_d, T_d, N_d, ranges=ranges, tol=TOL, precision=prec,
                                       workspace=ws, n_max=n_max, out=res_out, **phase)
            S2 = sg.Surplus(g, r2["u0"])
            sg.eval_feedback(S2, xq_d, mode=eval_mode, out=u_out)
            flush.zero_()
        torch.cuda.synchronize()
        sg.LIB.sg_timing_enable(0)
        launches = sg.LIB.sg_kernel_launches() - la
        kt = collect_kernel_times(sg)
        kt_form = "second timed region, same kernels launched one per phase"
    # FP64 / FP32 pipe peaks of this GPU, measured now, for the roofline fractions
    # (not in the launch-list mode, whose launches should be the step's alone)
    probe = measure_pipe_peaks(sg, stream, local) if not args.only_steps else {}
    step_ms = [ev[s][0].elapsed_time(ev[s][4]) for s in range(args.steps)]
    phase_ms = {name: sum(ev[s][i].elapsed_time(ev[s][i + 1]) for s in range(args.steps)) / args.steps
                for i, name in enumerate(["grid", "solve", "surplus", "eval"])}
    t_max = max_over_ranks(sum(step_ms) / 1e3, dev)
    total_solves = conv_per_step * args.steps
    value = total_solves / t_max

    if args.only_steps:
        roof, kernels = roofline(kt, iters[n0:n1], N_h[n0:n1], M, prec, q_loc, probe)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": total_solves / t_max, "unit": UNIT,
                              "only_steps": True, "ms_per_step": 1e3 * t_max / args.steps, "roofline": roof,
                              "kernels": kernels}), flush=True)
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    # ---------------- end to end through the public API with host buffers
    T_pin = torch.as_tensor(T_h).pin_memory()
    N_pin = torch.as_tensor(N_h, dtype=torch.int32).pin_memory()
    xq_pin = torch.as_tensor(xq_h).pin_memory()
    u_pin = torch.empty((q_loc, 3), dtype=torch.float64).pin_memory()
    node_pin = {k: torch.empty((M,) + shp, dtype=dt).pin_memory()
                for k, shp, dt in (("lambda0", (6,), torch.float64), ("u0", (3,), torch.float64),
                                   ("V", (), torch.float64), ("status", (), torch.int32))}

    # The queries are uploaded on a second stream while the grid, the solves and
    # the surpluses run; the evaluation waits for them.  It runs in E2E_EVAL_CHUNKS
    # calls, and each chunk's feedback goes down on a third stream while the next
    # one evaluates; the step ends when the last copy has landed.
    up_stream = torch.cuda.Stream(device=dev)
    down_stream = torch.cuda.Stream(device=dev)
    xq_ready = torch.cuda.Event()

    def chunk_down(a, b):
        ev = torch.cuda.Event()
        ev.record(stream)
        down_stream.wait_event(ev)
        with torch.cuda.stream(down_stream):
            u_pin[a:b].copy_(u_out[a:b], non_blocking=True)

    def e2e_step():
        T_d.copy_(T_pin, non_blocking=True)
        N_d.copy_(N_pin, non_blocking=True)
        up_stream.wait_stream(stream)   # the previous step's evaluation has read xq_d
        with torch.cuda.stream(up_stream):
            xq_d.copy_(xq_pin, non_blocking=True)
            xq_ready.record(up_stream)
        r = step(queries_ready=xq_ready, eval_chunks=E2E_EVAL_CHUNKS, after_chunk=chunk_down)
        for k in node_pin:
            node_pin[k].copy_(r[k], non_blocking=True)
        stream.wait_stream(down_stream)
        return r

    for _ in range(2):
        e2e_step()
        flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    for s in range(args.steps):
        e2e_ev[s][0].record(stream)
        e2e_step()
        e2e_ev[s][1].record(stream)
        torch.cuda.synchronize()
        flush.zero_()
    torch.cuda.synchronize()
    e2e_t = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev) / 1e3, dev)
    h2d = T_pin.numel() * 8 + N_pin.numel() * 4 + xq_pin.numel() * 8
    d2h = u_pin.numel() * 8 + sum(t.numel() * t.element_size() for t in node_pin.values())
    e2e_value = conv_per_step * args.steps / e2e_t

    # ---------------- FP64 form on the same GPU (speedup of the mixed form)
    fp64 = None
    if prec != sg.PREC_FP64 and not args.skip_fp64 and n_loc > 0:
        ws64 = torch.empty(max(sg.workspace_bytes(n_loc, n_max, sg.PREC_FP64), 1), dtype=torch.uint8, device=dev)
        g = sg.Grid(D, LEVEL, lo, hi)
        r64 = sg.solve_bvps(prob, g.coords[n0:n1], T_d[n0:n1], N_d[n0:n1], tol=TOL, precision=sg.PREC_FP64, workspace=ws64,
                            n_max=n_max)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            r64 = sg.solve_bvps(prob, g.coords[n0:n1], T_d[n0:n1], N_d[n0:n1], tol=TOL, precision=sg.PREC_FP64, workspace=ws64,
                                n_max=n_max)
        b.record(stream)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b) / 1e3 / args.steps
        c64 = int((r64["status"] == sg.CONVERGED).sum().item())
        # per-kernel times of the FP64 form (one launch per phase) for its roofline
        sg.LIB.sg_timing_enable(1)
        r64 = sg.solve_bvps(prob, g.coords[n0:n1], T_d[n0:n1], N_d[n0:n1], tol=TOL, precision=sg.PREC_FP64, workspace=ws64,
                            n_max=n_max)
        torch.cuda.synchronize()
        sg.LIB.sg_timing_enable(0)
        kt64 = collect_kernel_times(sg)
        it64 = r64["iters"].cpu().numpy().astype(np.int64)
        _, kern64 = roofline(kt64, it64, N_h[n0:n1], M, sg.PREC_FP64, q_loc, probe)
        mixed_solve_s = phase_ms["solve"] / 1e3
        dl = (r64["lambda0"] - res["lambda0"][n0:n1]).abs().max().item() / r64["lambda0"].abs().max().item()
        fp64 = {"solves_per_s": c64 / t64, "solve_ms": 1e3 * t64,
                "mixed_solve_ms": 1e3 * mixed_solve_s, "speedup_mixed_over_fp64": t64 / mixed_solve_s,
                "max_rel_diff_lambda0_mixed_vs_fp64": dl,
                "newton_iters_hist_fp64": np.bincount(r64["iters"].cpu().numpy()).tolist(),
                "kernels": dict(list(kern64.items())[:5])}
        # the other FP32-direction form (residual in FP64, or in pairs of
        # floats), in the timed form's execution form, on its workspace
        other = sg.PREC_MIXED_PAIR if prec == sg.PREC_MIXED else sg.PREC_MIXED
        rr = sg.solve_bvps(prob, g.coords[n0:n1], T_d[n0:n1], N_d[n0:n1], tol=TOL, precision=other, workspace=ws,
                           n_max=n_max, **form)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            rr = sg.solve_bvps(prob, g.coords[n0:n1], T_d[n0:n1], N_d[n0:n1], tol=TOL, precision=other, workspace=ws,
                               n_max=n_max, **form)
        b.record(stream)
        torch.cuda.synchronize()
        tr = a.elapsed_time(b) / 1e3 / args.steps
        cr = int((rr["status"] == sg.CONVERGED).sum().item())
        dr = (r64["lambda0"] - rr["lambda0"]).abs().max().item() / r64["lambda0"].abs().max().item()
        fp64["mixed_pair_residual" if other == sg.PREC_MIXED_PAIR else "mixed_fp64_residual"] = {
            "solves_per_s": cr / tr, "solve_ms": 1e3 * tr, "speedup_over_fp64": t64 / tr,
            "max_rel_diff_lambda0_vs_fp64": dr,
            "newton_iters_hist": np.bincount(rr["iters"].cpu().numpy()).tolist()}
        del ws64

    # ---------------- interpolant modes on the 1e6 queries (FP64, DF32, 3xTF32)
    eval_modes = {}
    if rank == 0:
        S_ref = sg.Surplus(g0, res["u0"])
        ref = sg.eval_feedback(S_ref, xq_d, mode=sg.EVAL_FP64)
        for name, md in (("fp64", sg.EVAL_FP64), ("df32", sg.EVAL_DF32), ("tf32x3", sg.EVAL_TF32X3)):
            outm = torch.empty_like(ref)
            for _ in range(2):
                sg.eval_feedback(S_ref, xq_d, mode=md, out=outm)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            sg.eval_feedback(S_ref, xq_d, mode=md, out=outm)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            err = ((outm - ref).abs().max() / ref.abs().max()).item()
            eval_modes[name] = {"ms_per_1e6": ms * 1e6 / q_loc, "evals_per_s": q_loc / (ms / 1e3),
                                "max_rel_err_vs_fp64": err}

    # ---------------- Example III: value function on the q = 12 grid in (t, x)
    # (18,945 nodes), against the printed closed form; and the Monte-Carlo
    # error amplification of Section 4.2 at q = 13, d = 6 (44,689 nodes)
    extensions = None
    if rank == 0 and not args.skip_extensions:
        from paper_1507_04769_gb300 import timegrid
        lo3, hi3 = synth.example3_box()
        prm3 = synth.example3_params()
        # a small surface first, so that first-use costs (module loading, the
        # first calls of the tensor operations the surface code uses) stay out
        # of the timed build
        timegrid.solve_value_surface(sg.problem_from(prm3), 3, 4, lo3, hi3, prm3.t_end, synth.example3_mesh,
                                     precision=prec, tol=TOL)
        torch.cuda.synchronize()
        a3, b3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a3.record(stream)
        vs = timegrid.solve_value_surface(sg.problem_from(prm3), 3, 8, lo3, hi3, prm3.t_end, synth.example3_mesh,
                                          precision=prec, tol=TOL)
        b3.record(stream)
        torch.cuda.synchronize()
        tx = synth.uniform_queries(1200, lo3, hi3, seed=5)
        out3 = vs.evaluate(torch.as_tensor(tx, device=dev)).cpu().numpy()
        tau3, x3 = prm3.t_end - tx[:, 0], tx[:, 1:].T
        g3 = 1.0 + x3[0] ** 2 + x3[1] ** 2
        e3 = out3[:, 0] - 0.5 * x3[2] ** 2 / g3 ** 2 * np.tanh(tau3)
        # Section 4.1: e_interp + e_bvp of the level-4 feedback at one horizon
        # (T = 20, N = 128), against error-controlled solves at 1,280 random states
        from paper_1507_04769_gb300 import validation as val
        gv = sg.Grid(D, LEVEL, lo, hi)
        rv = sg.solve_bvps(prob, gv.coords, torch.full((gv.M,), 20.0, dtype=torch.float64, device=dev),
                           torch.full((gv.M,), 128, dtype=torch.int32, device=dev), tol=1e-10, precision=prec)
        pts = torch.as_tensor(synth.uniform_queries(1280, lo, hi, seed=31), device=dev)
        a4, b4 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a4.record(stream)
        vres = val.validate_feedback(prob, sg.Surplus(gv, rv["u0"]), pts, 20.0, tol=1e-9)
        b4.record(stream)
        torch.cuda.synchronize()
        # Example II: the two-wheel attitude problem at q = 13 (44,689 nodes,
        # per-node target attitudes), V validated at 1,280 random states
        from paper_1507_04769_gb300 import surfaces
        prm2 = synth.example2_params()
        lo2, hi2 = synth.example2_box()
        a5, b5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a5.record(stream)
        srf2 = surfaces.two_wheel_surface(prm2, 7, lo2, hi2, synth.EXAMPLE2_T, precision=prec, tol=TOL)
        b5.record(stream)
        torch.cuda.synchronize()
        pts2 = torch.as_tensor(synth.uniform_queries(1280, lo2, hi2, seed=51), device=dev)
        tgt2, _ = sg.attitude_targets(sg.problem_from(prm2), pts2)
        v2 = val.validate_value(sg.problem_from(prm2), srf2.surplus, pts2, synth.EXAMPLE2_T, 1e-9, value_col=2,
                                target=tgt2)
        extensions = {
            "example2_q13": dict(v2.stats(0), nodes=srf2.grid.M, continued_nodes=srf2.continued,
                                 targets_solves_surplus_ms=a5.elapsed_time(b5), reference_tol=1e-9,
                                 paper={"relative_mae_V": 8.5e-3}),
            "validation_attitude_L4_T20": dict(vres.stats(0), reference_tol=1e-9, component="u1",
                                               ms=a4.elapsed_time(b4),
                                               all_components_mae=[vres.stats(c)["mae"] for c in range(3)]),
            "example3_q12": {"nodes": vs.grid.M, "t_end": prm3.t_end, "solve_and_surplus_ms": a3.elapsed_time(b3),
                             "newton_iters_hist": np.bincount(vs.result["iters"].cpu().numpy()).tolist(),
                             "continued_nodes": vs.continued, "points": 1200,
                             "mae_V": float(np.abs(e3).mean()), "var_V": float(np.var(e3)),
                             "paper": {"mae_V": 8.5e-4, "var_V": 2.8e-6}},
            "error_amplification_q13_d6": {
                "theorem1_bound": sg.theorem1_bound(6, 13),
                "monte_carlo_uniform_0_1": sg.mc_error_amplification(6, 7, 2000, seed=0),
                "monte_carlo_uniform_m1_1": sg.mc_error_amplification(6, 7, 2000, seed=0, symmetric=True),
                "points": 2000, "paper": {"theorem1_bound": 3.66e4, "monte_carlo": 66.60}},
        }

    # ---------------- serving: Poisson-arriving mixed requests, continuous batching,
    # swept over arrival rates to the knee of the p99 latency
    serving_rep = None
    if not args.skip_serving and rank == 0:
        from paper_1507_04769_gb300 import serving as srv
        server = srv.Server(slots=4, memory_budget=64 << 30, precision=prec, eval_mode=eval_mode)
        keys = [(2, 20.0), (3, 20.0), (4, 20.0)]
        counts = server.warm(levels=(2, 3, 4, 5), model_keys=keys)
        sweep = []
        for i, rate in enumerate(args.serve_rates):
            reqs = srv.make_requests(args.serve_requests, rate=rate, node_counts=counts, seed=11 + i,
                                     model_keys=keys)
            server.start()
            it0 = server.pool_iterations
            t0 = time.perf_counter()
            done = srv.replay(server, reqs, realtime=True)
            sweep.append({"arrival_rate_per_s": rate, "requests": len(done), "wall_s": time.perf_counter() - t0,
                          "pool_iterations": server.pool_iterations - it0,
                          "latency": srv.latency_report(done)})
        p99 = [e["latency"]["all"]["p99_ms"] for e in sweep]
        knee = next((sweep[i]["arrival_rate_per_s"] for i in range(1, len(sweep)) if p99[i] > 2.0 * p99[0]), None)
        serving_rep = {"slots": 4, "memory_budget_gb": 64, "pool_slots": srv.POOL_SLOTS,
                       "pool_gb": server.pool.nbytes / 2 ** 30, "sweep": sweep,
                       "p99_knee_rate_per_s": knee,
                       "sizes": "bvp 1..4096 states (full grid of level 2..5 when the draw reaches it), "
                                "T in {10,20,40}; eval 1..1e5 queries; sim 1..1024 trajectories x 2000 steps",
                       "batching": "bvp: solves share Newton iterations of the resident pool (mean_batch = "
                                   "requests in the pool together); eval/sim: merged launches"}
        del server
        torch.cuda.synchronize()

    # ---------------- roofline of the dominant kernel
    roof, kernels = roofline(kt, iters[n0:n1], N_h[n0:n1], M, prec, q_loc, probe)
    eval_ms_max = max_over_ranks(phase_ms["eval"], dev)   # every rank's share of the queries

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    cpu = None
    if world == 1 and not args.skip_cpu:
        # the oracle on every host core over the whole level-4 batch, and on
        # one core over a stratified sample of it
        cores = host_cores()
        model = cpu_model()
        r_all = run_cpu_baseline(M, seed=0, procs=cores)
        r_one = run_cpu_baseline(args.cpu_nodes, seed=123)
        cpu = {"value": r_all["converged"] / r_all["seconds"], "unit": UNIT, "cores": cores, "kind": "oracle",
               "cpu_model": model,
               "sample": f"all {M} level-4 nodes (N counts {r_all['N_counts']}) solved by the oracle to "
                         f"|F|_inf <= 1e-8 on {cores} processes x 1 thread ({model}), "
                         f"{r_all['seconds']:.1f} s",
               "single_core": {"value": r_one["converged"] / r_one["seconds"], "unit": UNIT, "cores": 1,
                               "sample": f"{args.cpu_nodes} of the nodes (N counts {r_one['N_counts']}), "
                                         f"{r_one['seconds']:.1f} s"}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None,
        "dtype": "f64+f32" if prec != sg.PREC_FP64 else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nodes": M, "grid_level": LEVEL, "d": D,
                   "horizons": "T in {10,20,40}, N = 6.4 T", "queries": N_QUERIES, "tol": TOL,
                   "precision": {"mixed": "FP32 Jacobian, elimination and direction; FP64 residual, "
                                           "boundary rows, line search and update",
                                 "mixed-pair": "FP32 direction; pair-of-floats residual; FP64 line search and update",
                                 "fp64": "FP64 throughout"}[args.precision],
                   "eval": args.eval,
                   "solve_form": form, "autotune_ms": tune_ms,
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": (f"{world} rank(s), one job: node ranges of equal cost, one all-gather of "
                                   "per-node results, surpluses replicated, queries split evenly")},
        "feedback_evals_per_s": N_QUERIES / (eval_ms_max / 1e3),
        "breakdown_ms": phase_ms,
        "newton_iters_hist": np.bincount(iters).tolist(),
        "converged_per_step": conv_per_step,
        "roofline": roof,
        "kernels": kernels,
        "kernel_timing": kt_form,
        "fp64_form": fp64,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_t / args.steps},
        "eval_modes": eval_modes,
        "pipe_peaks_probe": probe,
        "serving": serving_rep,
        "extensions": extensions,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def measure_pipe_peaks(sg, stream, gpu_index) -> dict:
    """FP64 and FP32 FMA rates of this GPU from the library's FMA-chain probe
    (152 x 8 blocks of 256 threads, dependent FMA chains), the best of three
    runs each, with the SM clocks sampled while it runs."""
    import ctypes as C
    import torch
    scratch = torch.empty(152 * 8 * 256 * 8, dtype=torch.uint8, device=torch.device("cuda", gpu_index))
    sg.LIB.sg_fma_probe.argtypes = [C.c_int, C.c_void_p, C.c_size_t, C.c_int, C.c_int, C.c_int,
                                    C.POINTER(C.c_double), C.c_void_p]
    probe = {}
    with ClockSampler(gpu_index) as clk:
        for name, pr, n_it in (("fp64", sg.PREC_FP64, 256), ("fp32", sg.PREC_MIXED, 4096)):
            fl = C.c_double()
            best = 0.0
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sg.LIB.sg_fma_probe(pr, C.c_void_p(scratch.data_ptr()), scratch.numel(), 152 * 8, 256, n_it,
                                    C.byref(fl), C.c_void_p(stream.cuda_stream))
                b.record(stream)
                torch.cuda.synchronize()
                best = max(best, fl.value / (a.elapsed_time(b) / 1e3) / 1e12)
            probe[name + "_tflops"] = best
    probe["clocks"] = clk.summary()
    return probe


def collect_kernel_times(sg):
    import ctypes as C
    n_max, name_len = 64, 64
    names = C.create_string_buffer(n_max * name_len)
    ms = (C.c_double * n_max)()
    cnt = (C.c_int64 * n_max)()
    nk = C.c_int()
    sg.LIB.sg_timing_collect.argtypes = [C.c_int, C.c_char_p, C.c_int, C.c_void_p, C.c_void_p,
                                         C.POINTER(C.c_int)]
    rc = sg.LIB.sg_timing_collect(n_max, names, name_len, C.cast(ms, C.c_void_p), C.cast(cnt, C.c_void_p),
                                  C.byref(nk))
    if rc != 0:
        raise RuntimeError(sg.LIB.sg_last_error().decode())
    out = {}
    raw = names.raw
    for i in range(nk.value):
        nm = raw[i * name_len:(i + 1) * name_len].split(b"\0", 1)[0].decode()
        out[nm] = (ms[i], cnt[i])
    return out


def roofline(kt, iters, N_h, M, prec, nq=N_QUERIES, peaks=None):
    """Per-kernel algorithmic work / measured time; the dominant kernel's entry
    is the roofline object.  iters and N_h are those of the nodes this rank
    solved; nq is the number of queries it evaluated per step.  peaks: the
    probe's measured {"fp32_tflops", "fp64_tflops"} (derived figures when
    absent)."""
    peaks = peaks or {}
    pk32 = peaks.get("fp32_tflops") or PEAK_FP32_TFLOPS
    pk64 = peaks.get("fp64_tflops") or PEAK_FP64_TFLOPS
    measured = bool(peaks.get("fp32_tflops")) and bool(peaks.get("fp64_tflops"))
    fp32 = prec != 0   # any form but SG_PREC_FP64 runs the direction in FP32
    suffix = "_fp32" if fp32 else "_fp64"
    tsize = 4 if fp32 else 8
    peak_lin = pk32 if fp32 else pk64
    int_units = float(np.sum(iters * N_h))           # interval-iterations per solve
    pt_units = float(np.sum(iters * (3 * N_h + 1)))  # point-iterations per solve
    seg = -(-N_h // SEG_LEN)                            # segments per node
    seg_units = float(np.sum(iters * (N_h - seg)))      # interior segment points (panels)
    red_units = float(np.sum(iters * seg))              # reduced block rows
    steps_timed = None
    models = {
        "k_condense" + suffix: ("alu", flops_condense_interval() * int_units, peak_lin, "TFLOP/s"),
        "k_condense_reg_fp32": ("alu", flops_condense_interval() * int_units, pk32, "TFLOP/s"),
        "k_abd" + suffix: ("alu", flops_abd_interval() * int_units, peak_lin, "TFLOP/s"),
        "k_abd_seg" + suffix: ("alu", flops_abd_seg_interval() * seg_units, peak_lin, "TFLOP/s"),
        "k_abd_red" + suffix: ("alu", flops_abd_interval() * red_units, peak_lin, "TFLOP/s"),
        "k_abd_segback" + suffix: ("alu", flops_abd_segback_interval() * seg_units, peak_lin, "TFLOP/s"),
        "k_recover" + suffix: ("alu", flops_recover_interval() * int_units, peak_lin, "TFLOP/s"),
        "k_newton_persistent" + suffix: ("alu", (flops_condense_interval() + flops_abd_interval()
                                                  + flops_recover_interval()) * int_units, peak_lin, "TFLOP/s"),
        "k_point" + suffix: ("hbm", bytes_point(tsize) * pt_units, None, "GB/s"),
        "k_condense_smem_fp64": ("alu", flops_condense_interval() * int_units, pk64, "TFLOP/s"),
        # the interpolant: the method's M (2k + 1) flops per query whatever the
        # arithmetic (pairs of floats and split TF32 do more operations)
        "k_eval_fp64": ("alu", flops_eval_query(M, 3) * nq, pk64, "TFLOP/s"),
        "k_eval_df32": ("alu", flops_eval_query(M, 3) * nq, pk32, "TFLOP/s"),
        "k_eval_tf32x3": ("alu", flops_eval_query(M, 3) * nq, pk32, "TFLOP/s"),
        "k_eval_sf_tf32x3": ("alu", flops_eval_query(M, 3) * nq, pk32, "TFLOP/s"),
    }
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak = 6785.9
    if os.path.exists(peaks_path):
        try:
            hbm_peak = float(json.load(open(peaks_path))["hbm_gbs"])
        except (KeyError, ValueError):
            pass
    kernels = {}
    total_ms = sum(v[0] for v in kt.values()) or 1.0
    for name, (ms, n) in sorted(kt.items(), key=lambda kv: -kv[1][0]):
        entry = {"total_ms": ms, "launches": int(n), "share": ms / total_ms}
        if name in models and n > 0:
            bound, work_per_solve, peak, unit = models[name]
            # every timed step repeats the same solve (work per step = work_per_solve)
            if name.startswith("k_eval"):
                work_total = work_per_solve * n
            else:
                steps_timed = steps_timed or max(1, round(kt.get("k_outputs", (0, 1))[1]))
                work_total = work_per_solve * steps_timed
            sec = ms / 1e3
            if unit == "TFLOP/s":
                achieved = work_total / sec / 1e12
            else:
                achieved = work_total / sec / 1e9
                peak = hbm_peak
            entry.update({"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                          "frac": achieved / peak})
        kernels[name] = entry
    dom = next((k for k in kernels if "achieved" in kernels[k]), None)
    roof = None
    if dom:
        e = kernels[dom]
        traffic = None
        if dom in DRAM_BYTES_PER_UNIT and e["launches"] > 0:
            # DRAM bytes per unit from one ncu capture of the same kernel on a
            # smaller case, times the units of an average timed launch
            per_unit, unit_kind = DRAM_BYTES_PER_UNIT[dom]
            units = {"interval": int_units}[unit_kind] * (steps_timed or 1)
            traffic = per_unit * units / e["launches"]
        roof = {"kernel": dom, "bound": e["bound"], "achieved": e["achieved"], "peak": e["peak"],
                "unit": e["unit"], "frac": e["frac"], "traffic": traffic,
                "peak_source": ("MEASURED_PEAKS.json hbm_gbs" if e["unit"] != "TFLOP/s" else
                                "measured in this run: FMA-chain probe (sg_fma_probe), "
                                + ("FP32" if e["peak"] == pk32 else "FP64") if measured else
                                "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz" if e["peak"] == pk32 else
                                "nominal GB300 FP64 1.25 TFLOP/s"),
                "share_of_gpu_time": e["share"]}
    return roof, kernels


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--precision", choices=["mixed", "mixed-pair", "fp64"], default="mixed",
                    help="mixed: FP32 direction, FP64 residual; mixed-pair: the residual in pairs of floats")
    ap.add_argument("--eval", choices=["df32", "fp64", "tf32x3"], default="tf32x3",
                    help="interpolant arithmetic: 3xTF32 on the tensor cores (the precision form), "
                         "DF32 (FP64-accurate on the FP32 pipe) or FP64")
    ap.add_argument("--form", choices=["auto", "phase", "phase-graph", "phase-graph-per-mesh", "persistent"],
                    default="auto",
                    help="execution form of the solve (auto: the library's autotuner picks)")
    ap.add_argument("--cpu-nodes", type=int, default=60, help="nodes of the single-core oracle sample")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-extensions", action="store_true",
                    help="skip the Example III value surface and the error-amplification estimates")
    ap.add_argument("--only-steps", action="store_true",
                    help="warm-up and timed steps only, one launch per phase (for kernel launch lists)")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[10.0, 25.0, 50.0, 100.0, 200.0],
                    help="arrival rates (requests/s) of the serving sweep")
    ap.add_argument("--serve-requests", type=int, default=100, help="requests per rate of the sweep")
    ap.add_argument("--cpu-worker", nargs=4, type=int, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_worker is not None:
        print(json.dumps(cpu_worker(*args.cpu_worker)))
        return 0
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
