"""Host-side logic of bench.py: the N > 1 path on CPU with gloo ranks, and the
reference arm's JSON line (the oracle timed on a bounded sample)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank seconds: the job time is the slowest rank's
        t = bench.max_over_ranks(1.0 + rank, torch.device("cpu"))
        n = bench.sum_over_ranks(100 + rank, torch.device("cpu"))
        # the bench's split of the level-4 job: node and query ranges of this rank
        import synth
        from paper_1507_04769_gb300 import sharded
        _, N = synth.mixed_horizons(1457, seed=2)
        nodes = sharded.partition(sharded.node_costs(N), world)[rank]
        queries = sharded.even_range(bench.N_QUERIES, rank, world)
        dist.barrier()
        q.put((rank, t, n, nodes, queries))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing_and_counts():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(world))
    assert [o[1] for o in out] == [2.0, 2.0]          # max over ranks
    assert [o[2] for o in out] == [201, 201]          # sum over ranks
    # the ranks split one job: node ranges and query ranges tile the whole
    assert out[0][3][0] == 0 and out[0][3][1] == out[1][3][0] and out[1][3][1] == 1457
    assert out[0][4] == (0, 500_000) and out[1][4] == (500_000, 1_000_000)


def test_helpers_without_process_group():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.sum_over_ranks(7, torch.device("cpu")) == 7


def _run_bench(args, env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True,
                          text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def bench_host_cores():
    sys.path.insert(0, ROOT)
    import bench
    return bench.host_cores()


@pytest.mark.slow
def test_reference_arm_json_line():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {})
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line
    assert line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == bench_host_cores()
    assert line["cpu_baseline"]["cpu_model"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]


def test_roofline_arithmetic_on_synthetic_kernel_times():
    """The bench's roofline object: the top modelled kernel, achieved = its
    algorithmic work / its time, frac = achieved / peak, and the DRAM traffic
    per launch from the captured bytes per interval."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    iters = np.array([5, 6, 4])
    N_h = np.array([64, 128, 256])
    M = 3
    int_units = float(np.sum(iters * N_h))
    # one timed step: 6 condensation launches in 12 ms, the outputs kernel once
    kt = {"k_condense_reg_fp32": (12.0, 6), "k_recover_fp32": (3.0, 6), "k_outputs": (0.1, 1),
          "k_ls_begin": (0.2, 6)}
    for prec in (1, 2):   # both FP32-direction forms
        roof, kernels = bench.roofline(kt, iters, N_h, M, prec)
        assert roof["kernel"] == "k_condense_reg_fp32" and roof["bound"] == "alu"
        work = bench.flops_condense_interval() * int_units
        assert abs(roof["achieved"] - work / 12e-3 / 1e12) <= 1e-9 * roof["achieved"]
        assert roof["peak"] == bench.PEAK_FP32_TFLOPS
        assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) <= 1e-12
        per_unit, kind = bench.DRAM_BYTES_PER_UNIT["k_condense_reg_fp32"]
        assert kind == "interval" and abs(roof["traffic"] - per_unit * int_units / 6) <= 1e-6 * roof["traffic"]
        assert abs(sum(k["share"] for k in kernels.values()) - 1.0) <= 1e-12
        assert "achieved" not in kernels["k_ls_begin"]   # unmodelled kernels carry time and share only
    # with the probe's measured rates the fractions divide by them
    roof_p, _ = bench.roofline(kt, iters, N_h, M, 1, peaks={"fp32_tflops": 70.0, "fp64_tflops": 1.0})
    assert roof_p["peak"] == 70.0 and "probe" in roof_p["peak_source"]
    assert abs(roof_p["frac"] - roof_p["achieved"] / 70.0) <= 1e-12
    # the interpolant's work is the method's M (2k + 1) flops per query in every mode
    kte = {"k_eval_df32": (3.0, 1)}
    _, ke = bench.roofline(kte, iters, N_h, 1457, 1, nq=1000, peaks={"fp32_tflops": 70.0, "fp64_tflops": 1.0})
    assert abs(ke["k_eval_df32"]["achieved"] - 1457 * 7 * 1000 / 3e-3 / 1e12) <= 1e-12
    # the FP64 form takes the FP64 kernels' models and peak
    kt64 = {"k_condense_smem_fp64": (70.0, 6), "k_outputs": (0.1, 1)}
    roof64, _ = bench.roofline(kt64, iters, N_h, M, 0)
    assert roof64["kernel"] == "k_condense_smem_fp64" and roof64["peak"] == bench.PEAK_FP64_TFLOPS
    assert roof64["traffic"] is None
