"""The multi-GPU split of one solve (sharded.py) on CPU ranks with gloo.

Partition: contiguous node ranges balanced by cost (N x expected iterations),
each node in exactly one range.  Sharded solve: each rank solves its range,
one all-gather returns every node's results to every rank in node order; the
result is bitwise the one-rank result.  Queries: contiguous equal ranges.
The per-range solver here is the oracle (the CUDA solver needs a GPU), which
is what makes the one-rank and two-rank runs comparable on the CPU.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1507_04769_gb300 import sharded  # noqa: E402


# ------------------------------------------------------------------ partition
def test_partition_covers_every_node_once_and_balances_cost():
    rng = np.random.default_rng(0)
    N = rng.choice([64, 128, 256], size=1457)
    for world in (1, 2, 3, 4, 8):
        r = sharded.partition(sharded.node_costs(N), world)
        assert len(r) == world and r[0][0] == 0 and r[-1][1] == len(N)
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))          # contiguous, no gap or overlap
        share = np.array([N[s:e].sum() for s, e in r]) / N.sum()
        assert share.max() <= 1.0 / world + N.max() / N.sum()       # within one node of even


def test_partition_edge_cases():
    assert sharded.partition([], 3) == [(0, 0)] * 3
    assert sharded.partition([5.0], 4) == [(0, 1), (1, 1), (1, 1), (1, 1)]
    r = sharded.partition([1, 1, 100, 1], 2)                          # one dominant node
    assert r[0][0] == 0 and r[-1][1] == 4 and 2 in range(*r[0])
    # the iteration hint weights the nodes
    r = sharded.partition(sharded.node_costs([10, 10, 10, 10], iters_hint=[3, 1, 1, 1]), 2)
    assert r == [(0, 1), (1, 4)]
    with pytest.raises(ValueError):
        sharded.partition([1.0], 0)


def test_even_query_ranges():
    for Q, world in ((10, 3), (1_000_000, 8), (2, 4), (0, 2)):
        r = [sharded.even_range(Q, k, world) for k in range(world)]
        assert r[0][0] == 0 and r[-1][1] == Q and all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [e - s for s, e in r]
        assert max(sizes) - min(sizes) <= 1


# ------------------------------------------------------------------ sharded solve on gloo ranks
def _oracle_solve(problem, x0, T, N):
    """The per-range solver of the test: one oracle solve per row (CPU tensors)."""
    from oracle import bvp
    x = x0.numpy()
    T = np.broadcast_to(np.asarray(T), (x.shape[0],))
    N = np.broadcast_to(np.asarray(N), (x.shape[0],))
    sols = [bvp.solve(problem, x[i], float(T[i]), int(N[i]), tol=1e-10) for i in range(x.shape[0])]
    return {"lambda0": torch.as_tensor(np.array([s.lambda0 for s in sols])),
            "u0": torch.as_tensor(np.array([s.u0 for s in sols])),
            "V": torch.as_tensor(np.array([s.V for s in sols])),
            "status": torch.as_tensor(np.array([s.status for s in sols], dtype=np.int32)),
            "iters": torch.as_tensor(np.array([s.iters for s in sols], dtype=np.int32))}


def _case():
    import synth
    from oracle import grid, problems
    lo, hi = synth.box(6)
    g = grid.Grid(6, 3, lo, hi)                        # level 3: 389 nodes
    rng = np.random.default_rng(9)
    T = rng.choice([0.5, 1.0, 2.0], size=g.M)
    N = np.rint(4 * T).astype(np.int32)                # 2 / 4 / 8 intervals
    return problems.make(synth.lq_params(0)), torch.as_tensor(g.x), T, N


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr, x0, T, N = _case()
        out = sharded.sharded_solve(pr, x0, torch.as_tensor(T), torch.as_tensor(N), solve_fn=_oracle_solve)
        q.put((rank, out["range"], {k: v.numpy() for k, v in out.items() if k != "range"}))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_match_one_rank_bitwise():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pr, x0, T, N = _case()
    ref = sharded.sharded_solve(pr, x0, torch.as_tensor(T), torch.as_tensor(N), solve_fn=_oracle_solve)
    assert ref["range"] == (0, x0.shape[0])
    ranges = sorted(g[1] for g in got)
    assert ranges[0][0] == 0 and ranges[-1][1] == x0.shape[0] and ranges[0][1] == ranges[1][0]
    assert 0 < ranges[0][1] < x0.shape[0]                  # both ranks had work
    for _, _, res in got:
        for key in ("lambda0", "u0", "V", "status", "iters"):
            assert np.array_equal(res[key], ref[key].numpy()), key
    assert np.all(ref["status"].numpy() == 0)
