"""Multi-GPU split of one sparse-grid solve (one process per GPU).

Section 3 of the paper solves one characteristic BVP per grid node with no
communication between nodes.  The split here follows that structure:

  1. every rank builds the same grid (integer enumeration plus one kernel; it
     is cheap and deterministic, so it is replicated rather than sent);
  2. the nodes are cut into contiguous ranges of about equal cost, the cost of
     a node being its number of mesh intervals N times an expected Newton
     iteration count; each rank solves its range;
  3. one all-gather of the per-node results (lambda(0), u*, V, status and the
     iteration count: 12 doubles per node, 140 KB at 1457 nodes) gives every
     rank the full set, in node order;
  4. the surpluses (Eq. interpo) need every node's value, so each rank builds
     them from the gathered u*, replicated;
  5. feedback queries are cut into contiguous equal ranges, one per rank, with
     no further exchange.

The all-gather in step 3 is the only collective on the data path, and it is a
real exchange: the surplus of a node depends on the values at all coarser
nodes.  The arithmetic of every node is the same as in a one-rank solve, so a
sharded solve gives bitwise the same results as the one-rank solve.
"""
from __future__ import annotations

import numpy as np
import torch

# per-node result columns of the gathered table
_LAM, _U, _V, _ST, _IT = slice(0, 6), slice(6, 9), 9, 10, 11
_COLS = 12


def _group_info(group=None):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def node_costs(N, iters_hint=None) -> np.ndarray:
    """Cost of each node's solve: mesh intervals times expected iterations
    (1 per node when no hint is given)."""
    c = np.asarray(N, dtype=np.float64).reshape(-1)
    if iters_hint is not None:
        c = c * np.broadcast_to(np.asarray(iters_hint, dtype=np.float64), c.shape)
    return c


def partition(costs, world: int) -> list[tuple[int, int]]:
    """Contiguous ranges [start, end) of the nodes, one per rank, cut where the
    running cost crosses k / world of the total (k = 1 .. world-1).  Every node
    is in exactly one range; a range may be empty when there are fewer nodes
    than ranks."""
    costs = np.asarray(costs, dtype=np.float64).reshape(-1)
    n = costs.shape[0]
    if world < 1:
        raise ValueError("world must be >= 1")
    if n == 0:
        return [(0, 0)] * world
    cum = np.cumsum(costs)
    total = cum[-1]
    cuts = [0]
    for k in range(1, world):
        # first node whose running cost (including itself) reaches k/world of
        # the total ends the range: the cut is after it
        j = int(np.searchsorted(cum, total * k / world, side="left")) + 1
        cuts.append(min(max(j, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def even_range(Q: int, rank: int, world: int) -> tuple[int, int]:
    """The rank's contiguous share of Q queries (sizes differ by at most 1)."""
    base, extra = divmod(Q, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _pack(res: dict, n: int, dev) -> torch.Tensor:
    t = torch.zeros((n, _COLS), dtype=torch.float64, device=dev)
    if n:
        t[:, _LAM] = res["lambda0"]
        t[:, _U] = res["u0"][:, :3]
        t[:, _V] = res["V"]
        t[:, _ST] = res["status"].to(torch.float64)
        t[:, _IT] = res["iters"].to(torch.float64)
    return t


def _unpack(t: torch.Tensor) -> dict:
    return {"lambda0": t[:, _LAM].contiguous(), "u0": t[:, _U].contiguous(), "V": t[:, _V].contiguous(),
            "status": t[:, _ST].to(torch.int32), "iters": t[:, _IT].to(torch.int32)}


def all_gather_rows(local: torch.Tensor, counts: list[int], group=None) -> torch.Tensor:
    """Concatenation over ranks (in rank order) of each rank's rows; the ranks
    may hold different numbers of rows (counts, known to every rank)."""
    import torch.distributed as dist
    rank, world = _group_info(group)
    if world == 1:
        return local
    m = max(max(counts), 1)
    buf = torch.zeros((m,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    buf[:local.shape[0]] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


def sharded_solve(problem, x0: torch.Tensor, T, N, *, group=None, iters_hint=None, ranges=None,
                  solve_fn=None, **solve_kw) -> dict:
    """Solves the BVPs of all rows of x0 across the ranks of `group` and
    returns, on every rank, the full per-node results in node order (keys
    lambda0, u0, V, status, iters) plus "range", this rank's [start, end).

    ranges: the node ranges of all ranks (partition()); computed from N and
    iters_hint when not given (which reads N on the host).
    solve_fn(problem, x0, T, N, **solve_kw) solves one contiguous range; it
    defaults to sg.solve_bvps (the library's CUDA solver).  With one rank this
    is a plain solve."""
    if solve_fn is None:
        from . import sg
        solve_fn = sg.solve_bvps
    rank, world = _group_info(group)
    n = x0.shape[0]
    if ranges is None:
        N_h = np.asarray(N.cpu() if torch.is_tensor(N) else N).reshape(-1)
        if N_h.size == 1 and n > 1:
            N_h = np.full(n, int(N_h[0]))
        ranges = partition(node_costs(N_h, iters_hint), world)
    if len(ranges) != world or ranges[0][0] != 0 or ranges[-1][1] != n:
        raise ValueError("ranges must cover the n nodes with one range per rank")
    s, e = ranges[rank]
    if world == 1:
        out = dict(solve_fn(problem, x0, T, N, **solve_kw)) if n else _unpack(_pack({}, 0, x0.device))
        out["range"] = (0, n)
        return out
    Tn = T[s:e] if torch.is_tensor(T) and T.dim() > 0 and T.numel() == n else T
    Nn = N[s:e] if torch.is_tensor(N) and N.dim() > 0 and N.numel() == n else N
    if e > s:
        local = solve_fn(problem, x0[s:e], Tn, Nn, **solve_kw)
    else:
        local = {}
    full = all_gather_rows(_pack(local, e - s, x0.device), [b - a for a, b in ranges], group)
    out = _unpack(full)
    out["range"] = (s, e)
    return out
