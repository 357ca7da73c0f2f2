"""Serving loop with continuous batching over the sparse grid characteristics
library.

Three request kinds arrive over time:
  * bvp   - characteristic BVP solves at n initial states (1..4096) for a
            horizon T; when the states are all nodes of a level-L grid, the
            solve also (re)builds the resident feedback model of (L, T): the
            surpluses of u* at that grid's nodes (Steps I-III of Section 3.3);
  * eval  - u*(x) at Q query states from a resident model (1..1e5 queries);
  * sim   - closed-loop simulations from a resident model (1..1024
            trajectories, zero-order hold + RK4, Section 5).

BVP solves run in a resident solver pool (sg.SolverPool): a fixed set of node
slots whose Newton state stays on the device.  One engine thread admits the
queued BVP requests into free slots (first come, first served), advances every
slot by one Newton iteration per pool iteration, and hands each request its
results when all of its nodes have finished.  A request that arrives while
others are iterating joins them at the next iteration, and slots freed by
finished nodes are refilled at once (continuous batching at Newton-iteration
granularity).  The pool's memory is reserved when the server starts.

Evaluations and simulations run on worker slots, each with its own CUDA
stream, so their work overlaps with the pool's and with each other's on the
device.  A worker takes the first queued request whose footprint fits the
device-memory budget left beside the pool (so a large request does not block
small ones), and merges compatible queued requests (same kind and model) into
one launch.  Grids and surplus models stay resident.

Every node, query and trajectory is computed independently, so a request's
result is bitwise the same alone and in any mix.
"""
from __future__ import annotations

import math
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

import synth
from . import sg

MAX_BVP_STATES = 4096
POOL_SLOTS = 8192             # node slots of the resident solver pool (a level-5 grid has 4865)
POOL_NMAX = 256               # mesh intervals per slot (T = 40)
MAX_EVAL_MERGE = 400_000      # queries per merged evaluation
MAX_SIM_MERGE = 2048          # trajectories per merged simulation


@dataclass
class Request:
    kind: str                 # "bvp" | "eval" | "sim"
    rid: int
    arrival: float            # seconds since the server clock started
    T: float = 20.0
    level: int = 2
    x: np.ndarray | None = None          # states / queries / initial states (n x 6)
    full_grid: bool = False              # bvp: the states are all nodes of `level`
    nsteps: int = 2000
    dt: float = 0.01
    # filled by the server
    admitted: float = math.nan
    done: float = math.nan
    result: dict = field(default_factory=dict)
    batch_size: int = 1


def horizon_mesh(T: float) -> int:
    """N = 6.4 T intervals (one mesh width, 5/32, for T in {10, 20, 40})."""
    return int(round(6.4 * T))


class Model:
    """A resident feedback model: the grid of one level and the surpluses of u*."""

    def __init__(self, grid: sg.Grid, surplus: sg.Surplus, T: float):
        self.grid, self.surplus, self.T = grid, surplus, T


class Server:
    def __init__(self, params=None, *, slots=4, memory_budget=32 << 30, precision=sg.PREC_MIXED,
                 eval_mode=sg.EVAL_DF32, tol=1e-8, merge=True, device=None, pool_slots=POOL_SLOTS,
                 pool_nmax=POOL_NMAX):
        self.params = params if params is not None else synth.attitude_params(0)
        self.problem = sg.problem_from(self.params)
        self.lo, self.hi = synth.box(6)
        self.precision, self.eval_mode, self.tol = precision, eval_mode, tol
        # closed loops evaluate the feedback inside their own kernel, in FP64 or
        # DF32; with 3xTF32 evaluations they take DF32
        self.sim_mode = sg.EVAL_FP64 if eval_mode == sg.EVAL_FP64 else sg.EVAL_DF32
        self.merge = merge
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.queue: deque[Request] = deque()        # eval and sim requests
        self.bvp_queue: deque[Request] = deque()    # BVP requests waiting for pool slots
        self.cv = threading.Condition()
        self.models: dict[tuple, Model] = {}
        self.grids: dict[int, sg.Grid] = {}
        self.completed: list[Request] = []
        self.n_slots = slots
        self.free_slots = slots
        self.stop = False
        self.t0 = time.perf_counter()
        self.workers = []
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.errors: list[BaseException] = []
        # the resident solver pool: its memory is reserved out of the budget
        self.pool_nmax = int(pool_nmax)
        self.pool = sg.SolverPool(self.problem, pool_slots, self.pool_nmax, tol=tol, precision=precision,
                                  device=self.device)
        self.pool_stream = torch.cuda.Stream(device=self.device)
        self.budget = max(int(memory_budget) - self.pool.nbytes, 0)
        self.in_use = 0
        self.in_pool: dict[int, tuple] = {}          # rid -> (request, slots)
        self.pool_iterations = 0

    # ------------------------------------------------------------ resident state
    def warm(self, levels=(2, 3, 4, 5), model_keys=()):
        """Builds the grids of `levels` and the models of `model_keys` before
        serving (grid construction synchronises the device)."""
        for L in levels:
            self.grid(L)
        for (L, T) in model_keys:
            self.build_model(L, T)
        torch.cuda.synchronize()
        return {L: self.grids[L].M for L in self.grids}

    def grid(self, level: int) -> sg.Grid:
        if level not in self.grids:
            self.grids[level] = sg.Grid(6, level, self.lo, self.hi)
        return self.grids[level]

    def build_model(self, level: int, T: float, stream=None):
        """Solves the full grid of `level` for horizon T and stores its model."""
        g = self.grid(level)
        N = horizon_mesh(T)
        st = stream or torch.cuda.current_stream()
        with torch.cuda.stream(st):
            res = sg.solve_bvps(self.problem, g.coords, T, N, tol=self.tol, precision=self.precision,
                                n_max=self.pool_nmax)
            S = sg.Surplus(g, res["u0"])
        st.synchronize()   # built before other streams can use the model
        self.models[(level, T)] = Model(g, S, T)
        return res

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # ------------------------------------------------------------ footprints
    def footprint(self, reqs) -> int:
        """Device bytes of an eval or sim batch (BVP solves live in the pool)."""
        r = reqs[0]
        n = sum(q.x.shape[0] for q in reqs)
        if r.kind == "eval":
            return n * 8 * (6 + 3) * 2
        return n * 8 * (6 + 6 + 1)

    def merge_key(self, r: Request):
        return (r.kind, r.level, r.T)

    # ------------------------------------------------------------ queue
    def submit(self, req: Request):
        with self.cv:
            (self.bvp_queue if req.kind == "bvp" else self.queue).append(req)
            self.cv.notify_all()

    def _take(self):
        """First request in the queue whose footprint fits, plus compatible
        queued requests merged behind it (caller holds the lock)."""
        for i, r in enumerate(self.queue):
            if r.kind in ("eval", "sim") and (r.level, r.T) not in self.models:
                continue   # its model is being built: leave it queued
            batch = [r]
            if self.merge:
                key = self.merge_key(r)
                cap = {"eval": MAX_EVAL_MERGE, "sim": MAX_SIM_MERGE}[r.kind]
                tot = r.x.shape[0]
                for q in list(self.queue)[i + 1:]:
                    if self.merge_key(q) == key and tot + q.x.shape[0] <= cap:
                        batch.append(q)
                        tot += q.x.shape[0]
            need = self.footprint(batch)
            if self.in_use + need <= self.budget or self.in_use == 0:
                for q in batch:
                    self.queue.remove(q)
                self.in_use += need
                return batch, need
        return None, 0

    # ------------------------------------------------------------ execution
    def _run(self, batch, stream):
        r = batch[0]
        x = torch.as_tensor(np.concatenate([q.x for q in batch]), dtype=torch.float64)
        with torch.cuda.stream(stream):
            xd = x.pin_memory().to(self.device, non_blocking=True)
            if r.kind == "eval":
                m = self.models[(r.level, r.T)]
                u = sg.eval_feedback(m.surplus, xd, mode=self.eval_mode, stream=stream)
                out = {"u": u.cpu()}
            else:
                m = self.models[(r.level, r.T)]
                o = sg.simulate_closed_loop(self.problem, m.surplus, xd, r.nsteps, r.dt, mode=self.sim_mode,
                                            stream=stream)
                out = {k: o[k].cpu() for k in ("xT", "cost")}
            stream.synchronize()
        off = 0
        t = self.now()
        for q in batch:
            n = q.x.shape[0]
            q.result = {k: v[off:off + n].numpy().copy() for k, v in out.items()}
            q.done = t
            q.batch_size = len(batch)
            off += n

    def _worker(self, slot: int):
        stream = self.streams[slot]
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while True:
                    if self.stop and not self.queue:
                        return
                    batch, need = self._take()
                    if batch is not None:
                        break
                    self.cv.wait(timeout=0.01)
                t = self.now()
                for q in batch:
                    q.admitted = t
            try:
                self._run(batch, stream)
            except BaseException as e:   # recorded and re-raised by drain()
                self.errors.append(e)
            with self.cv:
                self.in_use -= need
                self.completed.extend(batch)
                self.cv.notify_all()

    # ------------------------------------------------------------ BVP engine
    def _admit_bvp(self):
        """Admits queued BVP requests in arrival order while the pool has room
        (caller holds the lock).  Returns the requests admitted."""
        admitted = []
        n_free, _ = self.pool.info()
        while self.bvp_queue:
            r = self.bvp_queue[0]
            n = r.x.shape[0]
            if n > n_free:
                break
            self.bvp_queue.popleft()
            admitted.append(r)
            n_free -= n
        return admitted

    def _bvp_engine(self):
        torch.cuda.set_device(self.device)
        st = self.pool_stream
        while True:
            with self.cv:
                while True:
                    batch = self._admit_bvp()
                    if batch or self.in_pool:
                        break
                    if self.stop and not self.bvp_queue:
                        return
                    self.cv.wait(timeout=0.01)
            try:
                t = self.now()
                for r in batch:
                    r.admitted = t
                    with torch.cuda.stream(st):
                        if r.full_grid:
                            x0 = self.grid(r.level).coords
                        else:
                            x0 = torch.as_tensor(r.x, dtype=torch.float64).pin_memory().to(self.device,
                                                                                           non_blocking=True)
                        n = x0.shape[0]
                        T = torch.full((n,), r.T, dtype=torch.float64, device=self.device)
                        N = torch.full((n,), horizon_mesh(r.T), dtype=torch.int32, device=self.device)
                        slots = self.pool.admit(x0, T, N, stream=st)
                    self.in_pool[r.rid] = (r, slots)
                    r.batch_size = 0
                live = len(self.in_pool)
                for r, _ in self.in_pool.values():
                    r.batch_size = max(r.batch_size, live)   # requests sharing the pool iterations
                self.pool.iterate(stream=st)
                self.pool_iterations += 1
                done = set(self.pool.finished().tolist())
                finished = []
                for rid, (r, slots) in list(self.in_pool.items()):
                    if set(slots.tolist()) <= done:
                        out = self.pool.collect(slots, stream=st)
                        if r.full_grid:
                            g = self.grid(r.level)
                            with torch.cuda.stream(st):
                                S = sg.Surplus(g, out["u0"], stream=st)
                            st.synchronize()   # built before other streams can use the model
                            self.models[(r.level, r.T)] = Model(g, S, r.T)
                        with torch.cuda.stream(st):
                            r.result = {k: v.cpu().numpy() for k, v in out.items()}
                        del self.in_pool[rid]
                        finished.append(r)
                t = self.now()
                for r in finished:
                    r.done = t
            except BaseException as e:   # recorded and re-raised by drain()
                self.errors.append(e)
                with self.cv:
                    for r, _ in self.in_pool.values():
                        r.done = self.now()
                        self.completed.append(r)
                    self.in_pool.clear()
                    self.bvp_queue.clear()
                    self.cv.notify_all()
                return
            with self.cv:
                self.completed.extend(finished)
                self.cv.notify_all()

    def start(self):
        """Starts the workers and the BVP engine; a drained server can be
        started again (resident grids, models and the pool are kept)."""
        self.stop = False
        self.completed = []
        self.workers = []
        self.t0 = time.perf_counter()
        for s in range(self.n_slots):
            th = threading.Thread(target=self._worker, args=(s,), daemon=True)
            th.start()
            self.workers.append(th)
        th = threading.Thread(target=self._bvp_engine, daemon=True)
        th.start()
        self.workers.append(th)

    def drain(self, timeout=600.0):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for th in self.workers:
            th.join(timeout)
        if self.errors:
            raise self.errors[0]


# ---------------------------------------------------------------- workloads
def make_requests(n_requests: int, rate: float, node_counts: dict, seed: int = 1, levels=(2, 3, 4, 5),
                  horizons=(10.0, 20.0, 40.0), mix=(1, 1, 1), max_queries=100_000, max_traj=1024, nsteps=2000,
                  model_keys=None):
    """Poisson arrivals at `rate` per second.  Kinds drawn with weights `mix`
    (bvp, eval, sim); sizes log-uniform: BVP 1..4096 states (a draw at or
    above the node count of its level becomes the full grid of that level,
    which rebuilds the level's model), evals 1..max_queries, simulations
    1..max_traj trajectories.  Evaluations and simulations use the resident
    models in `model_keys` ((level, T) pairs).  node_counts: level -> nodes."""
    rng = np.random.default_rng(seed)
    lo, hi = synth.box(6)
    t = 0.0
    reqs = []
    kinds = rng.choice(3, size=n_requests, p=np.array(mix, dtype=float) / sum(mix))
    model_keys = list(model_keys or [(2, 20.0)])
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        k = kinds[i]
        sub = int(rng.integers(1 << 30))
        if k == 0:
            L = int(rng.choice(levels))
            T = float(rng.choice(horizons))
            n = int(np.exp(rng.uniform(0.0, np.log(MAX_BVP_STATES))))
            M = node_counts[L]
            if n >= M:
                reqs.append(Request("bvp", i, t, T=T, level=L, x=np.zeros((M, 6)), full_grid=True))
            else:
                reqs.append(Request("bvp", i, t, T=T, level=L, x=synth.uniform_queries(n, lo, hi, seed=sub)))
        elif k == 1:
            L, T = model_keys[int(rng.integers(len(model_keys)))]
            q = int(np.exp(rng.uniform(0.0, np.log(max_queries))))
            reqs.append(Request("eval", i, t, T=T, level=L, x=synth.mixed_queries(q, lo, hi, seed=sub)))
        else:
            L, T = model_keys[int(rng.integers(len(model_keys)))]
            m = int(np.exp(rng.uniform(0.0, np.log(max_traj))))
            reqs.append(Request("sim", i, t, T=T, level=L, nsteps=nsteps,
                                x=synth.mixed_queries(m, lo, hi, seed=sub)))
    return reqs


def replay(server: Server, reqs, realtime: bool = True):
    """Feeds `reqs` to a started server at their arrival times (or all at once)
    and waits for completion.  Returns the completed requests."""
    t_start = server.now()
    for r in reqs:
        if realtime:
            delay = r.arrival - (server.now() - t_start)
            if delay > 0:
                time.sleep(delay)
        r.arrival = server.now()
        server.submit(r)
    server.drain()
    return server.completed


def latency_report(done):
    """p50 / p99 latency (arrival to results on the host) and throughput per kind."""
    out = {}
    if not done:
        return out
    span = max(r.done for r in done) - min(r.arrival for r in done)
    for kind in ("bvp", "eval", "sim", "all"):
        rs = [r for r in done if kind == "all" or r.kind == kind]
        if not rs:
            continue
        lat = np.array([r.done - r.arrival for r in rs])
        items = sum(r.x.shape[0] for r in rs)
        out[kind] = {"requests": len(rs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                     "p99_ms": float(np.percentile(lat, 99) * 1e3), "items": int(items),
                     "requests_per_s": len(rs) / span, "items_per_s": items / span,
                     "mean_batch": float(np.mean([r.batch_size for r in rs]))}
    return out
