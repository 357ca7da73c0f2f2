"""Host logic of the serving loop without a GPU: BVP requests entering the
solver pool in arrival order while slots last; evaluations and simulations
admitted by device-memory footprint (first fit from the queue), merged up to
the per-kind caps, and waiting for their model."""
import os
import sys
from collections import deque

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _FakePool:
    """Stands in for sg.SolverPool: only its free-slot count matters here."""

    def __init__(self, free):
        self.free = free

    def info(self):
        return self.free, 0


@pytest.fixture()
def server():
    pytest.importorskip("torch")
    from paper_1507_04769_gb300 import serving, sg
    s = serving.Server.__new__(serving.Server)   # no streams, no device: only the queue logic
    s.queue = deque()
    s.bvp_queue = deque()
    s.models = {}
    s.merge = True
    s.precision = sg.PREC_MIXED
    s.budget = 1 << 30
    s.in_use = 0
    s.pool = _FakePool(100)
    return s


def _req(kind, rid, n, **kw):
    from paper_1507_04769_gb300 import serving
    return serving.Request(kind=kind, rid=rid, arrival=0.0, x=np.zeros((n, 6)), **kw)


def test_footprints_of_evaluations_and_simulations(server):
    assert server.footprint([_req("eval", 1, 1000)]) == 1000 * 8 * 9 * 2
    assert server.footprint([_req("sim", 2, 10), _req("sim", 3, 30)]) == 40 * 8 * 13


def test_bvp_requests_enter_the_pool_in_arrival_order_while_slots_last(server):
    for i, n in enumerate([30, 50, 40, 5]):
        server.bvp_queue.append(_req("bvp", i, n, T=20.0))
    # 100 free slots: the first two fit (80), the third (40) does not, and the
    # fourth waits behind it (first come, first served: no overtaking)
    assert [r.rid for r in server._admit_bvp()] == [0, 1]
    assert [r.rid for r in server.bvp_queue] == [2, 3]
    server.pool.free = 45
    assert [r.rid for r in server._admit_bvp()] == [2, 3]
    assert server._admit_bvp() == []


def test_submit_routes_by_kind(server):
    import threading
    server.cv = threading.Condition()
    server.submit(_req("bvp", 0, 3))
    server.submit(_req("eval", 1, 3))
    assert [r.rid for r in server.bvp_queue] == [0] and [r.rid for r in server.queue] == [1]


def test_first_fit_merges_compatible_requests(server):
    server.models[(2, 20.0)] = object()
    server.models[(2, 40.0)] = object()
    for i, (kind, n, T) in enumerate([("eval", 10, 20.0), ("sim", 500, 20.0), ("eval", 20, 20.0),
                                       ("eval", 5, 40.0), ("sim", 300, 20.0)]):
        server.queue.append(_req(kind, i, n, T=T, level=2))
    batch, need = server._take()
    # the head evaluation (T = 20) takes the other one of the same model, not the T = 40 one
    assert [q.rid for q in batch] == [0, 2] and need == server.footprint(batch)
    assert server.in_use == need
    batch, _ = server._take()
    assert [q.rid for q in batch] == [1, 4]            # the two simulations of one model
    batch, _ = server._take()
    assert [q.rid for q in batch] == [3]
    assert server._take() == (None, 0)


def test_budget_blocks_large_work_but_never_deadlocks(server):
    big = _req("eval", 0, 100_000, T=20.0, level=2)
    small = _req("sim", 1, 10, T=20.0, level=2)
    server.models[(2, 20.0)] = object()
    server.budget = server.footprint([big]) // 2
    server.queue.extend([big, small])
    # nothing in use: the head is admitted even above the budget (else it would wait forever)
    batch, need = server._take()
    assert [q.rid for q in batch] == [0]
    # now the small request fits only if the budget covers it next to the big one
    batch2, _ = server._take()
    assert batch2 is None
    server.in_use -= need
    batch3, _ = server._take()
    assert [q.rid for q in batch3] == [1]


def test_requests_wait_for_their_model_and_merges_respect_caps(server):
    from paper_1507_04769_gb300 import serving
    server.queue.append(_req("sim", 0, 10, T=20.0, level=3))     # model (3, 20) not resident yet
    server.queue.append(_req("eval", 1, serving.MAX_EVAL_MERGE - 5, T=20.0, level=2))
    server.queue.append(_req("eval", 2, 10, T=20.0, level=2))
    server.models[(2, 20.0)] = object()
    batch, _ = server._take()
    # the simulation is skipped (its model is missing); the evaluations do not merge past the cap
    assert [q.rid for q in batch] == [1]
    batch, _ = server._take()
    assert [q.rid for q in batch] == [2]
    assert server._take() == (None, 0)
    server.models[(3, 20.0)] = object()
    batch, _ = server._take()
    assert [q.rid for q in batch] == [0]
