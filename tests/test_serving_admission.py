"""Host logic of the serving loop without a GPU: admission by device-memory
footprint (first fit from the queue), merging of compatible requests up to the
per-kind caps, and requests that wait for their model."""
import os
import sys
from collections import deque

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture()
def server():
    pytest.importorskip("torch")
    from paper_1507_04769_gb300 import serving, sg
    s = serving.Server.__new__(serving.Server)   # no streams, no device: only the queue logic
    s.queue = deque()
    s.models = {}
    s.merge = True
    s.precision = sg.PREC_MIXED
    s.budget = 1 << 30
    s.in_use = 0
    return s


def _req(kind, rid, n, **kw):
    from paper_1507_04769_gb300 import serving
    return serving.Request(kind=kind, rid=rid, arrival=0.0, x=np.zeros((n, 6)), **kw)


def test_footprint_of_a_bvp_batch_is_its_workspace(server):
    from paper_1507_04769_gb300 import serving, sg
    r = _req("bvp", 0, 100, T=20.0)
    N = serving.horizon_mesh(20.0)
    assert N == 128
    assert server.footprint([r]) == sg.workspace_bytes(100, N, sg.PREC_MIXED) + 100 * 8 * 20
    assert server.footprint([_req("eval", 1, 1000)]) == 1000 * 8 * 9 * 2


def test_first_fit_merges_compatible_requests(server):
    server.models[(2, 20.0)] = object()
    for i, (kind, n, T) in enumerate([("bvp", 10, 20.0), ("eval", 500, 20.0), ("bvp", 20, 20.0),
                                       ("bvp", 5, 40.0), ("eval", 300, 20.0)]):
        server.queue.append(_req(kind, i, n, T=T, level=2))
    batch, need = server._take()
    # the head BVP (T = 20) takes the other BVP of the same horizon, not the T = 40 one
    assert [q.rid for q in batch] == [0, 2] and need == server.footprint(batch)
    assert server.in_use == need
    batch, _ = server._take()
    assert [q.rid for q in batch] == [1, 4]            # the two evaluations of one model
    batch, _ = server._take()
    assert [q.rid for q in batch] == [3]
    assert server._take() == (None, 0)


def test_budget_blocks_large_work_but_never_deadlocks(server):
    big = _req("bvp", 0, 4096, T=40.0)
    small = _req("eval", 1, 10, T=20.0, level=2)
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


def test_full_grid_solves_are_never_merged(server):
    server.queue.append(_req("bvp", 0, 85, T=20.0, level=2, full_grid=True))
    server.queue.append(_req("bvp", 1, 85, T=20.0, level=2, full_grid=True))
    batch, _ = server._take()
    assert [q.rid for q in batch] == [0]
