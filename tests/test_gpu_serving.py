"""Serving loop: continuous batching with memory admission, and every result
the same alone and in the mix (per-node / per-query / per-trajectory
independence, Section 3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1507_04769_gb300 import serving, sg  # noqa: E402

pytestmark = pytest.mark.gpu


def _solo(server, r):
    """The same request computed alone, directly through the library."""
    x = torch.as_tensor(r.x, device="cuda")
    if r.kind == "bvp":
        N = serving.horizon_mesh(r.T)
        if r.full_grid:
            g = server.grid(r.level)
            res = sg.solve_bvps(server.problem, g.coords, r.T, N, tol=server.tol, precision=server.precision,
                                n_max=N)
        else:
            res = sg.solve_bvps(server.problem, x, r.T, N, tol=server.tol, precision=server.precision, n_max=N)
        return {k: res[k].cpu().numpy() for k in ("lambda0", "u0", "V", "status", "iters")}
    m = server.models[(r.level, r.T)]
    if r.kind == "eval":
        return {"u": sg.eval_feedback(m.surplus, x, mode=server.eval_mode).cpu().numpy()}
    o = sg.simulate_closed_loop(server.problem, m.surplus, x, r.nsteps, r.dt, mode=server.eval_mode)
    return {k: o[k].cpu().numpy() for k in ("xT", "cost")}


@pytest.mark.parametrize("budget_gb", [64, 1])
def test_mixed_requests_match_solo_results(budget_gb):
    server = serving.Server(slots=3, memory_budget=budget_gb << 30)
    keys = [(2, 20.0), (3, 10.0)]
    counts = server.warm(levels=(2, 3), model_keys=keys)
    reqs = serving.make_requests(40, rate=1e4, node_counts=counts, seed=7, levels=(2, 3), horizons=(10.0, 20.0),
                                 max_queries=20_000, max_traj=32, nsteps=100, model_keys=keys)
    server.start()
    done = serving.replay(server, reqs, realtime=False)
    assert len(done) == len(reqs)
    assert any(r.batch_size > 1 for r in done)          # work was merged
    rep = serving.latency_report(done)
    assert rep["all"]["p99_ms"] >= rep["all"]["p50_ms"] > 0
    for r in done:
        solo = _solo(server, r)
        for k, v in solo.items():
            assert np.array_equal(r.result[k], v), (r.kind, r.rid, k)
        if r.kind == "bvp":
            assert np.all(r.result["status"] == sg.CONVERGED)


def test_admission_respects_memory_budget():
    server = serving.Server(slots=4, memory_budget=1 << 30)
    counts = server.warm(levels=(2,))
    reqs = serving.make_requests(12, rate=1e4, node_counts=counts, seed=9, levels=(2,), horizons=(40.0,),
                                 mix=(1, 0, 0))
    peak = []
    orig = server._take

    def take():
        batch, need = orig()
        peak.append(server.in_use)
        return batch, need

    server._take = take
    server.start()
    serving.replay(server, reqs, realtime=False)
    # more than one request in flight only when the budget allows it
    biggest = max(server.footprint([r]) for r in reqs)
    assert max(peak) <= max(server.budget, biggest)
