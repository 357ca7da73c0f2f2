"""Serving loop: BVP requests in the resident solver pool (continuous batching
at Newton-iteration granularity), evaluations and simulations on worker slots
with memory admission; every result the same alone and in the mix
(per-node / per-query / per-trajectory independence, Section 3), and a sample
of served results against the oracle."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import synth  # noqa: E402
from oracle import bvp as obvp  # noqa: E402
from oracle import grid as ogrid  # noqa: E402
from oracle import interp as ointerp  # noqa: E402
from oracle import problems as oprob  # noqa: E402
from paper_1507_04769_gb300 import serving, sg  # noqa: E402

pytestmark = pytest.mark.gpu


def _solo(server, r):
    """The same request computed alone, directly through the library."""
    x = torch.as_tensor(r.x, device="cuda")
    if r.kind == "bvp":
        N = serving.horizon_mesh(r.T)
        x0 = server.grid(r.level).coords if r.full_grid else x
        res = sg.solve_bvps(server.problem, x0, r.T, N, tol=server.tol, precision=server.precision,
                            n_max=server.pool_nmax)
        return {k: res[k].cpu().numpy() for k in ("lambda0", "u0", "V", "status", "iters")}
    m = server.models[(r.level, r.T)]
    if r.kind == "eval":
        return {"u": sg.eval_feedback(m.surplus, x, mode=server.eval_mode).cpu().numpy()}
    o = sg.simulate_closed_loop(server.problem, m.surplus, x, r.nsteps, r.dt, mode=server.sim_mode)
    return {k: o[k].cpu().numpy() for k in ("xT", "cost")}


@pytest.mark.parametrize("extra_gb", [32, 0])
def test_mixed_requests_match_solo_results(extra_gb):
    pool_bytes = sg.LIB.sg_pool_workspace_bytes(2048, serving.POOL_NMAX, sg.PREC_MIXED)
    server = serving.Server(slots=3, memory_budget=pool_bytes + (extra_gb << 30), pool_slots=2048)
    keys = [(2, 20.0), (3, 10.0)]
    counts = server.warm(levels=(2, 3), model_keys=keys)
    reqs = serving.make_requests(40, rate=1e4, node_counts=counts, seed=7, levels=(2, 3), horizons=(10.0, 20.0),
                                 max_queries=20_000, max_traj=32, nsteps=100, model_keys=keys)
    server.start()
    done = serving.replay(server, reqs, realtime=False)
    assert len(done) == len(reqs)
    assert any(r.batch_size > 1 for r in done if r.kind == "bvp")     # solves shared pool iterations
    assert any(r.batch_size > 1 for r in done if r.kind != "bvp")     # evaluations or simulations merged
    rep = serving.latency_report(done)
    assert rep["all"]["p99_ms"] >= rep["all"]["p50_ms"] > 0
    for r in done:
        solo = _solo(server, r)
        for k, v in solo.items():
            assert np.array_equal(r.result[k], v), (r.kind, r.rid, k)
        if r.kind == "bvp":
            assert np.all(r.result["status"] == sg.CONVERGED)
    assert server.pool.info()[1] == 0


def test_request_joins_a_batch_already_iterating():
    """A BVP request submitted while another is iterating in the pool is
    admitted before that one finishes, and both results equal their solo ones."""
    server = serving.Server(slots=1, pool_slots=4096)
    counts = server.warm(levels=(4,))
    big = serving.Request("bvp", 0, 0.0, T=40.0, level=4, x=np.zeros((counts[4], 6)), full_grid=True)
    small = serving.Request("bvp", 1, 0.0, T=10.0, level=4,
                            x=synth.uniform_queries(50, *synth.box(6), seed=3))
    server.start()
    server.submit(big)
    t_wait = time.perf_counter()
    while server.pool_iterations < 2 and time.perf_counter() - t_wait < 30:
        time.sleep(0.0005)
    assert server.pool_iterations >= 2 and 0 in server.in_pool   # the big solve is iterating
    server.submit(small)
    server.drain()
    assert small.admitted < big.done                              # joined the running batch
    assert small.batch_size >= 2 and big.batch_size >= 2
    for r in (big, small):
        solo = _solo(server, r)
        for k, v in solo.items():
            assert np.array_equal(r.result[k], v), (r.rid, k)
    assert (4, 40.0) in server.models                              # the full-grid solve rebuilt its model


def test_served_results_against_oracle():
    """Sampled BVP nodes of served requests against the oracle's root (the
    1e-6 bound stated for solves stopped at 1e-8), and served evaluations
    against the oracle's interpolant of the model's nodal values (1e-10)."""
    server = serving.Server(slots=2, pool_slots=1024)
    keys = [(2, 10.0)]
    counts = server.warm(levels=(2,), model_keys=keys)
    lo, hi = synth.box(6)
    rb = serving.Request("bvp", 0, 0.0, T=10.0, level=2, x=synth.uniform_queries(8, lo, hi, seed=41))
    re = serving.Request("eval", 1, 0.0, T=10.0, level=2, x=synth.mixed_queries(300, lo, hi, seed=42))
    server.start()
    done = serving.replay(server, [rb, re], realtime=False)
    assert len(done) == 2
    pr = oprob.make(server.params)
    sols = [obvp.solve(pr, rb.x[i], 10.0, serving.horizon_mesh(10.0)) for i in range(4)]
    for key, ref in (("lambda0", np.array([s.lambda0 for s in sols])), ("u0", np.array([s.u0 for s in sols])),
                     ("V", np.array([s.V for s in sols]))):
        assert np.max(np.abs(rb.result[key][:4] - ref)) <= 1e-6 * np.max(np.abs(ref)), key
    # the model's nodal values as the library holds them, interpolated by the oracle
    og = ogrid.Grid(6, 2, lo, hi)
    m = server.models[(2, 10.0)]
    w = ointerp.surpluses(og, _model_values(server, 2, 10.0))
    ref = ointerp.eval_surplus(og, w, re.x)
    assert np.max(np.abs(re.result["u"] - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert m.surplus.M == counts[2]


def _model_values(server, level, T):
    g = server.grid(level)
    res = sg.solve_bvps(server.problem, g.coords, T, serving.horizon_mesh(T), tol=server.tol,
                        precision=server.precision, n_max=server.pool_nmax)
    return res["u0"].cpu().numpy()


def test_tensor_core_evaluations_in_the_mix():
    """A server whose evaluations run 3xTF32 (the bench's mode): evaluations
    bitwise their solo results, simulations in DF32."""
    server = serving.Server(slots=2, pool_slots=256, eval_mode=sg.EVAL_TF32X3)
    keys = [(2, 20.0)]
    counts = server.warm(levels=(2,), model_keys=keys)
    reqs = serving.make_requests(12, rate=1e4, node_counts=counts, seed=5, levels=(2,), horizons=(20.0,),
                                 mix=(1, 1, 1), max_queries=5000, max_traj=16, nsteps=50, model_keys=keys)
    server.start()
    done = serving.replay(server, reqs, realtime=False)
    assert len(done) == len(reqs) and server.sim_mode == sg.EVAL_DF32
    for r in done:
        for k, v in _solo(server, r).items():
            assert np.array_equal(r.result[k], v), (r.kind, r.rid, k)


def test_admission_respects_memory_budget():
    """Evaluations and simulations: more than one batch in flight only when the
    budget left beside the pool allows it."""
    pool_bytes = sg.LIB.sg_pool_workspace_bytes(256, serving.POOL_NMAX, sg.PREC_MIXED)
    server = serving.Server(slots=4, memory_budget=pool_bytes + (8 << 20), pool_slots=256)
    keys = [(2, 20.0)]
    counts = server.warm(levels=(2,), model_keys=keys)
    reqs = serving.make_requests(16, rate=1e4, node_counts=counts, seed=9, levels=(2,), horizons=(20.0,),
                                 mix=(0, 1, 1), max_queries=100_000, max_traj=256, nsteps=50, model_keys=keys)
    peak = []
    orig = server._take

    def take():
        batch, need = orig()
        peak.append(server.in_use)
        return batch, need

    server._take = take
    server.start()
    serving.replay(server, reqs, realtime=False)
    biggest = max(server.footprint([r]) for r in reqs)
    assert max(peak) <= max(server.budget, biggest)
