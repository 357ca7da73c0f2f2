"""The calls that return once their work is queued (the graph forms of the
solve, the surplus build, the evaluation): results read in stream order are
those of the synchronous path, on the current stream and on a side stream.

The reference for each case is the same library call on the default stream
followed by a synchronisation; the surplus values are also checked against the
oracle, so a build that read its inputs too early cannot pass by agreeing with
itself.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import synth  # noqa: E402
from oracle import grid as ogrid  # noqa: E402
from oracle import interp as ointerp  # noqa: E402
from paper_1507_04769_gb300 import sg  # noqa: E402

pytestmark = pytest.mark.gpu

LO, HI = synth.box(6)


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    x0 = torch.as_tensor(synth.uniform_queries(n, LO, HI, seed=seed), device="cuda")
    T = rng.choice([10.0, 20.0], n)
    N = np.round(6.4 * T).astype(np.int32)
    return x0, torch.as_tensor(T, device="cuda"), torch.as_tensor(N, device="cuda"), int(N.max())


@pytest.mark.parametrize("graph", [1, 2])
def test_graph_solve_in_stream_order(graph):
    """A graph solve queued on a side stream, its outputs read after that
    stream is synchronised, and one queued on the current stream and read
    right away, both equal the host-loop solve bit for bit."""
    prob = sg.problem_from(synth.attitude_params(0))
    x0, T, N, n_max = _batch(96, 3)
    ref = sg.solve_bvps(prob, x0, T, N, tol=1e-8, precision=sg.PREC_MIXED, n_max=n_max, graph=0)
    torch.cuda.synchronize()
    cur = sg.solve_bvps(prob, x0, T, N, tol=1e-8, precision=sg.PREC_MIXED, n_max=n_max, graph=graph)
    for key in ("lambda0", "u0", "V", "status", "iters"):
        assert torch.equal(cur[key], ref[key]), key
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    got = sg.solve_bvps(prob, x0, T, N, tol=1e-8, precision=sg.PREC_MIXED, n_max=n_max, graph=graph,
                        stream=side)
    # the current stream queues more work meanwhile (allocations included)
    junk = [torch.empty(1 << 20, dtype=torch.float64, device="cuda").fill_(float(i)) for i in range(4)]
    side.synchronize()
    for key in ("lambda0", "u0", "V", "status", "iters"):
        assert torch.equal(got[key], ref[key]), key
    del junk


def test_surplus_build_and_eval_in_stream_order():
    """The surplus build queued on a side stream straight after the values are
    written there, then the evaluation on the same stream: the oracle's
    interpolant, and bitwise the default-stream result."""
    d, L, k = 6, 3, 3
    g = sg.Grid(d, L, LO, HI)
    og = ogrid.Grid(d, L, LO, HI)
    f = np.random.default_rng(5).standard_normal((og.M, k))
    xq = synth.uniform_queries(4096, LO, HI, seed=6)
    ref_w = ointerp.surpluses(og, f)
    ref_u = ointerp.eval_surplus(og, ref_w, xq)
    S0 = sg.Surplus(g, torch.as_tensor(f, device="cuda"))
    u0 = sg.eval_feedback(S0, torch.as_tensor(xq, device="cuda"), mode=sg.EVAL_FP64).cpu().numpy()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        # the values are produced on the side stream itself, right before the build
        vals = torch.as_tensor(f, device="cuda") * 1.0
        S = sg.Surplus(g, vals, stream=side)
        u = sg.eval_feedback(S, torch.as_tensor(xq, device="cuda"), mode=sg.EVAL_FP64, stream=side)
        del vals   # freed while the build may still be queued: the allocator must not reuse it early
        filler = torch.full((og.M, k), 1e30, dtype=torch.float64, device="cuda")
    side.synchronize()
    del filler
    assert np.array_equal(u.cpu().numpy(), u0)
    assert np.max(np.abs(S.W.cpu().numpy() - ref_w)) <= 1e-11 * np.max(np.abs(ref_w))
    assert np.max(np.abs(u0 - ref_u)) <= 1e-10 * np.max(np.abs(ref_u))


def test_surplus_builds_back_to_back():
    """Surplus builds queued back to back on one stream (the cached host
    tables reused) with their evaluations, read once at the end."""
    d, L, k = 6, 2, 3
    g = sg.Grid(d, L, LO, HI)
    og = ogrid.Grid(d, L, LO, HI)
    xq = synth.uniform_queries(512, LO, HI, seed=9)
    rng = np.random.default_rng(10)
    fs = [rng.standard_normal((og.M, k)) for _ in range(6)]
    outs = []
    keep = []
    for f in fs:
        S = sg.Surplus(g, torch.as_tensor(f, device="cuda"))
        outs.append(sg.eval_feedback(S, torch.as_tensor(xq, device="cuda"), mode=sg.EVAL_FP64))
        keep.append(S)
    torch.cuda.synchronize()
    for f, u in zip(fs, outs):
        ref = ointerp.eval_surplus(og, ointerp.surpluses(og, f), xq)
        assert np.max(np.abs(u.cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))
