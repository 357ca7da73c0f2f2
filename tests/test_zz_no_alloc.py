"""The allocation-free solve entry point, sg_solve_bvps_static.

Some callers cannot allocate device memory at solve time: a real-time or
on-board control loop that must not stall or fail on an allocation, or a
plugin whose host process owns the device memory pool.  This entry point
runs the same solver with its workspace in a fixed array inside the library.
Here it is called through the C ABI twice in a row, in the host-loop form and
in the persistent form, and each result is checked against sg_solve_bvps with
a caller workspace.  Both run the same kernels on the same inputs and only the
workspace address differs, so the results must be bitwise equal (every
per-node reduction has a fixed order).
"""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import synth  # noqa: E402
from paper_1507_04769_gb300 import sg  # noqa: E402

pytestmark = pytest.mark.gpu


def _static_solve(problem, x0, T, N, n_max, precision, persistent=0, graph=0):
    n = x0.shape[0]
    dev = x0.device
    out = {"lambda0": torch.empty((n, 6), dtype=torch.float64, device=dev),
           "u0": torch.empty((n, 3), dtype=torch.float64, device=dev),
           "V": torch.empty((n,), dtype=torch.float64, device=dev),
           "status": torch.empty((n,), dtype=torch.int32, device=dev),
           "iters": torch.empty((n,), dtype=torch.int32, device=dev)}
    opts = sg.SolveOpts(tol=1e-12, max_iter=50, precision=precision, damping=1, persistent=persistent,
                        graph=graph)
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = sg.LIB.sg_solve_bvps_static(C.byref(problem), p(x0), n, p(T), p(N), n_max, C.byref(opts),
                                     p(out["lambda0"]), p(out["u0"]), p(out["V"]), p(out["status"]),
                                     p(out["iters"]), None,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


@pytest.mark.parametrize("persistent", [0, 1], ids=["host-loop", "persistent"])
@pytest.mark.parametrize("precision", [sg.PREC_FP64, sg.PREC_MIXED, sg.PREC_MIXED_PAIR])
def test_static_solve_matches_workspace_solve_twice(precision, persistent):
    problem = sg.problem_from(synth.attitude_params(0))
    lo, hi = synth.box(6)
    # two different batches in a row: the second call reuses the array the first left behind
    for call, (n, seed, Tval, Nval) in enumerate([(12, 51, 10.0, 64), (7, 52, 20.0, 128)]):
        x0 = torch.as_tensor(synth.uniform_queries(n, lo, hi, seed=seed), device="cuda")
        T = torch.full((n,), Tval, dtype=torch.float64, device="cuda")
        N = torch.full((n,), Nval, dtype=torch.int32, device="cuda")
        rc, got = _static_solve(problem, x0, T, N, Nval, precision, persistent=persistent)
        assert rc == sg.SG_OK, sg.LIB.sg_last_error().decode()
        ref = sg.solve_bvps(problem, x0, T, N, tol=1e-12, precision=precision, n_max=Nval,
                            persistent=bool(persistent))
        torch.cuda.synchronize()
        assert torch.all(got["status"] == sg.CONVERGED), f"call {call}"
        for key in ("lambda0", "u0", "V", "status", "iters"):
            assert torch.equal(got[key], ref[key]), (call, key)


def test_static_solve_rejects_oversized_batch():
    problem = sg.problem_from(synth.attitude_params(0))
    n, n_max = 200, 256
    assert sg.workspace_bytes(n, n_max, sg.PREC_FP64) > 32 * 1024 * 1024
    x0 = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
    T = torch.full((n,), 40.0, dtype=torch.float64, device="cuda")
    N = torch.full((n,), n_max, dtype=torch.int32, device="cuda")
    rc, _ = _static_solve(problem, x0, T, N, n_max, sg.PREC_FP64)
    assert rc == sg.SG_EINVAL
    assert b"static array holds" in sg.LIB.sg_last_error()


def test_static_solve_rejects_graph_form():
    """The graph form instantiates CUDA graphs, which allocate: refused."""
    problem = sg.problem_from(synth.attitude_params(0))
    x0 = torch.zeros((2, 6), dtype=torch.float64, device="cuda")
    T = torch.full((2,), 10.0, dtype=torch.float64, device="cuda")
    N = torch.full((2,), 64, dtype=torch.int32, device="cuda")
    rc, _ = _static_solve(problem, x0, T, N, 64, sg.PREC_MIXED, graph=1)
    assert rc == sg.SG_EINVAL
    assert b"graph must be 0" in sg.LIB.sg_last_error()
