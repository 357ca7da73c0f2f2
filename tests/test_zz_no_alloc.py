"""The allocation-free solve entry point, sg_solve_bvps_static.

Some callers cannot allocate device memory at solve time: a real-time or
on-board control loop that must not stall or fail on an allocation, or a
plugin whose host process owns the device memory pool.  This entry point
runs the same solver with its workspace in a fixed array inside the library.
Here it is called through the C ABI twice in a row and each result is checked
against sg_solve_bvps (caller workspace) within the parity tolerance of the
GPU tests (1e-8 relative on lambda(0), u*(x0) and V).
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import synth  # noqa: E402
from paper_1507_04769_gb300 import sg  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _static_solve(problem, x0, T, N, n_max, precision):
    n = x0.shape[0]
    dev = x0.device
    out = {"lambda0": torch.empty((n, 6), dtype=torch.float64, device=dev),
           "u0": torch.empty((n, 3), dtype=torch.float64, device=dev),
           "V": torch.empty((n,), dtype=torch.float64, device=dev),
           "status": torch.empty((n,), dtype=torch.int32, device=dev),
           "iters": torch.empty((n,), dtype=torch.int32, device=dev)}
    opts = sg.SolveOpts(tol=1e-12, max_iter=50, precision=precision, damping=1, persistent=0)
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = sg.LIB.sg_solve_bvps_static(C.byref(problem), p(x0), n, p(T), p(N), n_max, C.byref(opts),
                                     p(out["lambda0"]), p(out["u0"]), p(out["V"]), p(out["status"]),
                                     p(out["iters"]), None,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


@pytest.mark.parametrize("precision", [sg.PREC_FP64, sg.PREC_MIXED, sg.PREC_MIXED_PAIR])
def test_static_solve_matches_workspace_solve_twice(precision):
    problem = sg.problem_from(synth.attitude_params(0))
    lo, hi = synth.box(6)
    # two different batches in a row: the second call reuses the array the first left behind
    for call, (n, seed, Tval, Nval) in enumerate([(12, 51, 10.0, 64), (7, 52, 20.0, 128)]):
        x0 = torch.as_tensor(synth.uniform_queries(n, lo, hi, seed=seed), device="cuda")
        T = torch.full((n,), Tval, dtype=torch.float64, device="cuda")
        N = torch.full((n,), Nval, dtype=torch.int32, device="cuda")
        rc, got = _static_solve(problem, x0, T, N, Nval, precision)
        assert rc == sg.SG_OK, sg.LIB.sg_last_error().decode()
        ref = sg.solve_bvps(problem, x0, T, N, tol=1e-12, precision=precision, n_max=Nval)
        torch.cuda.synchronize()
        assert torch.all(got["status"] == sg.CONVERGED), f"call {call}"
        for key in ("lambda0", "u0", "V"):
            assert _rel(got[key], ref[key]) <= TOL, (call, key)


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
