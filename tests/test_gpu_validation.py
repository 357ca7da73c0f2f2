"""Error-controlled solves (mesh doubling) and the pointwise validation of
Section 4.1 on the GPU.  The error control is pinned to continuous closed
forms: the Riccati solution of the LQ problem and the value function printed
with Example III."""
import numpy as np
import pytest
import torch

import synth
from oracle import problems as P
from oracle import riccati

pytestmark = pytest.mark.gpu


def _mods():
    from paper_1507_04769_gb300 import sg, validation
    return sg, validation


def test_error_control_reaches_continuous_riccati_solution():
    sg, validation = _mods()
    prm = synth.lq_params(0)
    pr = P.make(prm)
    rng = np.random.default_rng(21)
    x0 = rng.uniform(-0.5, 0.5, (8, 6))
    T = 2.0
    tol = 1e-9
    res = validation.solve_error_controlled(sg.problem_from(prm), torch.as_tensor(x0, device="cuda"),
                                            torch.full((8,), T, dtype=torch.float64, device="cuda"), tol)
    assert res.ok.all()
    P0 = riccati.riccati_p0(pr, T, 4096, discrete=False)
    lam_exact = x0 @ P0.T
    V_exact = 0.5 * np.einsum("ni,ij,nj->n", x0, P0, x0)
    assert np.abs(res.V.cpu().numpy() - V_exact).max() <= 20 * tol
    assert np.abs(res.lambda0.cpu().numpy() - lam_exact).max() <= 20 * tol * max(1.0, np.abs(lam_exact).max())
    assert np.all(res.err_est <= tol)


def test_error_control_reaches_example3_closed_form():
    sg, validation = _mods()
    rng = np.random.default_rng(22)
    n = 12
    x3 = rng.uniform(-1.0, 1.0, (n, 3))
    tau = rng.uniform(0.5, 4.0, n)
    x0 = np.zeros((n, 6))
    x0[:, :3] = x3
    tol = 1e-9
    res = validation.solve_error_controlled(sg.problem_from(synth.example3_params()),
                                            torch.as_tensor(x0, device="cuda"), torch.as_tensor(tau, device="cuda"),
                                            tol)
    assert res.ok.all()
    V = P.Example3.value(tau, x3.T)
    u = P.Example3.feedback(tau, x3.T)
    assert np.abs(res.V.cpu().numpy() - V).max() <= 20 * tol
    assert np.abs(res.u0.cpu().numpy()[:, 0] - u).max() <= 20 * tol * 10


def test_pointwise_validation_of_attitude_feedback():
    """Section 4.1: the level-3 interpolant of u* against error-controlled
    solves at random states; the reference error is far below the measured
    e_interp + e_bvp, as the method requires."""
    sg, validation = _mods()
    prm = synth.attitude_params(0)
    prob = sg.problem_from(prm)
    lo, hi = synth.box(6)
    g = sg.Grid(6, 3, lo, hi)
    T = 10.0
    N = int(round(6.4 * T))
    res = sg.solve_bvps(prob, g.coords, torch.full((g.M,), T, dtype=torch.float64, device="cuda"),
                        torch.full((g.M,), N, dtype=torch.int32, device="cuda"), tol=1e-10, precision=sg.PREC_MIXED)
    assert bool((res["status"] == sg.CONVERGED).all())
    S = sg.Surplus(g, res["u0"])
    pts = torch.as_tensor(synth.uniform_queries(48, lo, hi, seed=23), device="cuda")
    val = validation.validate_feedback(prob, S, pts, T, tol=1e-9)
    st = val.stats(0)
    assert st["points"] == 48
    assert st["reference_err_est_max"] <= 1e-9
    assert st["mae"] > 1e3 * st["reference_err_est_max"]
