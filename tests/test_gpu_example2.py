"""Example II (Section 5) on the GPU: the target attitudes against the
oracle's constrained maximisation, per-node solves against the oracle, and
the printed optimal trajectory."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import bvp, lobatto
from oracle import problems as P

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "example2_trajectory.txt")
PRM = synth.example2_params()


def _sg():
    from paper_1507_04769_gb300 import sg
    return sg


def _states(n, seed):
    lo, hi = synth.example2_box()
    return synth.uniform_queries(n, lo, hi, seed=seed)


def test_targets_match_oracle():
    sg = _sg()
    X = _states(24, 41)
    tgt, st = sg.attitude_targets(sg.problem_from(PRM), torch.as_tensor(X, device="cuda"))
    assert np.all(st.cpu().numpy() == 0)
    tgt = tgt.cpu().numpy()
    for i in range(len(X)):
        ref = P.target_attitude(PRM, X[i])
        assert np.abs(tgt[i] - ref).max() < 1e-9, (i, tgt[i], ref)


def test_targets_reject_three_wheel_problem():
    sg = _sg()
    with pytest.raises(sg.SGError):
        sg.attitude_targets(sg.problem_from(synth.attitude_params(0)),
                            torch.zeros((2, 6), device="cuda", dtype=torch.float64))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_example2_solves_match_oracle(precision):
    sg = _sg()
    prec = sg.PREC_FP64 if precision == "fp64" else sg.PREC_MIXED
    X = _states(10, 42)
    T, N = synth.EXAMPLE2_T, 192
    Xd = torch.as_tensor(X, device="cuda")
    tgt, _ = sg.attitude_targets(sg.problem_from(PRM), Xd)
    prob = sg.problem_from(PRM, target=tgt)
    res = sg.solve_bvps(prob, Xd, torch.full((len(X),), T, dtype=torch.float64, device="cuda"),
                        torch.full((len(X),), N, dtype=torch.int32, device="cuda"), tol=1e-12, precision=prec)
    assert np.all(res["status"].cpu().numpy() == sg.CONVERGED)
    lam, u, V = res["lambda0"].cpu().numpy(), res["u0"].cpu().numpy(), res["V"].cpu().numpy()
    tg = tgt.cpu().numpy()
    for i in range(len(X)):
        s = bvp.solve(P.make(PRM, target=tg[i]), X[i], T, N, tol=1e-12)
        assert np.abs(lam[i] - s.lambda0).max() <= 1e-10 * max(1.0, np.abs(s.lambda0).max())
        assert np.abs(u[i, :2] - s.u0).max() <= 1e-10 * max(1.0, np.abs(s.u0).max()) and u[i, 2] == 0.0
        assert abs(V[i] - s.V) <= 1e-10 * max(1.0, abs(s.V))


def test_printed_trajectory_on_gpu():
    """The collocation solution from x(0) = (0, pi/8, 0, 0, 0, 0) against the
    printed trajectory (16 times, 8 components) to 1e-6."""
    sg = _sg()
    x0 = np.array([[0.0, np.pi / 8, 0.0, 0.0, 0.0, 0.0]])
    T, N = synth.EXAMPLE2_T, 960
    Xd = torch.as_tensor(x0, device="cuda")
    tgt, _ = sg.attitude_targets(sg.problem_from(PRM), Xd)
    prob = sg.problem_from(PRM, target=tgt)
    res = sg.solve_bvps(prob, Xd, torch.full((1,), T, dtype=torch.float64, device="cuda"),
                        torch.full((1,), N, dtype=torch.int32, device="cuda"), tol=1e-12,
                        precision=sg.PREC_FP64, return_Y=True)
    Y = res["Y"][0].cpu().numpy()
    _, _, c = lobatto.tableau()
    h = T / N
    rows = [list(map(float, l.split())) for l in open(GOLDEN) if l.strip() and l[0] != "#"]
    B = np.asarray(PRM.B)
    for row in rows:
        t, ref = row[0], np.array(row[1:])
        i = min(int(t / h), N - 1)
        tau = (t - i * h) / h
        y = sum(np.prod([(tau - c[j]) / (c[k] - c[j]) for j in range(4) if j != k]) * Y[3 * i + k] for k in range(4))
        u = -B.T @ (y[9:12] / np.asarray(PRM.J)) / PRM.r
        assert np.abs(np.concatenate([y[:6], u]) - ref).max() < 1e-6, t


def test_two_wheel_surface_and_value_validation():
    """Level 3 of Example II: every node gets a target and converges, the
    interpolant reproduces the solved values at the nodes, and the pointwise
    validation of V runs against error-controlled solves with their own
    target attitudes."""
    sg = _sg()
    from paper_1507_04769_gb300 import surfaces, validation
    lo, hi = synth.example2_box()
    srf = surfaces.two_wheel_surface(PRM, 3, lo, hi, synth.EXAMPLE2_T)
    vals = torch.stack([srf.result["u0"][:, 0], srf.result["u0"][:, 1], srf.result["V"]], dim=1)
    at_nodes = srf.evaluate(srf.grid.coords)
    assert float((at_nodes - vals).abs().max()) <= 1e-10 * max(1.0, float(vals.abs().max()))
    pts = torch.as_tensor(_states(32, 43), device="cuda")
    tgt, st = sg.attitude_targets(sg.problem_from(PRM), pts)
    assert bool((st == 0).all())
    val = validation.validate_value(sg.problem_from(PRM), srf.surplus, pts, synth.EXAMPLE2_T, 1e-9,
                                    value_col=2, target=tgt)
    s = val.stats(0)
    assert s["points"] == 32 and s["reference_err_est_max"] <= 1e-9
    assert 0.0 < s["relative_mae"] < 1.0
