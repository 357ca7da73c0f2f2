"""GPU parity of the closed-loop simulation (zero-order hold + RK4 with the
interpolated feedback) against the oracle, on the same seeded inputs: the
feedback values at the nodes come from one seeded gain, each side builds its
own grid and surpluses."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import synth  # noqa: E402
from oracle import closed_loop as ocl  # noqa: E402
from oracle import grid as ogrid  # noqa: E402
from oracle import interp as ointerp  # noqa: E402
from oracle import problems as oprob  # noqa: E402
from paper_1507_04769_gb300 import sg  # noqa: E402

pytestmark = pytest.mark.gpu
LO, HI = synth.box(6)


def feedback_values(x):
    """A smooth nonlinear stand-in for u*(x): linear gain plus a quadratic term."""
    K = np.array([[1.0, 0.2, 0.0, 2.0, 0.1, 0.0],
                  [0.0, 1.2, 0.3, 0.0, 2.5, 0.2],
                  [0.1, 0.0, 0.9, 0.3, 0.0, 3.0]])
    return -(x @ K.T) - 0.1 * (x ** 2) @ np.ones((6, 3)) / 6.0


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("mode", [sg.EVAL_FP64, sg.EVAL_DF32], ids=["fp64", "df32"])
@pytest.mark.parametrize("level", [1, 2])
def test_closed_loop_matches_oracle(mode, level):
    params = synth.attitude_params(0)
    g = sg.Grid(6, level, LO, HI)
    og = ogrid.Grid(6, level, LO, HI)
    S = sg.Surplus(g, torch.as_tensor(feedback_values(g.coords.cpu().numpy()), device="cuda"))
    w = ointerp.surpluses(og, feedback_values(og.x))
    X0 = np.concatenate([synth.uniform_queries(4, LO, HI, seed=61), np.zeros((1, 6))])
    nsteps, dt = 150, 0.01
    out = sg.simulate_closed_loop(sg.problem_from(params), S, torch.as_tensor(X0, device="cuda"), nsteps, dt,
                                  mode=mode, keep_trajectory=True)
    pr = oprob.make(params)
    for i in range(X0.shape[0]):
        xs, us, z = ocl.simulate(pr, og, w, X0[i], nsteps, dt)
        assert rel(out["traj"][i].cpu().numpy(), xs) <= 1e-10
        assert rel(out["ctrl"][i].cpu().numpy(), us) <= 1e-10
        if z > 0:
            assert abs(out["cost"][i].item() - z) <= 1e-10 * z
        assert rel(out["xT"][i].cpu().numpy(), xs[-1]) <= 1e-10
    # the origin is an equilibrium of the closed loop: the node at the centre
    # interpolates u*(0) = 0 exactly
    assert torch.all(out["xT"][-1] == 0.0) and out["cost"][-1].item() == 0.0


def test_closed_loop_full_size_sampled():
    """Level-4 surpluses, 1024 trajectories x 2000 steps of dt = 0.01 (the
    largest closed-loop request); one trajectory re-simulated by the oracle."""
    params = synth.attitude_params(0)
    g = sg.Grid(6, 4, LO, HI)
    og = ogrid.Grid(6, 4, LO, HI)
    S = sg.Surplus(g, torch.as_tensor(feedback_values(g.coords.cpu().numpy()), device="cuda"))
    X0 = synth.mixed_queries(1024, LO, HI, seed=62)
    out = sg.simulate_closed_loop(sg.problem_from(params), S, torch.as_tensor(X0, device="cuda"), 2000, 0.01)
    assert torch.all(torch.isfinite(out["xT"]))
    w = ointerp.surpluses(og, feedback_values(og.x))
    i = 17
    xs, _, z = ocl.simulate(oprob.make(params), og, w, X0[i], 2000, 0.01)
    assert rel(out["xT"][i].cpu().numpy(), xs[-1]) <= 1e-9
    assert abs(out["cost"][i].item() - z) <= 1e-9 * z


def test_closed_loop_bad_arguments():
    g = sg.Grid(6, 1, LO, HI)
    S1 = sg.Surplus(g, torch.ones((g.M, 1), dtype=torch.float64, device="cuda"))
    with pytest.raises(sg.SGError):
        sg.simulate_closed_loop(sg.problem_from(synth.attitude_params(0)), S1,
                                torch.zeros((1, 6), dtype=torch.float64, device="cuda"), 10, 0.01)


def test_concurrent_host_threads_with_different_levels():
    """Host threads launching the same kernels with different shared-memory
    sizes at once (closed loops and evaluations of a level-2 and a level-4
    model, each thread on its own stream): no launch fails, and each result is
    bitwise the one computed alone."""
    import threading
    prob = sg.problem_from(synth.attitude_params(0))
    surf = {}
    for L in (2, 4):
        g = sg.Grid(6, L, LO, HI)
        surf[L] = (g, sg.Surplus(g, torch.as_tensor(feedback_values(g.coords.cpu().numpy()), device="cuda")))
    x0 = torch.as_tensor(synth.mixed_queries(64, LO, HI, seed=3), device="cuda")
    alone = {L: (sg.simulate_closed_loop(prob, surf[L][1], x0, 50, 0.01)["xT"].clone(),
                 sg.eval_feedback(surf[L][1], x0, mode=sg.EVAL_DF32).clone()) for L in (2, 4)}
    torch.cuda.synchronize()
    errors, outs = [], {}

    def work(L):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                for _ in range(30):
                    xT = sg.simulate_closed_loop(prob, surf[L][1], x0, 50, 0.01, stream=st)["xT"]
                    u = sg.eval_feedback(surf[L][1], x0, mode=sg.EVAL_DF32, stream=st)
                st.synchronize()
            outs[L] = (xT, u)
        except BaseException as e:   # reported below
            errors.append(e)

    ths = [threading.Thread(target=work, args=(L,)) for L in (2, 4, 2, 4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errors, errors[0]
    for L in (2, 4):
        assert torch.equal(outs[L][0], alone[L][0]) and torch.equal(outs[L][1], alone[L][1])
