"""The resident solver pool (sg_pool_*): solves admitted between Newton
iterations, into a batch already iterating on the device, give bitwise the
results of the same nodes solved alone by sg_solve_bvps; freed slots are
reused without leaking state; sampled results match the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import synth  # noqa: E402
from oracle import bvp as obvp  # noqa: E402
from oracle import problems as oprob  # noqa: E402
from paper_1507_04769_gb300 import sg  # noqa: E402

pytestmark = pytest.mark.gpu

LO, HI = synth.box(6)
NMAX = 128
KEYS = ("lambda0", "u0", "V", "status", "iters")


def _request(n, seed):
    x0 = synth.uniform_queries(n, LO, HI, seed=seed)
    T = np.random.default_rng(seed).choice([5.0, 10.0, 20.0], size=n)
    N = np.rint(6.4 * T).astype(np.int32)
    return x0, T, N


def _solo(prob, req, prec):
    x0, T, N = req
    return sg.solve_bvps(prob, torch.as_tensor(x0, device="cuda"), torch.as_tensor(T, device="cuda"),
                         torch.as_tensor(N, dtype=torch.int32, device="cuda"), tol=1e-8, precision=prec, n_max=NMAX)


def _drive(pool, schedule, max_iters=200):
    """Runs the pool; schedule maps an iteration number to requests admitted
    just before it.  Returns {request index: outputs in request order}."""
    slots_of, got, pending = {}, {}, {}
    it = 0
    while it < max_iters:
        for k, req in schedule.get(it, []):
            x0, T, N = req
            slots_of[k] = pool.admit(x0, T, N)
            pending[k] = set(slots_of[k].tolist())
        active = pool.iterate()
        done = set(pool.finished().tolist())
        for k in list(pending):
            if pending[k] <= done:
                got[k] = {key: v.cpu().numpy() for key, v in pool.collect(slots_of[k]).items()}
                done -= pending.pop(k)
        it += 1
        if not pending and active == 0 and all(i < it for i in schedule):
            break
    assert not pending, "pool did not finish"
    return got, slots_of


@pytest.mark.parametrize("prec", [sg.PREC_MIXED, sg.PREC_FP64, sg.PREC_MIXED_PAIR], ids=["mixed", "fp64", "pair"])
def test_requests_admitted_mid_batch_match_solo(prec):
    prob = sg.problem_from(synth.attitude_params(0))
    pool = sg.SolverPool(prob, 64, NMAX, tol=1e-8, precision=prec)
    reqs = [_request(20, 1), _request(9, 2), _request(17, 3)]
    reqs[1][0][4] = 0.0                                  # the origin: converged at admission
    # B joins after two iterations of A, C after four (while A and B iterate)
    got, slots = _drive(pool, {0: [(0, reqs[0])], 2: [(1, reqs[1])], 4: [(2, reqs[2])]})
    for k, req in enumerate(reqs):
        solo = _solo(prob, req, prec)
        for key in KEYS:
            assert np.array_equal(got[k][key], solo[key].cpu().numpy()), (k, key)
        assert np.all(got[k]["status"] == sg.CONVERGED)
    assert got[1]["iters"][4] == 0 and got[1]["V"][4] == 0.0
    assert pool.info() == (64, 0)                        # every slot returned


def test_freed_slots_are_reused_cleanly():
    """Slots freed by one request and refilled by the next give the solo result
    (nothing of the previous solve leaks); the pool's slots are all reused."""
    prob = sg.problem_from(synth.attitude_params(0))
    pool = sg.SolverPool(prob, 24, NMAX, precision=sg.PREC_MIXED)
    first = _request(24, 11)
    got1, s1 = _drive(pool, {0: [(0, first)]})
    second = _request(24, 12)
    got2, s2 = _drive(pool, {0: [(0, second)]})
    assert set(s1[0].tolist()) == set(s2[0].tolist()) == set(range(24))
    for req, got in ((first, got1[0]), (second, got2[0])):
        solo = _solo(prob, req, sg.PREC_MIXED)
        for key in KEYS:
            assert np.array_equal(got[key], solo[key].cpu().numpy()), key


def test_pool_errors_and_bad_input():
    prob = sg.problem_from(synth.attitude_params(0))
    pool = sg.SolverPool(prob, 4, NMAX, precision=sg.PREC_MIXED)
    x0, T, N = _request(3, 21)
    N[1] = NMAX + 1                                      # outside the pool's meshes
    slots = pool.admit(x0, T, N)
    with pytest.raises(sg.SGError, match="slots asked"):  # SG_EFULL: 2 asked, 1 free
        pool.admit(x0[:2], T[:2], N[:2])
    with pytest.raises(sg.SGError, match="no finished solve"):
        pool.collect(slots[:1])
    while pool.iterate() > 0:
        pass
    out = pool.collect(pool.finished())
    st = out["status"].cpu().numpy()
    assert sorted(st.tolist()) == sorted([sg.CONVERGED, sg.BADINPUT, sg.CONVERGED])
    assert torch.isnan(out["V"][st == sg.BADINPUT]).all()
    assert pool.iterate() == 0                           # empty pool: nothing launched


def test_pool_results_against_oracle():
    """A sample of pool results against the oracle's polished root, within
    the a-priori bound stated for solves stopped at 1e-8 (1e-6 relative)."""
    params = synth.attitude_params(0)
    prob = sg.problem_from(params)
    pool = sg.SolverPool(prob, 16, NMAX, precision=sg.PREC_MIXED)
    x0 = synth.uniform_queries(6, LO, HI, seed=31)
    T = np.array([5.0, 10.0, 10.0, 5.0, 10.0, 5.0])
    N = np.rint(6.4 * T).astype(np.int32)
    got, _ = _drive(pool, {0: [(0, (x0, T, N))]})
    pr = oprob.make(params)
    sols = [obvp.solve(pr, x0[i], float(T[i]), int(N[i])) for i in range(6)]
    for key, ref in (("lambda0", np.array([s.lambda0 for s in sols])), ("u0", np.array([s.u0 for s in sols])),
                     ("V", np.array([s.V for s in sols]))):
        assert np.max(np.abs(got[0][key] - ref)) <= 1e-6 * np.max(np.abs(ref)), key
