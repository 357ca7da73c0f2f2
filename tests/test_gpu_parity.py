"""GPU parity: every CUDA step against the CPU oracle on the same seeded inputs.

Tolerances: 1e-8 relative (max |gpu - oracle| / max |oracle| over the batch)
for lambda(0), u*(x0) and V from the FP64 and mixed solvers, which both
iterate to the same FP64 root; 1e-10 for the interpolant, whose FP64 path is
an exact linear identity up to rounding; bit-exact for integer structure.
"""
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
from oracle import riccati  # noqa: E402
from paper_1507_04769_gb300 import sg  # noqa: E402

pytestmark = pytest.mark.gpu

LO, HI = synth.box(6)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def cuda(x, dtype=torch.float64):
    return torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda")


# ------------------------------------------------------------------ grid
@pytest.mark.parametrize("d,L", [(6, 0), (6, 1), (6, 2), (6, 4), (2, 6), (3, 5), (1, 7)])
def test_grid_matches_oracle(d, L):
    lo, hi = -np.arange(1, d + 1) * 0.3, np.arange(1, d + 1) * 0.5
    g = sg.Grid(d, L, lo, hi)
    og = ogrid.Grid(d, L, lo, hi)
    assert g.M == og.M == ogrid.count_nodes(d, d + L)
    assert np.array_equal(g.levels.cpu().numpy(), og.lev)
    assert np.array_equal(g.index.cpu().numpy(), og.kidx)
    assert np.max(np.abs(g.coords.cpu().numpy() - og.x)) <= 4e-16 * np.max(np.abs(hi - lo))


# ------------------------------------------------------------------ surpluses + eval
@pytest.mark.parametrize("d,L,k", [(6, 2, 3), (6, 3, 1), (3, 5, 2), (2, 6, 4), (1, 7, 1), (6, 0, 2),
                                   (4, 3, 6), (2, 4, 16)])   # k > 4: the kernel's wide-output form
def test_surpluses_match_oracle(d, L, k):
    lo, hi = synth.box(d)
    g = sg.Grid(d, L, lo, hi)
    og = ogrid.Grid(d, L, lo, hi)
    f = np.random.default_rng(10 + L).standard_normal((og.M, k))
    S = sg.Surplus(g, cuda(f))
    w = ointerp.surpluses(og, f)
    assert rel(S.W.cpu().numpy(), w) <= 1e-11


EVAL_MODES = [sg.EVAL_FP64, sg.EVAL_DF32]


@pytest.mark.parametrize("mode", EVAL_MODES, ids=["fp64", "df32"])
@pytest.mark.parametrize("d,L", [(6, 2), (6, 3), (3, 5), (2, 6)])
def test_eval_matches_oracle(d, L, mode):
    lo, hi = synth.box(d)
    g = sg.Grid(d, L, lo, hi)
    og = ogrid.Grid(d, L, lo, hi)
    f = np.random.default_rng(20 + L).standard_normal((og.M, 3))
    S = sg.Surplus(g, cuda(f))
    w = ointerp.surpluses(og, f)
    # ragged query count; uniform + clustered + exact nodes + box corners + outside
    xq = np.concatenate([synth.mixed_queries(301, lo, hi, seed=3), og.x[:17],
                         np.array([lo, hi, 0.5 * (lo + hi)])])
    u = sg.eval_feedback(S, cuda(xq), mode=mode).cpu().numpy()
    ref = ointerp.eval_surplus(og, w, xq)
    assert rel(u, ref) <= 1e-10
    # interpolation is exact at the nodes
    assert np.max(np.abs(u[301:318] - f[:17])) <= 1e-12 * np.max(np.abs(f))


@pytest.mark.parametrize("mode", EVAL_MODES, ids=["fp64", "df32"])
def test_eval_slightly_outside_box(mode):
    """Outside the box the same polynomial is evaluated; at low degree this is
    well conditioned, so the two forms still agree."""
    g = sg.Grid(6, 2, LO, HI)
    og = ogrid.Grid(6, 2, LO, HI)
    f = np.random.default_rng(8).standard_normal((og.M, 3))
    S = sg.Surplus(g, cuda(f))
    xq = np.array([1.05 * HI, 1.05 * LO, [0.9, -0.9, 0.0, 0.2, -0.85, 0.81]])
    u = sg.eval_feedback(S, cuda(xq), mode=mode).cpu().numpy()
    ref = ointerp.eval_surplus(og, ointerp.surpluses(og, f), xq)
    assert rel(u, ref) <= 1e-10


def test_eval_df32_agrees_with_fp64_everywhere():
    """Pair-of-floats evaluation against the FP64 kernel on every query of a
    level-4 batch (mixed distribution), 1e-12 relative to the largest value."""
    g = sg.Grid(6, 4, LO, HI)
    f = np.random.default_rng(12).standard_normal((g.M, 3))
    S = sg.Surplus(g, cuda(f))
    xq = cuda(synth.mixed_queries(200_000, LO, HI, seed=13))
    a = sg.eval_feedback(S, xq, mode=sg.EVAL_DF32)
    b = sg.eval_feedback(S, xq, mode=sg.EVAL_FP64)
    assert ((a - b).abs().max() / b.abs().max()).item() <= 1e-12


def test_eval_empty_and_single():
    g = sg.Grid(6, 2, LO, HI)
    S = sg.Surplus(g, cuda(np.ones((g.M, 3))))
    assert sg.eval_feedback(S, torch.empty((0, 6), dtype=torch.float64, device="cuda")).shape == (0, 3)
    u = sg.eval_feedback(S, cuda(np.zeros((1, 6)))).cpu().numpy()
    assert np.allclose(u, 1.0, atol=1e-14)   # the constant is reproduced


@pytest.mark.parametrize("mode", EVAL_MODES, ids=["fp64", "df32"])
def test_eval_full_size_sampled(mode):
    """Level-4 grid (1457 nodes) at 1e6 mixed queries, in the launch the benchmark
    times; 256 sampled queries are recomputed by the oracle."""
    g = sg.Grid(6, 4, LO, HI)
    og = ogrid.Grid(6, 4, LO, HI)
    f = np.random.default_rng(4).standard_normal((og.M, 3))
    S = sg.Surplus(g, cuda(f))
    xq = synth.mixed_queries(1_000_000, LO, HI, seed=1)
    u = sg.eval_feedback(S, cuda(xq), mode=mode).cpu().numpy()
    idx = np.random.default_rng(5).choice(xq.shape[0], 256, replace=False)
    w = ointerp.surpluses(og, f)
    ref = ointerp.eval_surplus(og, w, xq[idx])
    assert rel(u[idx], ref) <= 1e-10
    assert np.all(np.isfinite(u))


# ------------------------------------------------------------------ BVP: LQ closed form
@pytest.mark.parametrize("prec", [sg.PREC_FP64, sg.PREC_MIXED])
def test_lq_matches_discrete_riccati(prec):
    params = synth.lq_params(0)
    pr = oprob.make(params)
    X0 = synth.uniform_queries(40, LO, HI, seed=21)
    for T, N in ((1.0, 4), (2.0, 16), (10.0, 128)):
        res = sg.solve_bvps(sg.problem_from(params), cuda(X0), T, N, tol=1e-12, precision=prec)
        st = res["status"].cpu().numpy()
        assert np.all(st == sg.CONVERGED)
        P0 = riccati.riccati_p0(pr, T, N, discrete=True)
        ref = X0 @ P0.T
        assert rel(res["lambda0"].cpu().numpy(), ref) <= 1e-10
        if prec == sg.PREC_FP64:
            assert np.all(res["iters"].cpu().numpy() <= 2)


def test_lq_continuous_value_fine_mesh():
    params = synth.lq_params(0)
    pr = oprob.make(params)
    X0 = synth.uniform_queries(8, LO, HI, seed=22)
    res = sg.solve_bvps(sg.problem_from(params), cuda(X0), 10.0, 1024, tol=1e-12)
    V = np.array([riccati.lq_value(pr, x, 10.0) for x in X0])
    assert rel(res["V"].cpu().numpy(), V) <= 1e-8


# ------------------------------------------------------------------ BVP: attitude vs oracle
def _oracle(params, X0, T, N):
    pr = oprob.make(params)
    T = np.broadcast_to(T, (X0.shape[0],))
    N = np.broadcast_to(N, (X0.shape[0],))
    sols = [obvp.solve(pr, X0[i], float(T[i]), int(N[i])) for i in range(X0.shape[0])]
    assert all(s.status == obvp.CONVERGED for s in sols)
    return (np.array([s.lambda0 for s in sols]), np.array([s.u0 for s in sols]),
            np.array([s.V for s in sols]), sols)


@pytest.fixture(scope="module")
def att_case():
    params = synth.attitude_params(0)
    X0 = np.concatenate([synth.uniform_queries(10, LO, HI, seed=31), np.zeros((1, 6))])
    T = np.array([5.0, 10.0, 20.0, 3.0, 7.5, 20.0, 10.0, 5.0, 12.0, 20.0, 20.0])
    N = np.array([8, 17, 64, 1, 33, 128, 40, 16, 3, 100, 64])   # ragged, incl. N = 1
    return params, X0, T, N, _oracle(params, X0, T, N)


FORMS = [(sg.PREC_FP64, False), (sg.PREC_MIXED, False), (sg.PREC_FP64, True), (sg.PREC_MIXED, True),
         (sg.PREC_MIXED_PAIR, False), (sg.PREC_MIXED_PAIR, True)]
FORM_IDS = ["fp64", "mixed", "fp64-persistent", "mixed-persistent", "mixedpair", "mixedpair-persistent"]
GFORMS = [(p, q, g) for (p, q) in FORMS for g in (False, True)]
GFORM_IDS = [f"{i}{'-graph' if g else ''}" for i in FORM_IDS for g in (False, True)]


@pytest.mark.parametrize("prec,persistent,graph", GFORMS, ids=GFORM_IDS)
def test_attitude_matches_oracle(att_case, prec, persistent, graph):
    params, X0, T, N, (lam, u, V, _) = att_case
    res = sg.solve_bvps(sg.problem_from(params), cuda(X0), cuda(T), cuda(N, torch.int32),
                        tol=1e-12, precision=prec, persistent=persistent, graph=graph)
    assert np.all(res["status"].cpu().numpy() == sg.CONVERGED)
    assert rel(res["lambda0"].cpu().numpy(), lam) <= 1e-8
    assert rel(res["u0"].cpu().numpy(), u) <= 1e-8
    assert rel(res["V"].cpu().numpy(), V) <= 1e-8
    # the origin is an equilibrium: 0 iterations, exact zeros
    assert res["iters"][-1].item() == 0 and res["V"][-1].item() == 0.0


def test_attitude_residual_at_default_tolerance(att_case):
    """At the default 1e-8 residual tolerance the oracle, recomputing the
    residual of the collocation system on the GPU's solution, agrees."""
    params, X0, T, N, _ = att_case
    res = sg.solve_bvps(sg.problem_from(params), cuda(X0), cuda(T), cuda(N, torch.int32), return_Y=True)
    Y = res["Y"].cpu().numpy()
    pr = oprob.make(params)
    for i in range(X0.shape[0]):
        F = obvp.residual(pr, Y[i, :3 * N[i] + 1], X0[i], T[i], N[i])
        assert np.max(np.abs(F)) <= 1e-8


def test_attitude_oracle_solution_trajectory(att_case):
    params, X0, T, N, (_, _, _, sols) = att_case
    res = sg.solve_bvps(sg.problem_from(params), cuda(X0), cuda(T), cuda(N, torch.int32), tol=1e-12,
                        return_Y=True)
    Y = res["Y"].cpu().numpy()
    for i in (0, 2, 5):
        ref = sols[i].Y
        assert rel(Y[i, :3 * N[i] + 1], ref) <= 1e-8


@pytest.mark.parametrize("prec,persistent", FORMS, ids=FORM_IDS)
def test_batch_independence_bitwise(att_case, prec, persistent):
    """Each node's result is the same alone and inside a batch (Section 3: no
    communication between nodes)."""
    params, X0, T, N, _ = att_case
    prob = sg.problem_from(params)
    kw = dict(n_max=128, precision=prec, persistent=persistent)
    full = sg.solve_bvps(prob, cuda(X0), cuda(T), cuda(N, torch.int32), **kw)
    perm = np.random.default_rng(0).permutation(X0.shape[0])
    shuf = sg.solve_bvps(prob, cuda(X0[perm]), cuda(T[perm]), cuda(N[perm], torch.int32), **kw)
    for key in ("lambda0", "u0", "V", "iters"):
        assert torch.equal(full[key][perm], shuf[key])
    alone = sg.solve_bvps(prob, cuda(X0[2:3]), cuda(T[2:3]), cuda(N[2:3], torch.int32), **kw)
    assert torch.equal(alone["lambda0"][0], full["lambda0"][2])


@pytest.mark.parametrize("persistent", [False, True])
def test_graph_replay_reuses_buffers(att_case, persistent):
    """The cached graph is replayed when the same buffers come back; a replay on
    new inputs written into the same input tensors gives the host-loop result."""
    params, X0, T, N, _ = att_case
    prob = sg.problem_from(params)
    x0, Tt, Nt = cuda(X0), cuda(T), cuda(N, torch.int32)
    nmax = int(N.max())
    ws = torch.empty(sg.workspace_bytes(len(X0), nmax, sg.PREC_MIXED), dtype=torch.uint8, device="cuda")
    out = None
    for rep in range(3):
        if rep == 2:
            x0.copy_(cuda(0.5 * X0))
        out = sg.solve_bvps(prob, x0, Tt, Nt, precision=sg.PREC_MIXED, persistent=persistent, graph=True,
                            workspace=ws, n_max=nmax, out=out)
        ref = sg.solve_bvps(prob, x0, Tt, Nt, precision=sg.PREC_MIXED, persistent=persistent, n_max=nmax)
        for key in ("lambda0", "V", "status", "iters"):
            assert torch.equal(out[key], ref[key]), (rep, key)


@pytest.mark.parametrize("prec", [sg.PREC_MIXED, sg.PREC_FP64], ids=["mixed", "fp64"])
def test_graph_per_mesh_size_matches_one_graph_bitwise(prec):
    """graph = 2 (the nodes of each mesh size gathered into a sub-batch with a
    graph and a stream of its own) gives bitwise the one-graph results, on a
    batch of three mesh sizes, with invalid inputs among the nodes."""
    params = synth.attitude_params(0)
    prob = sg.problem_from(params)
    X0 = synth.uniform_queries(300, LO, HI, seed=61)
    T, N = synth.mixed_horizons(300, seed=62)
    N = N.copy()
    N[7] = 300                                   # above n_max: SG_BADINPUT
    X0[11, 2] = np.nan                           # non-finite state: SG_BADINPUT
    args = (prob, cuda(X0), cuda(T), cuda(N, torch.int32))
    one = sg.solve_bvps(*args, precision=prec, graph=1, n_max=256)
    for rep in range(2):                         # the second call replays the cached graphs
        per = sg.solve_bvps(*args, precision=prec, graph=2, n_max=256)
        for key in ("lambda0", "u0", "V", "status", "iters"):
            assert torch.equal(torch.nan_to_num(one[key]), torch.nan_to_num(per[key])), (rep, key)
    st = one["status"].cpu().numpy()
    assert st[7] == sg.BADINPUT and st[11] == sg.BADINPUT and np.sum(st == sg.CONVERGED) == 298


def test_condensation_block_shape_is_bitwise_neutral(att_case):
    """cond_warps (intervals per block of the FP32 condensation) is a launch
    shape: 2, 4 and 8 give bitwise the same solve, in the host loop and the
    graph per mesh size."""
    params, X0, T, N, _ = att_case
    prob = sg.problem_from(params)
    args = (prob, cuda(X0), cuda(T), cuda(N, torch.int32))
    ref = sg.solve_bvps(*args, precision=sg.PREC_MIXED, n_max=128, cond_warps=4)
    for cw in (2, 8):
        for graph in (0, 2):
            got = sg.solve_bvps(*args, precision=sg.PREC_MIXED, n_max=128, cond_warps=cw, graph=graph)
            for key in ("lambda0", "u0", "V", "status", "iters"):
                assert torch.equal(got[key], ref[key]), (cw, graph, key)


def test_autotuner_picks_a_form_and_caches_it(att_case):
    params, X0, T, N, _ = att_case
    prob = sg.problem_from(params)
    choice, ms = sg.autotune_solve(prob, cuda(X0), cuda(T), cuda(N, torch.int32), precision=sg.PREC_MIXED,
                                   force=True)
    assert set(ms) == set(sg.FORM_NAMES) and all(v > 0 for v in ms.values())
    again, ms2 = sg.autotune_solve(prob, cuda(X0), cuda(T), cuda(N, torch.int32), precision=sg.PREC_MIXED)
    assert again == choice and all(v != v for v in ms2.values())   # cached: nothing re-timed
    a = sg.solve_bvps(prob, cuda(X0), cuda(T), cuda(N, torch.int32), precision=sg.PREC_MIXED, **choice)
    b = sg.solve_bvps(prob, cuda(X0), cuda(T), cuda(N, torch.int32), precision=sg.PREC_MIXED)
    assert rel(a["lambda0"].cpu().numpy(), b["lambda0"].cpu().numpy()) <= 1e-8


def test_persistent_and_phase_forms_agree(att_case):
    """Both forms take the same Newton steps (same residual, elimination and
    line search), so they agree to rounding at every tolerance."""
    params, X0, T, N, _ = att_case
    prob = sg.problem_from(params)
    for prec in (sg.PREC_FP64, sg.PREC_MIXED):
        a = sg.solve_bvps(prob, cuda(X0), cuda(T), cuda(N, torch.int32), precision=prec)
        b = sg.solve_bvps(prob, cuda(X0), cuda(T), cuda(N, torch.int32), precision=prec, persistent=True)
        assert torch.equal(a["status"], b["status"])
        assert rel(b["lambda0"].cpu().numpy(), a["lambda0"].cpu().numpy()) <= 1e-8


def test_edge_cases_and_bad_input():
    params = synth.attitude_params(0)
    prob = sg.problem_from(params)
    empty = sg.solve_bvps(prob, torch.empty((0, 6), dtype=torch.float64, device="cuda"), 1.0, 4, n_max=4)
    assert empty["V"].numel() == 0
    X0 = np.array([[0.1] * 6, [np.nan] + [0.0] * 5, [0.1] * 6, [0.1] * 6])
    T = np.array([1.0, 1.0, -1.0, 1.0])
    N = np.array([4, 4, 4, 9])          # last one exceeds n_max
    res = sg.solve_bvps(prob, cuda(X0), cuda(T), cuda(N, torch.int32), n_max=8)
    st = res["status"].cpu().numpy()
    assert st[0] == sg.CONVERGED
    assert list(st[1:]) == [sg.BADINPUT] * 3
    with pytest.raises(sg.SGError):
        sg.solve_bvps(prob, cuda(X0[:1]), 1.0, 4, n_max=4,
                      workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))


def test_max_iter_reported():
    params = synth.attitude_params(0)
    X0 = synth.uniform_queries(4, LO, HI, seed=41)
    res = sg.solve_bvps(sg.problem_from(params), cuda(X0), 20.0, 64, max_iter=1)
    assert np.all(res["status"].cpu().numpy() == sg.MAXITER)
    assert np.all(res["iters"].cpu().numpy() == 1)


def test_full_size_batched_solve_sampled():
    """Level-4 grid, 1457 nodes, horizons {10, 20, 40} with N = 64/128/256, in
    the launch the benchmark times; 6 sampled nodes are re-solved by the oracle."""
    params = synth.attitude_params(0)
    g = sg.Grid(6, 4, LO, HI)
    og = ogrid.Grid(6, 4, LO, HI)
    T, N = synth.mixed_horizons(g.M, seed=2)
    for prec, persistent in FORMS:
        res = sg.solve_bvps(sg.problem_from(params), g.coords, cuda(T), cuda(N, torch.int32), tol=1e-12,
                            precision=prec, persistent=persistent)
        st = res["status"].cpu().numpy()
        assert np.all(st == sg.CONVERGED), np.bincount(st)
        idx = np.random.default_rng(7).choice(g.M, 6, replace=False)
        lam, u, V, _ = _oracle(params, og.x[idx], T[idx], N[idx])
        assert rel(res["lambda0"].cpu().numpy()[idx], lam) <= 1e-8
        assert rel(res["u0"].cpu().numpy()[idx], u) <= 1e-8
        assert rel(res["V"].cpu().numpy()[idx], V) <= 1e-8


# ------------------------------------------------------------------ 3xTF32 tensor-core contraction
def _tf32x3_bound(og, w, xq):
    """A-priori bound of the split-TF32 contraction: |du_q| <= gamma sum_m |phi_qm| |w_m|,
    gamma = (d + 3) 2^-22 + ceil(log2 M) 2^-23 (TF32 splitting of both operands,
    FP32 basis values and FP32 accumulation)."""
    phi = ointerp.basis_table(og, ointerp.to_unit(og, xq))
    gamma = (og.d + 3) * 2.0 ** -22 + np.ceil(np.log2(og.M)) * 2.0 ** -23
    return gamma * (np.abs(phi) @ np.abs(w))


@pytest.mark.parametrize("d,L,k", [(6, 2, 3), (6, 4, 3), (3, 5, 2), (6, 3, 8), (1, 5, 2), (4, 3, 5), (2, 6, 1)])
def test_tf32x3_within_stated_bound(d, L, k):
    lo, hi = synth.box(d)
    g = sg.Grid(d, L, lo, hi)
    og = ogrid.Grid(d, L, lo, hi)
    f = np.random.default_rng(30 + L).standard_normal((og.M, k))
    S = sg.Surplus(g, cuda(f))
    w = ointerp.surpluses(og, f)
    xq = np.concatenate([synth.mixed_queries(333, lo, hi, seed=31), og.x[:5]])
    u = sg.eval_feedback(S, cuda(xq), mode=sg.EVAL_TF32X3).cpu().numpy()
    ref = ointerp.eval_surplus(og, w, xq)
    bound = _tf32x3_bound(og, w, xq)
    assert np.all(np.isfinite(u))
    assert np.max(np.abs(u - ref) / bound) <= 1.0
    assert rel(u, ref) <= 1e-5


def _kernels_launched(fn):
    """Names of the library kernels launched by fn (per-launch timing)."""
    import ctypes as C
    sg.LIB.sg_timing_enable(1)
    try:
        fn()
        torch.cuda.synchronize()
    finally:
        sg.LIB.sg_timing_enable(0)
    n_max, name_len = 64, 64
    names = C.create_string_buffer(n_max * name_len)
    nk = C.c_int()
    sg.LIB.sg_timing_collect.argtypes = [C.c_int, C.c_char_p, C.c_int, C.c_void_p, C.c_void_p,
                                         C.POINTER(C.c_int)]
    assert sg.LIB.sg_timing_collect(n_max, names, name_len, None, None, C.byref(nk)) == 0
    raw = names.raw
    return {raw[i * name_len:(i + 1) * name_len].split(b"\0", 1)[0].decode() for i in range(nk.value)}


@pytest.mark.parametrize("d,L,k,kernel", [(6, 4, 3, "k_eval_sf_tf32x3"), (6, 2, 8, "k_eval_sf_tf32x3"),
                                          (1, 5, 2, "k_eval_tf32x3")])
def test_tf32x3_kernel_for_the_shape(d, L, k, kernel):
    """The sum-factorised kernel serves grids whose plan fits (d >= 2); others
    keep the per-node contraction.  Both agree with the FP64 evaluation."""
    lo, hi = synth.box(d)
    g = sg.Grid(d, L, lo, hi)
    f = np.random.default_rng(3).standard_normal((g.M, k))
    S = sg.Surplus(g, cuda(f))
    xq = cuda(synth.mixed_queries(5000, lo, hi, seed=4))
    out = {}
    names = _kernels_launched(lambda: out.setdefault("u", sg.eval_feedback(S, xq, mode=sg.EVAL_TF32X3)))
    assert kernel in names, names
    ref = sg.eval_feedback(S, xq, mode=sg.EVAL_FP64)
    assert ((out["u"] - ref).abs().max() / ref.abs().max()).item() <= 1e-5


def test_surplus_tables_reused_across_grids():
    """Surplus builds on grids of the same structure reuse the host-made tables
    (cached per d, L, k): grids on different boxes, a different k and a
    different level in between all give the oracle's surpluses and values."""
    rng = np.random.default_rng(21)
    for d, L, k, half in [(4, 3, 2, 1.0), (4, 3, 2, 0.3), (4, 3, 3, 0.3), (4, 2, 2, 0.3), (4, 3, 2, 2.0)]:
        lo, hi = -half * np.ones(d), half * np.ones(d)
        lo[0] -= 0.5
        g = sg.Grid(d, L, lo, hi)
        og = ogrid.Grid(d, L, lo, hi)
        f = rng.standard_normal((og.M, k))
        S = sg.Surplus(g, cuda(f))
        w = ointerp.surpluses(og, f)
        xq = synth.uniform_queries(200, lo, hi, seed=22)
        ref = ointerp.eval_surplus(og, w, xq)
        for mode in (sg.EVAL_FP64, sg.EVAL_DF32):
            u = sg.eval_feedback(S, cuda(xq), mode=mode).cpu().numpy()
            assert rel(u, ref) <= 1e-10, (d, L, k, half, mode)
        u = sg.eval_feedback(S, cuda(xq), mode=sg.EVAL_TF32X3).cpu().numpy()
        assert np.max(np.abs(u - ref) / _tf32x3_bound(og, w, xq)) <= 1.0, (d, L, k, half)


def test_tf32x3_at_nodes_edges_and_outside():
    """Queries on grid nodes (up to the last bit), next to them, on the box
    faces and outside the box: finite and within the stated bound."""
    d, L, k = 6, 4, 3
    lo, hi = synth.box(d)
    g = sg.Grid(d, L, lo, hi)
    og = ogrid.Grid(d, L, lo, hi)
    f = np.random.default_rng(8).standard_normal((og.M, k))
    S = sg.Surplus(g, cuda(f))
    w = ointerp.surpluses(og, f)
    rng = np.random.default_rng(9)
    nodes = og.x[rng.choice(og.M, 200, replace=False)]
    near = nodes * (1 + rng.choice([-1, 1], nodes.shape) * 1e-15)
    faces = synth.uniform_queries(100, lo, hi, seed=10)
    faces[np.arange(100), rng.integers(0, d, 100)] = np.where(rng.random(100) < 0.5, lo[0], hi[0])
    outside = synth.uniform_queries(100, lo - 0.2 * (hi - lo), hi + 0.2 * (hi - lo), seed=11)
    xq = np.concatenate([nodes, near, faces, outside])
    u = sg.eval_feedback(S, cuda(xq), mode=sg.EVAL_TF32X3).cpu().numpy()
    ref = ointerp.eval_surplus(og, w, xq)
    assert np.all(np.isfinite(u))
    assert np.max(np.abs(u - ref) / _tf32x3_bound(og, w, xq)) <= 1.0


def test_tf32x3_smooth_feedback_at_full_size():
    """A smooth feedback-like function interpolated on the level-4 grid and
    evaluated at the 1e6 mixed queries of the benchmark: 3xTF32 on the tensor
    cores within 2e-6 of the FP64 evaluation, relative to max |u| (the FP64
    evaluation matches the oracle to 1e-10, test_eval_full_size_sampled)."""
    g = sg.Grid(6, 4, LO, HI)
    x = g.coords.cpu().numpy()
    K = np.random.default_rng(0).standard_normal((3, 6))
    f = -(x @ K.T) + 0.3 * np.sin(x @ K.T) + 0.1 * np.prod(np.cos(x), axis=1)[:, None]
    S = sg.Surplus(g, cuda(f))
    xq = cuda(synth.mixed_queries(1_000_000, LO, HI, seed=1))
    u = sg.eval_feedback(S, xq, mode=sg.EVAL_TF32X3)
    ref = sg.eval_feedback(S, xq, mode=sg.EVAL_FP64)
    assert torch.isfinite(u).all()
    assert ((u - ref).abs().max() / ref.abs().max()).item() <= 2e-6


def test_tf32x3_full_size_sampled():
    g = sg.Grid(6, 4, LO, HI)
    og = ogrid.Grid(6, 4, LO, HI)
    f = np.random.default_rng(4).standard_normal((og.M, 3))
    S = sg.Surplus(g, cuda(f))
    xq = synth.mixed_queries(1_000_000, LO, HI, seed=1)
    u = sg.eval_feedback(S, cuda(xq), mode=sg.EVAL_TF32X3).cpu().numpy()
    assert np.all(np.isfinite(u))
    idx = np.random.default_rng(5).choice(xq.shape[0], 256, replace=False)
    w = ointerp.surpluses(og, f)
    ref = ointerp.eval_surplus(og, w, xq[idx])
    assert np.max(np.abs(u[idx] - ref) / _tf32x3_bound(og, w, xq[idx])) <= 1.0


@pytest.mark.gpu
def test_library_sincos_within_few_ulp():
    """The FP64 sine/cosine inside the right-hand side (minimax polynomials on
    |x| <= pi/4, the CUDA library beyond) against numpy's, within 4 ulp."""
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(-np.pi / 4, np.pi / 4, 200_000),
                        np.linspace(-np.pi / 4, np.pi / 4, 10_001),
                        [0.0, -0.0, np.pi / 4, -np.pi / 4, np.nextafter(np.pi / 4, 1.0), 1e-300, -1e-12],
                        rng.uniform(-20.0, 20.0, 50_000)])
    s, c = sg.sincos_probe(torch.as_tensor(x, device="cuda"))
    s, c = s.cpu().numpy(), c.cpu().numpy()
    eps = np.finfo(np.float64).eps
    for got, ref in ((s, np.sin(x)), (c, np.cos(x))):
        err = np.abs(got - ref)
        assert np.all(err <= 4 * eps * np.abs(ref) + 1e-300), float(np.max(err / np.maximum(np.abs(ref), 1e-300)))
    assert np.all(s[x == 0.0] == 0.0) and np.all(c[x == 0.0] == 1.0)
