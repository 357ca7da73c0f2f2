"""Runs one step of the hot path at a chosen size, for profiling.

  python -m paper_1507_04769_gb300.cases solve --nodes 300 --precision mixed
  python -m paper_1507_04769_gb300.cases eval --queries 200000 --mode fp64

The inputs are the benchmark's (level-4 attitude grid, horizons {10, 20, 40}
with N = 6.4 T, mixed query distribution), cut to the requested size.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import torch  # noqa: E402

import synth  # noqa: E402
from paper_1507_04769_gb300 import sg  # noqa: E402

MODES = {"fp64": sg.EVAL_FP64, "tf32x3": sg.EVAL_TF32X3, "df32": sg.EVAL_DF32}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["solve", "eval"])
    ap.add_argument("--nodes", type=int, default=1457)
    ap.add_argument("--precision", choices=["fp64", "mixed", "mixed-pair"], default="mixed")
    ap.add_argument("--queries", type=int, default=200_000)
    ap.add_argument("--mode", choices=sorted(MODES), default="fp64")
    ap.add_argument("--level", type=int, default=4)
    ap.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args(argv)
    lo, hi = synth.box(6)
    g = sg.Grid(6, a.level, lo, hi)
    prob = sg.problem_from(synth.attitude_params(0))
    T, N = synth.mixed_horizons(g.M, seed=2)
    n = min(a.nodes, g.M)
    x0 = g.coords[:n]
    Td = torch.as_tensor(T[:n], device="cuda")
    Nd = torch.as_tensor(N[:n], dtype=torch.int32, device="cuda")
    prec = {"mixed": sg.PREC_MIXED, "mixed-pair": sg.PREC_MIXED_PAIR, "fp64": sg.PREC_FP64}[a.precision]
    if a.what == "solve":
        for _ in range(a.repeat):
            res = sg.solve_bvps(prob, x0, Td, Nd, precision=prec, n_max=int(N[:n].max()))
        torch.cuda.synchronize()
        print("converged", int((res["status"] == sg.CONVERGED).sum()), "of", n)
        return 0
    vals = torch.sin(g.coords).sum(dim=1, keepdim=True).repeat(1, 3).contiguous()
    S = sg.Surplus(g, vals)
    xq = torch.as_tensor(synth.mixed_queries(a.queries, lo, hi, seed=1), device="cuda")
    for _ in range(a.repeat):
        u = sg.eval_feedback(S, xq, mode=MODES[a.mode])
    torch.cuda.synchronize()
    print("eval", tuple(u.shape), float(u.abs().max()))
    return 0


if __name__ == "__main__":
    sys.exit(main())
