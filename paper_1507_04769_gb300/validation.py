"""Error-controlled solves and the pointwise validation of Section 4.1.

The total error of the interpolated value function at a point x,
e_interp + e_bvp = I^q(V)(x) - V(x), is estimated by solving the
characteristic BVP at x itself with an error-controlled solver whose tolerance
is far below that error (Section 4.1, Eq. validate), in parallel over the
sample points (causality free).

Error control here is mesh doubling on the fixed-width Lobatto IIIA mesh: a
node is solved on N and 2N intervals; at the mesh points the four-stage
Lobatto IIIA solution converges at order 2s - 2 = 6, so |V_N - V_2N| / 63 (and
the same for lambda(0)) estimates the error of the 2N solution.  Nodes whose
estimate is above the tolerance double again.  Every solve runs in the
library (sg_solve_bvps); this module only keeps the per-node bookkeeping.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import sg, surfaces

ORDER = 6   # superconvergence order of four-stage Lobatto IIIA at the mesh points


@dataclass
class Controlled:
    lambda0: torch.Tensor   # (n, 6)
    u0: torch.Tensor        # (n, 3)
    V: torch.Tensor         # (n,)
    N: np.ndarray           # intervals of the accepted solve per node
    err_est: np.ndarray     # estimated error of V (and lambda0, the larger) per node
    ok: np.ndarray          # estimate within tolerance and every solve converged


def solve_error_controlled(problem: sg.Problem, x0: torch.Tensor, T: torch.Tensor, tol: float,
                           h0: float = 5.0 / 32.0, max_doublings: int = 5, precision: int = sg.PREC_FP64,
                           newton_tol: float = 1e-12, max_iter: int = 100,
                           target: torch.Tensor | None = None) -> Controlled:
    """Solves every node to an estimated error of V and lambda(0) below `tol`.
    target: per-node target attitudes (n, 3) for the attitude family, or None."""
    x0 = x0.to(torch.float64).contiguous()
    T = T.to(torch.float64).contiguous()
    n = x0.shape[0]
    dev = x0.device
    Th = T.cpu().numpy()
    N = np.maximum(1, np.ceil(Th / h0 - 1e-9)).astype(np.int64)

    def solve(idx, Nsub):
        Nd = torch.as_tensor(Nsub.astype(np.int32), device=dev)
        tg = target[idx].contiguous() if target is not None else None
        prob = surfaces._with_target(problem, tg) if target is not None else problem
        return sg.solve_bvps(prob, x0[idx].contiguous(), T[idx].contiguous(), Nd, tol=newton_tol,
                             max_iter=max_iter, precision=precision, n_max=int(Nsub.max()))

    out = {"lambda0": torch.full((n, 6), float("nan"), dtype=torch.float64, device=dev),
           "u0": torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev),
           "V": torch.full((n,), float("nan"), dtype=torch.float64, device=dev)}
    err = np.full(n, np.inf)
    ok = np.zeros(n, dtype=bool)
    idx = torch.arange(n, device=dev)
    prev = solve(idx, N)
    for _ in range(max_doublings):
        if idx.numel() == 0:
            break
        sub_N = N[idx.cpu().numpy()] * 2
        cur = solve(idx, sub_N)
        dV = (cur["V"] - prev["V"]).abs()
        dl = (cur["lambda0"] - prev["lambda0"]).abs().amax(dim=1)
        est = (torch.maximum(dV, dl) / (2 ** ORDER - 1)).cpu().numpy()
        conv = ((cur["status"] == sg.CONVERGED) & (prev["status"] == sg.CONVERGED)).cpu().numpy()
        done = conv & (est <= tol)
        ii = idx.cpu().numpy()
        N[ii] = sub_N
        err[ii] = np.where(conv, est, np.inf)
        if done.any():
            sel = torch.as_tensor(np.nonzero(done)[0], device=dev)
            gi = idx[sel]
            for k in out:
                out[k][gi] = cur[k][sel]
            ok[ii[done]] = True
        keep = torch.as_tensor(np.nonzero(~done)[0], device=dev)
        idx = idx[keep]
        prev = {k: v[keep] for k, v in cur.items()}
    if idx.numel():   # not within tolerance: keep the finest solve, flagged
        for k in out:
            out[k][idx] = prev[k]
    return Controlled(lambda0=out["lambda0"], u0=out["u0"], V=out["V"], N=N, err_est=err, ok=ok)


@dataclass
class Validation:
    points: np.ndarray
    interp: np.ndarray      # I^q(.)(x) at the points, (Q, k)
    reference: np.ndarray   # error-controlled solution at the points, (Q, k)
    err_est: np.ndarray     # error estimate of the reference per point
    ok: np.ndarray

    def stats(self, col: int = 0) -> dict:
        e = self.interp[self.ok, col] - self.reference[self.ok, col]
        ref = np.abs(self.reference[self.ok, col])
        rel = np.abs(e) / np.where(ref > 0, ref, np.inf)
        return {"points": int(self.ok.sum()), "mae": float(np.abs(e).mean()), "max": float(np.abs(e).max()),
                "var": float(np.var(e)), "relative_mae": float(rel.mean()),
                "reference_err_est_max": float(self.err_est[self.ok].max())}


def validate_feedback(problem: sg.Problem, surplus: sg.Surplus, points: torch.Tensor, T: float, tol: float,
                      mode: int = sg.EVAL_DF32, **kw) -> Validation:
    """Section 4.1 for the feedback: I^q(u*)(x) against u*(x) from error-controlled
    solves at the sample points (state space, horizon T)."""
    pts = points.to(torch.float64).contiguous()
    Tq = torch.full((pts.shape[0],), float(T), dtype=torch.float64, device=pts.device)
    ref = solve_error_controlled(problem, pts, Tq, tol, **kw)
    interp = sg.eval_feedback(surplus, pts, mode=mode).cpu().numpy()
    return Validation(points=pts.cpu().numpy(), interp=interp, reference=ref.u0.cpu().numpy()[:, :interp.shape[1]],
                      err_est=ref.err_est, ok=ref.ok)


def validate_value(problem: sg.Problem, surplus: sg.Surplus, points: torch.Tensor, T: float, tol: float,
                   value_col: int, mode: int = sg.EVAL_DF32, target: torch.Tensor | None = None,
                   **kw) -> Validation:
    """Section 4.1 for the value function: I^q(V)(x) (output `value_col` of the
    surplus handle) against V(x) from error-controlled solves at the points
    (state space, horizon T; per-point target attitudes for Example II)."""
    pts = points.to(torch.float64).contiguous()
    Tq = torch.full((pts.shape[0],), float(T), dtype=torch.float64, device=pts.device)
    ref = solve_error_controlled(problem, pts, Tq, tol, target=target, **kw)
    interp = sg.eval_feedback(surplus, pts, mode=mode).cpu().numpy()[:, value_col:value_col + 1]
    return Validation(points=pts.cpu().numpy(), interp=interp, reference=ref.V.cpu().numpy()[:, None],
                      err_est=ref.err_est, ok=ref.ok)
