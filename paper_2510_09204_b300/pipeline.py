"""The three-stage selection around the SF (the paper's planning pipeline, Sec. V):
rank many candidates of each problem by constraint violation, refine the best few with
the SF, and return per problem the feasible refined trajectory of least smoothness cost.

Every stage runs in the library: sf_metrics scores the candidates, sf_select ranks
them, sf_solve refines; this module only arranges the batches.
"""
from __future__ import annotations

import numpy as np
import torch

from .sf import SFSolver, select


def refine_candidates(problems, candidates, keep=10, iters=200, precision="fp32", proj="structured",
                      tol=1e-3, rho=0.3, dt=0.05, n_xi=11, autotune=False, stream=None):
    """problems: instance dicts (shape and data; their "xi" is not used); candidates: per
    problem an array [m][n_d][n][n_xi] of candidate coefficients.  autotune: time the launch
    geometries of the refinement batch first (worth it when the same batch shape recurs).
    Returns per problem a
    dict with the chosen coefficients, the candidate's index, its metrics
    (||r_p||, max residual, smoothness cost, path length) after refinement, whether it is
    feasible (max residual <= tol), and the indices that were refined."""
    nd = int(problems[0]["n_d"])
    dev = torch.device("cuda")
    sizes = [len(c) for c in candidates]
    flat = [dict(p, xi=np.asarray(x, dtype=np.float64)) for p, cs in zip(problems, candidates) for x in cs]
    # stage 1: every candidate's max residual, keep the `keep` least violating per problem
    s1 = SFSolver(flat, nd, n_xi, rho=rho, precision=precision, proj=proj, max_iters=1, dt=dt, stream=stream)
    d1 = s1.pack(flat, device=dev)
    m1 = s1.metrics(d1, d1["xi"], stream=stream)
    kept = select(sizes, m1[:, 1].contiguous(), None, float("-inf"), keep, stream=stream).cpu().numpy()
    s1.close()
    chosen = [[j for j in kept[g] if j >= 0] for g in range(len(problems))]
    # stage 2: the SF on the kept candidates of every problem in one batch
    batch = [dict(problems[g], xi=np.asarray(candidates[g][j], dtype=np.float64))
             for g in range(len(problems)) for j in chosen[g]]
    s2 = SFSolver(batch, nd, n_xi, rho=rho, precision=precision, proj=proj, max_iters=max(iters, 1), tol=tol,
                  dt=dt, stream=stream)
    d2 = s2.pack(batch, device=dev)
    if autotune:   # costs several solves; the automatic geometry covers the SMs already
        s2.autotune(d2, d2["xi"], max(iters, 1), reps=1, stream=stream)
    xo, _, _ = s2.solve(d2, d2["xi"], iters, want_resid=False, stream=stream)
    # stage 3: feasible first by smoothness cost, else least residual
    m2 = s2.metrics(d2, xo, stream=stream)
    best = select([len(c) for c in chosen], m2[:, 1].contiguous(), m2[:, 2].contiguous(), tol, 1,
                  stream=stream).cpu().numpy()[:, 0]
    m2h = m2.cpu().numpy()
    out, base = [], 0
    for g in range(len(problems)):
        b = int(best[g])
        out.append(dict(xi=s2.unpack(xo, base + b).double().cpu().numpy(), index=int(chosen[g][b]),
                        metrics=m2h[base + b], feasible=bool(m2h[base + b, 1] <= tol), refined=list(chosen[g])))
        base += len(chosen[g])
    s2.close()
    return out
