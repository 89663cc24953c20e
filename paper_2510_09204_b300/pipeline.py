"""The three-stage selection around the SF (the paper's planning pipeline, Sec. V):
rank many candidates of each problem by constraint violation, refine the best few with
the SF, and return per problem the feasible refined trajectory of least smoothness cost.

Every stage runs in the library: sf_metrics scores the candidates, sf_select ranks
them, sf_solve refines; this module only arranges the batches.
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np
import torch

from .sf import SFSolver, select


class HandleCache:
    """SFSolver handles kept per (instance shapes, solver settings), least recently used
    first out: a planner that refines batches of the same shapes again and again pays
    sf_create (the FP64 factorisation of every shape, the launch plan, the allocations)
    once.  The instance data (boundary values, obstacles, candidates) are arguments of
    each solve, so a handle serves any batch with the same shapes."""

    def __init__(self, capacity=8):
        self.capacity = int(capacity)
        self._h = OrderedDict()

    @staticmethod
    def _shape_key(inst):
        f = lambda v: tuple(float(x) for x in np.ravel(v))
        return (int(inst["n"]), int(inst["n_obs"]), int(inst["H"]), bool(inst.get("dyn_obs", False)),
                float(inst["a"]), float(inst["b"]), f(inst["pmin"]), f(inst["pmax"]))

    def get(self, insts, n_d, n_xi, **settings):
        key = (tuple(self._shape_key(i) for i in insts), int(n_d), int(n_xi), tuple(sorted(settings.items())))
        s = self._h.pop(key, None)
        if s is None:
            s = SFSolver(insts, n_d, n_xi, **settings)
            while len(self._h) >= self.capacity:
                self._h.popitem(last=False)[1].close()
        self._h[key] = s
        return s

    def close(self):
        while self._h:
            self._h.popitem()[1].close()


def refine_candidates(problems, candidates, keep=10, iters=200, precision="fp32", proj="structured",
                      tol=1e-3, rho=0.3, dt=0.05, n_xi=11, autotune=False, stream=None, cache=None):
    """problems: instance dicts (shape and data; their "xi" is not used); candidates: per
    problem an array [m][n_d][n][n_xi] of candidate coefficients.  autotune: time the launch
    geometries of the refinement batch first (worth it when the same batch shape recurs).
    Returns per problem a
    dict with the chosen coefficients, the candidate's index, its metrics
    (||r_p||, max residual, smoothness cost, path length) after refinement, whether it is
    feasible (max residual <= tol), and the indices that were refined.
    cache: a HandleCache to take the two stages' handles from (and leave them in)."""
    def handle(insts, **kw):
        if cache is not None:
            return cache.get(insts, nd, n_xi, rho=rho, precision=precision, proj=proj, dt=dt, stream=stream, **kw)
        return SFSolver(insts, nd, n_xi, rho=rho, precision=precision, proj=proj, dt=dt, stream=stream, **kw)

    nd = int(problems[0]["n_d"])
    dev = torch.device("cuda")
    sizes = [len(c) for c in candidates]
    flat = [dict(p, xi=np.asarray(x, dtype=np.float64)) for p, cs in zip(problems, candidates) for x in cs]
    # stage 1: every candidate's max residual, keep the `keep` least violating per problem
    s1 = handle(flat, max_iters=1)
    d1 = s1.pack(flat, device=dev)
    m1 = s1.metrics(d1, d1["xi"], stream=stream)
    kept = select(sizes, m1[:, 1].contiguous(), None, float("-inf"), keep, stream=stream).cpu().numpy()
    if cache is None:
        s1.close()
    chosen = [[j for j in kept[g] if j >= 0] for g in range(len(problems))]
    # stage 2: the SF on the kept candidates of every problem in one batch
    batch = [dict(problems[g], xi=np.asarray(candidates[g][j], dtype=np.float64))
             for g in range(len(problems)) for j in chosen[g]]
    s2 = handle(batch, max_iters=max(iters, 1), tol=tol)
    d2 = s2.pack(batch, device=dev)
    if autotune:   # costs several solves; the automatic geometry covers the SMs already
        s2.autotune(d2, d2["xi"], max(iters, 1), reps=1, stream=stream)
    xo, _, _ = s2.solve(d2, d2["xi"], iters, want_resid=False, stream=stream)
    # stage 3: feasible first by smoothness cost, else least residual
    m2 = s2.metrics(d2, xo, stream=stream)
    best = select([len(c) for c in chosen], m2[:, 1].contiguous(), m2[:, 2].contiguous(), tol, 1,
                  stream=stream).cpu().numpy()[:, 0]
    m2h = m2.cpu().numpy()
    xh = xo.double().cpu()   # one copy to the host, sliced per problem below
    out, base = [], 0
    for g in range(len(problems)):
        b = int(best[g])
        out.append(dict(xi=s2.unpack(xh, base + b).numpy(), index=int(chosen[g][b]),
                        metrics=m2h[base + b], feasible=bool(m2h[base + b, 1] <= tol), refined=list(chosen[g])))
        base += len(chosen[g])
    if cache is None:
        s2.close()
    return out
