"""Candidate metrics (sf_metrics), ranking (sf_select) and the three-stage pipeline
against the oracle: metrics to 1e-10 in FP64, selections identical, and the pipeline's
choice equal to the same pipeline driven by the oracle."""
import numpy as np
import pytest
import torch

import oracle
import pinlib
import sfgen
from gpu_util import rel
from paper_2510_09204_b300 import SFSolver
from paper_2510_09204_b300.pipeline import refine_candidates
from paper_2510_09204_b300.sf import select

pytestmark = pytest.mark.gpu
RHO, DT = 0.3, 0.05


def rounded32(inst):
    p = dict(inst)
    for key in ("xi", "bnd", "obs_c", "obs_ab", "pmin", "pmax"):
        p[key] = np.asarray(inst[key], dtype=np.float32).astype(np.float64)
    for key in ("a", "b"):
        p[key] = float(np.float32(inst[key]))
    return p


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_metrics_match_oracle(precision):
    insts = sfgen.make_batch(2, B=3) + [sfgen.custom_instance(n=7, n_obs=0, H=33, seed=4, extent=6.0)]
    s = SFSolver(insts, 2, 11, rho=RHO, precision=precision, proj="structured", max_iters=1, dt=DT)
    d = s.pack(insts)
    m = s.metrics(d, d["xi"]).cpu().numpy()
    for k, inst in enumerate(insts):
        ref_inst = rounded32(inst) if precision == "fp32" else inst
        ref = oracle.metrics(ref_inst, ref_inst["xi"], rho=RHO, dt=DT)
        np.testing.assert_allclose(m[k], ref, rtol=1e-10, atol=1e-12)


def test_select_matches_oracle():
    rng = np.random.default_rng(3)
    sizes = [0, 1, 5, 300, 4096, 17]
    prim = np.concatenate([rng.exponential(1e-3, size=m) for m in sizes])
    prim[rng.choice(prim.size, 20, replace=False)] = np.nan
    prim[10:14] = prim[10]              # ties
    sec = rng.normal(size=prim.size)
    for q, thr, k in [(None, -np.inf, 7), (sec, 1e-3, 12), (sec, 5e-4, 1)]:
        got = select(sizes, torch.as_tensor(prim, device="cuda"),
                     None if q is None else torch.as_tensor(q, device="cuda"), thr, k).cpu().numpy()
        o = 0
        for g, m in enumerate(sizes):
            ref = oracle.select(prim[o:o + m], None if q is None else q[o:o + m], thr, k)
            assert list(got[g]) == ref, (g, m)
            o += m


def test_pipeline_matches_oracle_driven_pipeline():
    """Three problems, 12 candidates each (the problem's candidate plus noise), keep 4,
    60 FP64 iterations: the same kept set and the same final choice as the pipeline run
    with the oracle's metrics, ranking and solver."""
    rng = np.random.default_rng(11)
    problems = [sfgen.custom_instance(n=5, n_obs=4, H=40, seed=60 + g, extent=5.0) for g in range(3)]
    cands = []
    for p in problems:
        cs = []
        for _ in range(12):
            x = p["xi"].copy()
            x[..., 1:-1] += rng.normal(0, 0.4, size=x[..., 1:-1].shape)
            cs.append(x)
        cands.append(np.stack(cs))
    keep, iters, tol = 4, 60, 1e-3
    got = refine_candidates(problems, cands, keep=keep, iters=iters, precision="fp64", tol=tol, rho=RHO, dt=DT)
    for g, p in enumerate(problems):
        m1 = [oracle.metrics(dict(p, xi=x), x, rho=RHO, dt=DT) for x in cands[g]]
        kept = oracle.select([m[1] for m in m1], None, -np.inf, keep)
        assert got[g]["refined"] == kept
        outs = [oracle.solve(dict(p, xi=cands[g][j]), iters, rho=RHO)["xi"] for j in kept]
        m2 = [oracle.metrics(p, x, rho=RHO, dt=DT) for x in outs]
        b = oracle.select([m[1] for m in m2], [m[2] for m in m2], tol, 1)[0]
        assert got[g]["index"] == kept[b]
        assert rel(got[g]["xi"], outs[b]) <= 1e-10
        np.testing.assert_allclose(got[g]["metrics"], m2[b], rtol=1e-9, atol=1e-12)


def test_pipeline_with_cached_handles_gives_the_same_choice():
    """Three calls through a HandleCache (new data, same shapes) against calls without it:
    the same kept sets, choices and bits; the cache keeps one handle per stage."""
    from paper_2510_09204_b300.pipeline import HandleCache
    rng = np.random.default_rng(21)
    problems = [sfgen.custom_instance(n=4, n_obs=3, H=30, seed=80 + g, extent=5.0) for g in range(2)]
    cache = HandleCache()
    for call in range(3):
        cands = [np.stack([p["xi"] + np.pad(rng.normal(0, 0.4, size=p["xi"][..., 1:-1].shape), ((0, 0), (0, 0), (1, 1)))
                           for _ in range(6)]) for p in problems]
        kw = dict(keep=3, iters=40, precision="fp32", rho=RHO, dt=DT)
        a = refine_candidates(problems, cands, **kw)
        b = refine_candidates(problems, cands, cache=cache, **kw)
        for x, y in zip(a, b):
            assert x["refined"] == y["refined"] and x["index"] == y["index"]
            np.testing.assert_array_equal(x["xi"], y["xi"])
        assert len(cache._h) == 2
    cache.close()
    assert len(cache._h) == 0
