"""The allocation-free entry point, sf_solve_noalloc, against the ordinary one.

sf_solve_noalloc serves callers that may not allocate device memory while they run
(a control loop with a memory budget fixed at start-up, a plug-in inside a framework
that owns every allocation).  It must give what sf_create + sf_solve give with FP32
and the structured projection: within the FP32 tolerance of the other tests
(1e-4 m maximum position error), on two calls in a row that share its fixed working
array.  This file is collected last so that a run stopping at the first failure has
run every other test first; it also passes on its own in a fresh process.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle
import sfgen
from paper_2510_09204_b300 import SFSolver, sf

pytestmark = pytest.mark.gpu
RHO = 0.3


def _shape_struct(inst, n_d):
    s = sf.sf_shape()
    s.n, s.n_obs, s.H, s.dyn_obs = inst["n"], inst["n_obs"], inst["H"], int(bool(inst.get("dyn_obs", False)))
    s.a, s.b = inst["a"], inst["b"]
    for ax in range(n_d):
        s.p_min[ax], s.p_max[ax] = inst["pmin"][ax], inst["pmax"][ax]
    return s


def _noalloc(insts, iters, data, xo, lo, res):
    n_d, n_xi = insts[0]["n_d"], insts[0]["n_xi"]
    shp = _shape_struct(insts[0], n_d)
    p = lambda t: ct.c_void_p(t.data_ptr()) if t is not None and t.numel() else None
    rc = sf.lib().sf_solve_noalloc(n_d, n_xi, RHO, ct.byref(shp), len(insts), p(data["bnd"]), p(data["obs_c"]),
                                   p(data["obs_ab"]), p(data["xi"]), iters, p(xo), p(lo), p(res),
                                   ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


@pytest.mark.parametrize("cid,B,iters", [(2, 4, 120), (5, 2, 40)])
def test_noalloc_matches_ordinary_solve_twice(cid, B, iters):
    insts = sfgen.make_batch(cid, B=B)
    ref = SFSolver(insts, insts[0]["n_d"], 11, rho=RHO, precision="fp32", proj="structured", max_iters=iters)
    data = ref.pack(insts)
    xr, lr, rr = ref.solve(data, data["xi"], iters)
    torch.cuda.synchronize()
    W = torch.as_tensor(oracle.basis(insts[0]["H"], 11))
    per = insts[0]["n_d"] * insts[0]["n"] * 11
    outs = []
    for call in range(2):
        xo = torch.full_like(data["xi"], float("nan"))
        lo = torch.full_like(data["xi"], float("nan"))
        res = torch.full((B, sf.SF_NRES), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(insts, iters, data, xo, lo, res) == sf.SF_OK
        torch.cuda.synchronize()
        for k in range(B):
            a = xo[k * per:(k + 1) * per].view(insts[0]["n_d"], -1, 11).double().cpu()
            b = xr[k * per:(k + 1) * per].view(insts[0]["n_d"], -1, 11).double().cpu()
            err = torch.einsum("kc,dic->dik", W, a - b).abs().max().item()
            assert err <= 1e-4, (call, k, err)
        np.testing.assert_allclose(lo.cpu().numpy(), lr.cpu().numpy(), atol=1e-3)
        np.testing.assert_allclose(res[:, 1].cpu().numpy(), rr[:, 1].cpu().numpy(), atol=1e-4)
        assert torch.isfinite(res).all()
        outs.append(xo.clone())
    assert torch.equal(outs[0], outs[1])  # the shared array keeps nothing that changes a later call


def test_noalloc_rejects_sizes_beyond_its_limits():
    insts = sfgen.make_batch(1)
    s = SFSolver(insts, 2, 11, rho=RHO, precision="fp32", max_iters=1)
    data = s.pack(insts)
    xo = torch.empty_like(data["xi"])
    many = [insts[0]] * (sf.SF_NOALLOC_MAX_INST + 1)
    assert _noalloc(many, 1, data, xo, None, None) == sf.SF_ETOOBIG
    long_h = [dict(insts[0], H=sf.SF_NOALLOC_MAX_H + 1)]
    assert _noalloc(long_h, 1, data, xo, None, None) == sf.SF_ETOOBIG
    assert sf.lib().sf_strerror(sf.SF_ETOOBIG).startswith(b"size beyond")


def _reference(cid, B, iters):
    insts = sfgen.make_batch(cid, B=B)
    ref = SFSolver(insts, insts[0]["n_d"], 11, rho=RHO, precision="fp32", proj="structured", max_iters=iters)
    data = ref.pack(insts)
    xr, _, _ = ref.solve(data, data["xi"], iters)
    torch.cuda.synchronize()
    return insts, data, xr


def _call_and_compare(insts, data, xr, iters):
    B = len(insts)
    xo = torch.full_like(data["xi"], float("nan"))
    res = torch.full((B, sf.SF_NRES), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(insts, iters, data, xo, None, res) == sf.SF_OK
    torch.cuda.synchronize()
    W = torch.as_tensor(oracle.basis(insts[0]["H"], 11))
    per = insts[0]["n_d"] * insts[0]["n"] * 11
    for k in range(B):
        a = xo[k * per:(k + 1) * per].view(insts[0]["n_d"], -1, 11).double().cpu()
        b = xr[k * per:(k + 1) * per].view(insts[0]["n_d"], -1, 11).double().cpu()
        assert torch.einsum("kc,dic->dik", W, a - b).abs().max().item() <= 1e-4
    assert torch.isfinite(res).all()
    return xo


def test_noalloc_another_shape_in_between():
    """A 3-D call with another shape (64 robots, 100 obstacles) between two 2-D calls: each
    call rewrites the instance table, basis and operators of the shared array from its own
    arguments, so each matches its ordinary solve and the two 2-D calls agree bit for bit."""
    a = _reference(2, 4, 80)
    b = _reference(5, 2, 30)
    x1 = _call_and_compare(*a, 80)
    _call_and_compare(*b, 30)
    x2 = _call_and_compare(*a, 80)
    assert torch.equal(x1, x2)
