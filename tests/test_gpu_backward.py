"""Hand-written adjoint (sf_solve_backward) against the oracle's reverse pass.

Instances are chosen clear of the kinks (every row's d-clamp and every box test
farther than 1e-3 from switching in every iteration), where the unrolled map is
differentiable; seeds are random on xi_bar^L, lambda^L and ||r_p(xi_bar^L)||^2.
"""
import numpy as np
import pytest
import torch

import oracle
import pinlib
import sfgen
from gpu_util import pack_list, rel
from paper_2510_09204_b300 import SFSolver, SFSolve

pytestmark = pytest.mark.gpu
RHO = 0.3


def kink_free(make, iters, tries=200):
    for s in range(tries):
        inst = make(s)
        h = oracle.solve(inst, iters, rho=RHO, hist=True)["hist"]
        fin = oracle.residual(inst, oracle.solve(inst, iters, rho=RHO)["xi"])
        if h[:, 3].min() > 1e-3 and fin[2] > 1e-3 and h[0, 1] > 0.05:
            return inst
    raise RuntimeError("no kink-free instance")


def gpu_grad(insts, iters, gxo, glo, grp2, precision="fp64", proj="dense", ckpt=3, cluster=None, threads=0,
             xi0=None, lam0=None):
    s = SFSolver(insts, insts[0]["n_d"], insts[0]["n_xi"], rho=RHO, precision=precision, proj=proj,
                 max_iters=iters, ckpt_every=ckpt)
    if cluster is not None:
        s.set_launch(cluster, threads)
    data = s.pack(insts)
    x0 = pack_list(s, xi0) if xi0 is not None else None
    l0 = pack_list(s, lam0) if lam0 is not None else None
    s.solve(data, data["xi"], iters, xi0=x0, lam0=l0)
    g_rp2 = torch.as_tensor(np.asarray(grp2, dtype=np.float64), device="cuda")
    gx, gx0, gl0 = s.backward(pack_list(s, gxo), pack_list(s, glo), g_rp2)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    un = lambda t: [s.unpack(t, k).double().cpu().numpy() for k in range(len(insts))]
    return un(gx), un(gx0), un(gl0)


def seeds(insts, seed=0):
    rng = np.random.default_rng(seed)
    gxo = [rng.normal(size=i["xi"].shape) for i in insts]
    glo = [rng.normal(size=i["xi"].shape) for i in insts]
    grp2 = rng.uniform(0.5, 1.5, size=len(insts))
    return gxo, glo, grp2


def oracle_grads(inst, iters, gxo, glo, grp2, xi0=None, lam0=None):
    return oracle.solve_backward(inst, iters, gxo, glo, grp2, rho=RHO, xi0=xi0, lam0=lam0)


def close(got, ref, tol):
    return np.linalg.norm(got - ref) <= tol * max(np.linalg.norm(ref), 1e-12)


@pytest.mark.parametrize("nd,aniso", [(2, False), (3, False), (3, True)])
def test_fp64_adjoint_matches_oracle_reverse_pass(nd, aniso):
    iters = 12
    insts = [kink_free(lambda s: pinlib.small_instance(n=4, n_obs=3, H=14, n_d=nd, n_xi=7, seed=50 * nd + s,
                                                       aniso=aniso), iters)]
    gxo, glo, grp2 = seeds(insts)
    gx, gx0, gl0 = gpu_grad(insts, iters, gxo, glo, grp2)
    r = oracle_grads(insts[0], iters, gxo[0], glo[0], grp2[0])
    # xi0 = NULL: the candidate's gradient includes the path through xi_bar^0
    for got, ref in zip((gx[0], gx0[0], gl0[0]), r):
        assert close(got, ref, 1e-9), rel(got, ref)


def test_fp64_adjoint_with_warm_start_and_boundary_gap():
    iters = 10
    inst = kink_free(lambda s: pinlib.small_instance(n=3, n_obs=2, H=12, n_d=2, n_xi=6, seed=300 + s), iters)
    rng = np.random.default_rng(7)
    xi0 = inst["xi"] + rng.normal(0, 0.02, size=inst["xi"].shape)   # misses A xi = b
    lam0 = rng.normal(0, 0.05, size=inst["xi"].shape)
    gxo, glo, grp2 = seeds([inst], 3)
    gx, gx0, gl0 = gpu_grad([inst], iters, gxo, glo, grp2, xi0=[xi0], lam0=[lam0])
    r = oracle_grads(inst, iters, gxo[0], glo[0], grp2[0], xi0=xi0, lam0=lam0)
    for got, ref in zip((gx[0], gx0[0], gl0[0]), r):
        assert close(got, ref, 1e-9), rel(got, ref)


@pytest.mark.parametrize("ckpt,cluster,proj", [(1, 1, "dense"), (4, 3, "dense"), (25, 2, "structured"),
                                               (7, 4, "structured")])
def test_adjoint_does_not_depend_on_checkpoints_geometry_or_projection_form(ckpt, cluster, proj):
    iters = 20
    insts = sfgen.make_batch(2, B=2)
    gxo, glo, grp2 = seeds(insts, 1)
    ref = gpu_grad(insts, iters, gxo, glo, grp2, ckpt=10, cluster=1, threads=256)
    got = gpu_grad(insts, iters, gxo, glo, grp2, ckpt=ckpt, cluster=cluster, threads=128, proj=proj)
    for a, b in zip(got, ref):
        for k in range(2):
            assert close(a[k], b[k], 1e-10), rel(a[k], b[k])


def test_fp64_adjoint_dynamic_obstacles():
    iters = 8
    inst = kink_free(lambda s: sfgen.custom_instance(n=4, n_obs=3, H=16, seed=600 + s, extent=5.0, dyn_obs=True,
                                                     n_xi=7), iters)
    gxo, glo, grp2 = seeds([inst], 5)
    gx, gx0, gl0 = gpu_grad([inst], iters, gxo, glo, grp2)
    r = oracle_grads(inst, iters, gxo[0], glo[0], grp2[0])
    for got, ref in zip((gx[0], gx0[0], gl0[0]), r):
        assert close(got, ref, 1e-9), rel(got, ref)


def test_fp32_adjoint_within_tolerance():
    iters = 12
    inst = kink_free(lambda s: pinlib.small_instance(n=4, n_obs=3, H=14, n_d=2, n_xi=7, seed=900 + s), iters)
    gxo, glo, grp2 = seeds([inst], 9)
    gx, gx0, gl0 = gpu_grad([inst], iters, gxo, glo, grp2, precision="fp32")
    r = oracle_grads(inst, iters, gxo[0], glo[0], grp2[0])
    for got, ref in zip((gx[0], gx0[0], gl0[0]), r):
        assert close(got, ref, 1e-4), rel(got, ref)


@pytest.mark.parametrize("proj", ["dense", "structured"])
@pytest.mark.parametrize("cluster", [4, 3])
def test_fp32_specialised_kernels_forward_and_adjoint(proj, cluster):
    """The compile-time kernels of the default configuration (FP32, n_xi = 11, culling) on
    a 100-step horizon: split over 4 CTAs every chunk has 25 timesteps (the unrolled W'
    aggregation), over 3 it has 33 or 34 (the runtime-length loop).  Forward iterate and
    adjoint against the oracle."""
    iters = 12
    inst = kink_free(lambda s: pinlib.small_instance(n=4, n_obs=3, H=100, n_d=2, n_xi=11, seed=1200 + s,
                                                     extent=5.0), iters)
    gxo, glo, grp2 = seeds([inst], 11)
    s = SFSolver([inst], 2, 11, rho=RHO, precision="fp32", proj=proj, max_iters=iters, ckpt_every=1)
    s.set_launch(cluster, 0)
    assert s.launch()[0] == cluster
    data = s.pack([inst])
    xo, lo, _ = s.solve(data, data["xi"], iters)
    g_rp2 = torch.as_tensor(np.asarray(grp2, dtype=np.float64), device="cuda")
    gx, gx0, gl0 = s.backward(pack_list(s, gxo), pack_list(s, glo), g_rp2)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    ref = oracle.solve(inst, iters, rho=RHO)
    W = oracle.basis(100, 11)
    got_x = s.unpack(xo, 0).double().cpu().numpy()
    assert np.abs(np.einsum("kc,dic->dik", W, got_x - ref["xi"])).max() <= 1e-4
    r = oracle_grads(inst, iters, gxo[0], glo[0], grp2[0])
    for got, want in zip((gx, gx0, gl0), r):
        g = s.unpack(got, 0).double().cpu().numpy()
        assert close(g, want, 1e-4), rel(g, want)
    s.close()


def test_autograd_function_loss_of_config4_form():
    """loss = sum ||r_p(out)||^2 + 0.1 ||out - candidate||^2 through SFSolve, against the
    oracle's reverse pass with the matching seeds."""
    iters = 10
    inst = kink_free(lambda s: pinlib.small_instance(n=3, n_obs=2, H=12, n_d=2, n_xi=6, seed=700 + s), iters)
    s = SFSolver([inst], 2, inst["n_xi"], rho=RHO, precision="fp64", max_iters=iters, ckpt_every=4)
    data = s.pack([inst])
    xc = data["xi"].clone().requires_grad_(True)
    x0 = xc.detach().clone().requires_grad_(True)
    l0 = torch.zeros_like(xc, requires_grad=True)
    xo, lo, rp2, _ = SFSolve.apply(xc, x0, l0, s, data, iters)
    loss = rp2.sum() + 0.1 * ((xo - xc) ** 2).sum()
    loss.backward()
    out = s.unpack(xo.detach(), 0).cpu().numpy()
    gx, gx0, gl0 = oracle.solve_backward(inst, iters, 0.2 * (out - inst["xi"]), None, 1.0, rho=RHO,
                                         xi0=inst["xi"], lam0=np.zeros_like(inst["xi"]))
    ref_xc = gx - 0.2 * (out - inst["xi"])
    assert close(s.unpack(xc.grad, 0).cpu().numpy(), ref_xc, 1e-9)
    assert close(s.unpack(x0.grad, 0).cpu().numpy(), gx0, 1e-9)
    assert close(s.unpack(l0.grad, 0).cpu().numpy(), gl0, 1e-9)


@pytest.mark.parametrize("ckpt,proj,nd", [(1, "dense", 2), (4, "structured", 2), (3, "dense", 3)])
def test_self_supervised_loss_matches_oracle(ckpt, proj, nd):
    """The loss of eq. NN_loss, sum_l ||z^{l+1} - z^l||^2 + ||xi_bar^L - xi||^2, through
    SFSolve (its fp_sum output) against the oracle's reverse pass with g_fp = 1, FP64; with
    checkpoints every iteration and with recomputed segments."""
    iters = 10
    inst = kink_free(lambda s: pinlib.small_instance(n=3, n_obs=2, H=12, n_d=nd, n_xi=6, seed=800 + s), iters)
    rng = np.random.default_rng(ckpt)
    xi0 = inst["xi"] + rng.normal(0, 0.05, size=inst["xi"].shape)
    lam0 = rng.normal(0, 0.1, size=inst["xi"].shape)
    s = SFSolver([inst], nd, inst["n_xi"], rho=RHO, precision="fp64", proj=proj, max_iters=iters, ckpt_every=ckpt)
    data = s.pack([inst])
    xc = data["xi"].clone().requires_grad_(True)
    x0 = pack_list(s, [xi0]).requires_grad_(True)
    l0 = pack_list(s, [lam0]).requires_grad_(True)
    xo, lo, rp2, fps = SFSolve.apply(xc, x0, l0, s, data, iters)
    loss = fps.sum() + ((xo - xc) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    tr = oracle.solve(inst, iters, rho=RHO, xi0=xi0, lam0=lam0, traj=True)["traj"]
    assert abs(float(fps[0]) - np.sum(np.diff(tr, axis=0) ** 2)) <= 1e-10 * np.sum(np.diff(tr, axis=0) ** 2)
    xL = tr[-1, 0]
    gx, gx0, gl0 = oracle.solve_backward(inst, iters, 2 * (xL - inst["xi"]), None, 0.0, rho=RHO, xi0=xi0,
                                         lam0=lam0, g_fp=1.0)
    assert close(s.unpack(xc.grad, 0).cpu().numpy(), gx - 2 * (xL - inst["xi"]), 1e-9)
    assert close(s.unpack(x0.grad, 0).cpu().numpy(), gx0, 1e-9)
    assert close(s.unpack(l0.grad, 0).cpu().numpy(), gl0, 1e-9)


def test_self_supervised_loss_fp32_batch_against_fp64():
    """The fixed-point seed on a 32-robot batch in FP32 against the same seed in FP64 (the
    FP64 path is pinned to the oracle above): per instance within 1e-3 relative."""
    insts = sfgen.make_batch(4, B=8)
    iters = 20
    out = {}
    for prec in ("fp64", "fp32"):
        s = SFSolver(insts, 2, 11, rho=RHO, precision=prec, proj="structured", max_iters=iters, ckpt_every=5)
        d = s.pack(insts)
        xo, _, res = s.solve(d, d["xi"], iters)
        ones = torch.ones(len(insts), dtype=torch.float64, device="cuda")
        gx, gx0, gl0 = s.backward(torch.zeros_like(xo), None, None, g_fp=ones)
        torch.cuda.synchronize()
        assert (s.status() == 0).all()
        out[prec] = [[s.unpack(t, k).double().cpu().numpy() for k in range(len(insts))] for t in (gx, gx0, gl0)]
        s.close()
    for a, b in zip(out["fp32"], out["fp64"]):
        for k in range(len(insts)):
            assert rel(a[k], b[k]) <= 1e-3, (k, rel(a[k], b[k]))


def test_backward_requires_checkpoints():
    from paper_2510_09204_b300 import SFError
    insts = sfgen.make_batch(1)
    s = SFSolver(insts, 2, 11, rho=RHO, precision="fp64", max_iters=5, ckpt_every=0)
    data = s.pack(insts)
    s.solve(data, data["xi"], 5)
    with pytest.raises(SFError):
        s.backward(torch.zeros_like(data["xi"]))
