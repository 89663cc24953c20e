"""The trajectory optimiser (SF_COST_SMOOTHNESS: eq. eq::form with the smoothness cost
of eq. cost) on the GPU against the oracle: the cost block, every iterate in FP64
(dense and Kronecker projection, 2D and 3D), the adjoint, FP32 on a full batch and the
unconstrained straight-line optimum."""
import numpy as np
import pytest
import torch

import oracle
import pinlib
import sfgen
from gpu_util import max_pos_err, pack_list, rel
from paper_2510_09204_b300 import SFSolver

pytestmark = pytest.mark.gpu
RHO = 0.3
DT = 0.05


def solver(insts, precision, proj, iters, ckpt=0, cluster=None, threads=0):
    s = SFSolver(insts, insts[0]["n_d"], insts[0]["n_xi"], rho=RHO, precision=precision, proj=proj,
                 max_iters=max(iters, 1), ckpt_every=ckpt, cost="smoothness", dt=DT)
    if cluster is not None:
        s.set_launch(cluster, threads)
    return s


def test_cost_block_matches_oracle():
    inst = sfgen.make_batch(2, B=1)[0]
    s = solver([inst], "fp64", "structured", 1)
    blk = s.operator(0, 3)[2 * 121 + 44:].reshape(11, 11)
    Wdd = oracle.basis_dd(100, 11, DT)
    ref = Wdd.T @ Wdd
    np.testing.assert_allclose(blk, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("proj", ["dense", "structured"])
@pytest.mark.parametrize("nd", [2, 3])
def test_fp64_every_iterate_matches_oracle(proj, nd):
    insts = [sfgen.custom_instance(n=6, n_obs=5, H=40, n_d=nd, seed=11 + nd,
                                   extent=6.0 if nd == 2 else (6.0, 6.0, 3.0)) for _ in range(1)]
    insts.append(sfgen.custom_instance(n=4, n_obs=3, H=25, n_d=nd, seed=21 + nd,
                                       extent=5.0 if nd == 2 else (5.0, 5.0, 2.5)))
    for it in (1, 2, 7, 25):
        s = solver(insts, "fp64", proj, it, cluster=2, threads=128)
        d = s.pack(insts)
        xo, lo, _ = s.solve(d, d["xi"], it)
        torch.cuda.synchronize()
        for k, inst in enumerate(insts):
            ref = oracle.solve(inst, it, rho=RHO, cost="smoothness", dt=DT)
            z = np.concatenate([s.unpack(xo, k).cpu().numpy().ravel(), s.unpack(lo, k).cpu().numpy().ravel()])
            zr = np.concatenate([ref["xi"].ravel(), ref["lam"].ravel()])
            assert rel(z, zr) <= 1e-10, (it, k, rel(z, zr))


def test_fp64_adjoint_matches_oracle():
    iters = 8
    inst = pinlib.small_instance(n=4, n_obs=3, H=14, n_d=2, n_xi=7, seed=31)
    rng = np.random.default_rng(9)
    gxo = rng.normal(size=inst["xi"].shape)
    glo = rng.normal(size=inst["xi"].shape)
    s = solver([inst], "fp64", "dense", iters, ckpt=3)
    d = s.pack([inst])
    s.solve(d, d["xi"], iters)
    gx, gx0, gl0 = s.backward(pack_list(s, [gxo]), pack_list(s, [glo]),
                              torch.tensor([0.8], dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    rx, rx0, rl0 = oracle.solve_backward(inst, iters, gxo, glo, 0.8, rho=RHO, xi0=inst["xi"],
                                         lam0=np.zeros_like(inst["xi"]), cost="smoothness", dt=DT)
    # the handle's xi0 is NULL: the candidate is the initial iterate, so its gradient is g_xi0
    assert rel(s.unpack(gx, 0).cpu().numpy(), rx0) <= 1e-9
    assert rel(s.unpack(gx0, 0).cpu().numpy(), rx0) <= 1e-9
    assert rel(s.unpack(gl0, 0).cpu().numpy(), rl0) <= 1e-9
    assert np.abs(rx).max() == 0.0


def test_fp32_full_batch_within_tolerance():
    insts = sfgen.make_batch(2)
    iters = 200
    s = solver(insts, "fp32", "structured", iters)
    d = s.pack(insts)
    xo, _, res = s.solve(d, d["xi"], iters)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    W = oracle.basis(100, 11)
    for k in (0, 17):
        ref = oracle.solve(insts[k], iters, rho=RHO, cost="smoothness", dt=DT)
        assert max_pos_err(insts[k], s.unpack(xo, k).double().cpu().numpy(), ref["xi"], W) <= 1e-4
        assert abs(res.cpu().numpy()[k, 1] - oracle.residual(insts[k], ref["xi"], rho=RHO)[1]) <= 1e-3


def test_unconstrained_optimum_is_the_straight_line():
    inst = pinlib.small_instance(n=1, n_obs=0, H=30, n_d=2, n_xi=8, seed=5, sigma=0.4, extent=40.0)
    s = SFSolver([inst], 2, 8, rho=1.0, precision="fp64", proj="structured", max_iters=3000,
                 cost="smoothness", dt=0.02)
    d = s.pack([inst])
    xo, _, res = s.solve(d, d["xi"], 3000)
    torch.cuda.synchronize()
    b = inst["bnd"]
    ramp = b[..., :1] + (b[..., 1:] - b[..., :1]) * np.linspace(0.0, 1.0, 8)
    np.testing.assert_allclose(s.unpack(xo, 0).cpu().numpy(), ramp, atol=1e-8)
    assert res.cpu().numpy()[0, 1] == 0.0


@pytest.mark.parametrize("dyn", [False, True])
def test_fp32_3d_and_moving_obstacles_within_tolerance(dyn):
    """The compile-time kernel of the optimiser (FP32, n_xi = 11, culling, structured) in 3-D
    with an anisotropic body, and in 2-D with moving obstacles, against the oracle."""
    if dyn:
        insts = [sfgen.custom_instance(n=8, n_obs=6, H=60, seed=40 + k, extent=7.0, dyn_obs=True) for k in range(2)]
    else:
        insts = [sfgen.custom_instance(n=10, n_obs=8, H=60, n_d=3, seed=50 + k, extent=(7.0, 7.0, 3.0))
                 for k in range(2)]
        for i in insts:
            i["b"] = 0.7 * i["a"]
    iters = 120
    s = solver(insts, "fp32", "structured", iters)
    d = s.pack(insts)
    xo, _, res = s.solve(d, d["xi"], iters)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    W = oracle.basis(60, 11)
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, iters, rho=RHO, cost="smoothness", dt=DT)
        assert max_pos_err(inst, s.unpack(xo, k).double().cpu().numpy(), ref["xi"], W) <= 1e-4
        assert abs(res.cpu().numpy()[k, 1] - oracle.residual(inst, ref["xi"], rho=RHO)[1]) <= 1e-3
