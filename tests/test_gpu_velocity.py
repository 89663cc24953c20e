"""Initial-velocity boundary rows (n_bc = 3; Sec. V, the planner conditioned on the
robots' current velocities) on the GPU against the FP64 oracle, through the C ABI.

With the velocity row p'(0) = v_0 (time t = tau (H - 1) dt, dt = 0.1 s on both sides),
A fixes Bernstein coefficients 0, 1 and n_xi - 1.  The generated candidates do not meet
the velocity row, so the first step's P_b (b - A xi_bar^0) term is exercised in every
run.  Tolerances as elsewhere: FP64 1e-10 relative per iterate, operators 1e-12, FP32
1e-4 m in position and 1e-3 m in the final residual, FP64 adjoint 1e-9.
"""
import numpy as np
import pytest
import torch

import oracle
import pinlib
import sfgen
from gpu_util import gpu_solve, max_pos_err, pack_list, rel
from paper_2510_09204_b300 import SFSolver

pytestmark = pytest.mark.gpu
RHO, DT = 0.3, 0.1   # DT: the oracle's default time step


def vbatch(cid, B):
    return [sfgen.with_initial_velocity(i, k) for k, i in enumerate(sfgen.make_batch(cid, B=B))]


@pytest.mark.parametrize("proj", ["dense", "structured"])
def test_velocity_operators_match_oracle(proj):
    inst = vbatch(2, 1)[0]
    s = SFSolver([inst], 2, 11, rho=RHO, precision="fp64", proj=proj, max_iters=1, dt=DT)
    assert s.n_bc == 3
    _, Pe, Pb = oracle.kkt(2, 11, RHO, inst["n"], inst["n_obs"], inst["H"], dt=DT, n_bc=3)
    np.testing.assert_allclose(s.operator(0, 1), Pe, atol=1e-12 * np.abs(Pe).max())
    np.testing.assert_allclose(s.operator(0, 2), Pb, atol=1e-12 * np.abs(Pb).max())


@pytest.mark.parametrize("proj", ["dense", "structured"])
def test_velocity_fp64_every_iterate_matches_oracle(proj):
    inst = vbatch(1, 1)[0]
    tr = oracle.solve(inst, 20, rho=RHO, dt=DT, traj=True)["traj"]
    x, l = inst["xi"], np.zeros_like(inst["xi"])
    for it in range(20):
        out = gpu_solve([inst], 1, proj=proj, xi0=[x], lam0=[l])
        x, l = out["xi"][0], out["lam"][0]
        z = np.concatenate([x.ravel(), l.ravel()])
        zr = np.concatenate([tr[it + 1, 0].ravel(), tr[it + 1, 1].ravel()])
        assert rel(z, zr) <= 1e-10, (it, rel(z, zr))


@pytest.mark.parametrize("cid,B,iters,proj", [(1, 1, 100, "dense"), (2, 3, 200, "structured"), (2, 2, 120, "dense")])
def test_velocity_fp64_run_matches_oracle_and_holds_the_rows(cid, B, iters, proj):
    insts = vbatch(cid, B)
    out = gpu_solve(insts, iters, proj=proj)
    assert (out["status"] == 0).all()
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, iters, rho=RHO, dt=DT)
        z = np.concatenate([out["xi"][k].ravel(), out["lam"][k].ravel()])
        zr = np.concatenate([ref["xi"].ravel(), ref["lam"].ravel()])
        assert rel(z, zr) <= 1e-10, rel(z, zr)
        x = out["xi"][k]
        assert np.array_equal(x[..., 0], inst["bnd"][..., 0]) and np.array_equal(x[..., -1], inst["bnd"][..., 1])
        wd0 = pinlib.bernstein_d(inst["H"], 11, DT)[0]
        np.testing.assert_allclose(x @ wd0, inst["bnd"][..., 2], atol=1e-11)


def test_velocity_3d():
    inst = sfgen.with_initial_velocity(
        sfgen.custom_instance(n=6, n_obs=5, H=30, n_d=3, seed=4, extent=(6.0, 6.0, 3.0)), 5)
    ref = oracle.solve(inst, 50, rho=RHO, dt=DT)
    for proj in ("dense", "structured"):
        out = gpu_solve([inst], 50, proj=proj)
        z = np.concatenate([out["xi"][0].ravel(), out["lam"][0].ravel()])
        assert rel(z, np.concatenate([ref["xi"].ravel(), ref["lam"].ravel()])) <= 1e-10


@pytest.mark.parametrize("precision,proj,n_refine", [("fp32", "structured", 0), ("fp32", "dense", 0),
                                                     ("tf32", "dense", 2), ("bf16x3", "dense", 1)])
def test_velocity_reduced_precision(precision, proj, n_refine):
    insts = vbatch(2, 3)
    out = gpu_solve(insts, 200, precision=precision, proj=proj, n_refine=n_refine)
    assert (out["status"] == 0).all()
    W = oracle.basis(100, 11)
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, 200, rho=RHO, dt=DT)
        assert max_pos_err(inst, out["xi"][k], ref["xi"], W) <= 1e-4
        assert abs(out["resid"][k, 1] - oracle.residual(inst, ref["xi"], rho=RHO)[1]) <= 1e-3


def _kink_free_vel(iters, nd=2):
    for s in range(200):
        inst = sfgen.with_initial_velocity(
            pinlib.small_instance(n=3, n_obs=2, H=12, n_d=nd, n_xi=6, seed=900 + s), s)
        h = oracle.solve(inst, iters, rho=RHO, dt=DT, hist=True)["hist"]
        fin = oracle.residual(inst, oracle.solve(inst, iters, rho=RHO, dt=DT)["xi"])
        if h[:, 3].min() > 1e-3 and fin[2] > 1e-3 and h[0, 1] > 0.05:
            return inst
    raise RuntimeError("no kink-free instance")


@pytest.mark.parametrize("ckpt,proj,nd", [(1, "dense", 2), (4, "structured", 2), (3, "structured", 3)])
def test_velocity_adjoint_matches_oracle(ckpt, proj, nd):
    """The adjoint with the velocity rows, from an initial iterate that misses all three rows
    (so the gradient to xi_bar^0 runs through -A'P_b' at the first step), FP64."""
    iters = 10
    inst = _kink_free_vel(iters, nd)
    rng = np.random.default_rng(ckpt)
    xi0 = inst["xi"] + rng.normal(0, 0.05, size=inst["xi"].shape)
    lam0 = rng.normal(0, 0.1, size=inst["xi"].shape)
    gxo = rng.normal(size=inst["xi"].shape)
    glo = rng.normal(size=inst["xi"].shape)
    s = SFSolver([inst], nd, 6, rho=RHO, precision="fp64", proj=proj, max_iters=iters, ckpt_every=ckpt, dt=DT)
    data = s.pack([inst])
    s.solve(data, data["xi"], iters, xi0=pack_list(s, [xi0]), lam0=pack_list(s, [lam0]))
    g_rp2 = torch.full((1,), 0.6, dtype=torch.float64, device="cuda")
    gx, gx0, gl0 = s.backward(pack_list(s, [gxo]), pack_list(s, [glo]), g_rp2)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    ref = oracle.solve_backward(inst, iters, gxo, glo, 0.6, rho=RHO, xi0=xi0, lam0=lam0, dt=DT)
    for got, want in zip((gx, gx0, gl0), ref):
        g = s.unpack(got, 0).cpu().numpy()
        assert rel(g, want) <= 1e-9, rel(g, want)
