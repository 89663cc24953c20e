"""The largest sizes the launch plan supports, and a clean SF_EUNSUPPORTED beyond them.

Every CTA keeps its share of the horizon's basis rows, its iterate, multipliers and the
instance's obstacle records in shared memory (227 KB per CTA):
- H = 4096 timesteps: supported in FP32 and FP64 (8 CTAs of 512 timesteps);
- n_obs = 4096 obstacles: FP32 (the FP64 records do not fit: SF_EUNSUPPORTED);
- n = 256 robots: the 2-D FP32 forward (the adjoint's state does not fit beside it, so a
  handle that keeps checkpoints is SF_EUNSUPPORTED, as are FP64 and 3-D);
- n_xi = 4 (the fewest the basis allows) to 32 coefficients.
Where the oracle is affordable the results are compared with it; the 256-robot case uses
the feasible-fixed-point property (a conflict-free candidate is returned unchanged)."""
import numpy as np
import pytest
import torch

import oracle
import sfgen
from gpu_util import rel
from paper_2510_09204_b300 import SFSolver, SFError
from paper_2510_09204_b300.sf import SF_EUNSUPPORTED

pytestmark = pytest.mark.gpu
RHO = 0.3


def solve(insts, precision, proj, iters, ckpt=0, backward=False):
    s = SFSolver(insts, insts[0]["n_d"], insts[0]["n_xi"], rho=RHO, precision=precision, proj=proj,
                 max_iters=iters, ckpt_every=ckpt)
    d = s.pack(insts)
    xo, lo, res = s.solve(d, d["xi"], iters)
    g = None
    if backward:
        g = s.backward(torch.ones_like(xo) * 1e-2)[0]
    torch.cuda.synchronize()
    st = s.status()
    out = dict(xi=[s.unpack(xo, k).double().cpu().numpy() for k in range(len(insts))],
               lam=[s.unpack(lo, k).double().cpu().numpy() for k in range(len(insts))], status=st,
               g=None if g is None else g.double().cpu().numpy(), launch=s.launch())
    s.close()
    return out


def pos_err(inst, a, b):
    W = oracle.basis(inst["H"], inst["n_xi"])
    return np.abs(np.einsum("kc,dic->dik", W, a - b)).max()


@pytest.mark.parametrize("precision,proj", [("fp32", "structured"), ("fp64", "dense"), ("fp64", "structured")])
def test_longest_horizon(precision, proj):
    inst = sfgen.custom_instance(n=2, n_obs=2, H=4096, seed=3, extent=4.0, sigma=0.8)
    iters = 4
    out = solve([inst], precision, proj, iters, ckpt=1, backward=True)
    assert (out["status"] == 0).all()
    assert out["launch"][0] == 8
    assert np.isfinite(out["g"]).all()
    ref = oracle.solve(inst, iters, rho=RHO)
    if precision == "fp64":
        assert rel(out["xi"][0], ref["xi"]) <= 1e-10
    else:
        assert pos_err(inst, out["xi"][0], ref["xi"]) <= 1e-4


def test_most_obstacles():
    inst = sfgen.custom_instance(n=2, n_obs=4096, H=20, seed=5, extent=60.0)
    iters = 6
    out = solve([inst], "fp32", "structured", iters, ckpt=1, backward=True)
    assert (out["status"] == 0).all()
    assert np.isfinite(out["g"]).all()
    ref = oracle.solve(inst, iters, rho=RHO)
    assert pos_err(inst, out["xi"][0], ref["xi"]) <= 1e-4
    with pytest.raises(SFError) as e:
        SFSolver([inst], 2, inst["n_xi"], rho=RHO, precision="fp64", proj="structured", max_iters=iters)
    assert e.value.code == SF_EUNSUPPORTED


def conflict_free_grid(n_side=16, spacing=2.0, H=20, n_xi=11):
    """n_side^2 robots on a grid, each moving 1 m along x: never within a of another."""
    n = n_side * n_side
    xs, ys = np.meshgrid(np.arange(n_side) * spacing, np.arange(n_side) * spacing, indexing="ij")
    start = np.stack([xs.ravel(), ys.ravel()])            # [2][n]
    goal = start + np.array([[1.0], [0.0]])
    ramp = np.linspace(0.0, 1.0, n_xi)
    xi = start[:, :, None] * (1 - ramp) + goal[:, :, None] * ramp
    ext = n_side * spacing + 4.0
    return dict(n=n, n_obs=0, H=H, n_d=2, n_xi=n_xi, a=0.5, b=0.5, pmin=np.full(2, -2.0), pmax=np.full(2, ext),
                obs_c=np.zeros((0, 2)), obs_ab=np.zeros((0, 2)), bnd=np.stack([start, goal], axis=-1), xi=xi)


def test_most_robots_feasible_fixed_point():
    inst = conflict_free_grid()
    assert inst["n"] == 256
    out = solve([inst], "fp32", "structured", 5)
    assert (out["status"] == 0).all()
    np.testing.assert_array_equal(out["xi"][0], inst["xi"].astype(np.float32).astype(np.float64))
    assert np.abs(out["lam"][0]).max() == 0.0
    for precision, ckpt, nd in (("fp32", 1, 2), ("fp64", 0, 2)):
        with pytest.raises(SFError) as e:
            SFSolver([inst], nd, 11, rho=RHO, precision=precision, proj="structured", max_iters=5, ckpt_every=ckpt)
        assert e.value.code == SF_EUNSUPPORTED


@pytest.mark.parametrize("n_xi", [4, 32])
@pytest.mark.parametrize("precision,proj", [("fp32", "structured"), ("fp64", "dense")])
def test_fewest_and_most_coefficients(precision, proj, n_xi):
    inst = sfgen.custom_instance(n=4, n_obs=3, H=50, n_xi=n_xi, seed=7, extent=5.0)
    iters = 20
    out = solve([inst], precision, proj, iters, ckpt=1, backward=True)
    assert (out["status"] == 0).all()
    ref = oracle.solve(inst, iters, rho=RHO)
    if precision == "fp64":
        assert rel(out["xi"][0], ref["xi"]) <= 1e-9
    else:
        assert pos_err(inst, out["xi"][0], ref["xi"]) <= 1e-4
