"""Row culling (SF_OPT_CULL) is exact: the forward outputs and the adjoint's gradients
with culling on and off are the same bits, on batches whose chunks see few candidates
(sparse maps), many (a crowded map where every box overlaps) and the special cases
(coincident robots, 3D anisotropic bodies, moving obstacles, uneven shapes)."""
import numpy as np
import pytest
import torch

import sfgen
from paper_2510_09204_b300 import SFSolver
from paper_2510_09204_b300.sf import SF_OPT_CULL

pytestmark = pytest.mark.gpu
RHO = 0.3


def batches():
    sparse = sfgen.make_batch(2, B=4)
    crowded = [sfgen.custom_instance(n=12, n_obs=12, H=40, seed=s, extent=5.0, sigma=0.8) for s in range(3)]
    coincident = [sfgen.custom_instance(n=6, n_obs=3, H=30, seed=9, extent=6.0)]
    c = coincident[0]
    c["xi"] = c["xi"].copy()
    c["xi"][:, 1, 3:8] = c["xi"][:, 0, 3:8]   # robots 0 and 1 share interior coefficients
    aniso = [sfgen.custom_instance(n=9, n_obs=12, H=50, n_d=3, seed=s, extent=(6.0, 6.0, 2.0)) for s in range(2)]
    for i in aniso:
        i["b"] = 0.7 * i["a"]
    dyn = [sfgen.custom_instance(n=10, n_obs=8, H=60, seed=20 + s, extent=7.0, dyn_obs=True) for s in range(2)]
    uneven = [sfgen.custom_instance(n=n, n_obs=o, H=H, seed=30 + k, extent=9.0)
              for k, (n, o, H) in enumerate([(5, 0, 33), (17, 21, 64), (8, 40, 50)])]
    return {"sparse": sparse, "crowded": crowded, "coincident": coincident, "aniso3d": aniso, "dyn": dyn,
            "uneven": uneven}


def run(insts, precision, cull, iters=40, proj="dense", cost="projection"):
    s = SFSolver(insts, insts[0]["n_d"], 11, rho=RHO, precision=precision, proj=proj, max_iters=iters,
                 ckpt_every=10, cost=cost, dt=0.05)
    s.set_option(SF_OPT_CULL, cull)
    assert s.option(SF_OPT_CULL) == cull
    data = s.pack(insts)
    xo, lo, res = s.solve(data, data["xi"], iters)
    g = torch.as_tensor(np.random.default_rng(1).normal(size=xo.numel()), dtype=xo.dtype, device=xo.device)
    grp2 = torch.full((len(insts),), 0.7, dtype=torch.float64, device=xo.device)
    gx, gx0, gl0 = s.backward(g, g * 0.5, grp2)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    return [t.cpu() for t in (xo, lo, res, gx, gx0, gl0)]


# FP32 with culling runs the compile-time kernels (dense projection, structured projection,
# and the structured projection with the smoothness cost); without culling, the generic
# kernel: the two must agree bit for bit
@pytest.mark.parametrize("proj,cost", [("dense", "projection"), ("structured", "projection"),
                                       ("structured", "smoothness")])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", ["sparse", "crowded", "coincident", "aniso3d", "dyn", "uneven"])
def test_culling_is_bit_exact(name, precision, proj, cost):
    insts = batches()[name]
    on = run(insts, precision, 1, proj=proj, cost=cost)
    off = run(insts, precision, 0, proj=proj, cost=cost)
    for a, b in zip(on, off):
        assert torch.equal(a, b)


def test_culled_run_is_active():
    """the crowded batch does have active rows (so the comparison above is not vacuous)"""
    insts = batches()["crowded"]
    res = run(insts, "fp64", 1, iters=1)[2].numpy()
    assert (res[:, 1] > 0.05).all()
