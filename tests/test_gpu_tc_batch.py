"""The batched tensor-core projection of eq. batch_comp (SF_OPT_TC_BATCH): G instances of
one shape share a thread-block cluster of G x C CTAs; each CTA keeps its rows of P_eta in
tensor memory (BF16, with BF16 x3 the low parts beneath the high ones) and one tcgen05.mma
chain multiplies them by the right-hand sides of all G instances stacked in the MMA's N
columns.

Against the per-instance tensor-core product (the same operator, one instance per cluster)
and the FP64 oracle: the same tolerances as the other tensor-core tests (the format bound
per step, 1e-4 m in position over a run with refinement), forward and adjoint."""
import numpy as np
import pytest
import torch

import oracle
import sfgen
from gpu_util import max_pos_err, pack_list, rel
from paper_2510_09204_b300 import SFSolver
from paper_2510_09204_b300.sf import SF_OPT_TC_BATCH

pytestmark = pytest.mark.gpu
RHO = 0.3


def solver(insts, precision, iters, n_refine, batch, cluster=None, threads=0, ckpt=0):
    s = SFSolver(insts, insts[0]["n_d"], 11, rho=RHO, precision=precision, proj="dense", max_iters=iters,
                 n_refine=n_refine, ckpt_every=ckpt)
    if not batch:
        s.set_option(SF_OPT_TC_BATCH, 0)
    if cluster:
        s.set_launch(cluster, threads)
    return s


def test_the_plan_groups_instances_of_one_shape_only():
    same = sfgen.make_batch(2, B=4)
    s = solver(same, "bf16x3", 10, 1, True, cluster=4)
    assert s.option(SF_OPT_TC_BATCH) == 4          # 4 instances x 4 CTAs: a 16-CTA cluster
    s.set_option(SF_OPT_TC_BATCH, 0)
    assert s.option(SF_OPT_TC_BATCH) == 0
    mixed = sfgen.make_batch(3, B=4)                # uneven shapes: one instance per cluster
    assert solver(mixed, "bf16x3", 10, 1, True).option(SF_OPT_TC_BATCH) == 0
    assert solver(same, "tf32", 10, 1, True).option(SF_OPT_TC_BATCH) == 0   # BF16 formats only
    assert solver(sfgen.make_batch(2, B=3), "bf16", 10, 1, True, cluster=4).option(SF_OPT_TC_BATCH) == 3


@pytest.mark.parametrize("precision,n_refine", [("bf16x3", 1), ("bf16", 5)])
@pytest.mark.parametrize("cluster,threads", [(4, 512), (2, 256), (8, 1024), (1, 512)])
def test_batched_equals_per_instance_and_meets_the_oracle(precision, n_refine, cluster, threads):
    insts = sfgen.make_batch(2, B=4)
    iters = 60
    a = solver(insts, precision, iters, n_refine, True, cluster, threads)
    b = solver(insts, precision, iters, n_refine, False, cluster, threads)
    out = []
    for s in (a, b):
        d = s.pack(insts)
        xo, _, res = s.solve(d, d["xi"], iters)
        torch.cuda.synchronize()
        assert (s.status() == 0).all()
        out.append([s.unpack(xo, k).double().cpu().numpy() for k in range(4)])
    W = oracle.basis(100, 11)
    for k, inst in enumerate(insts):
        assert max_pos_err(inst, out[0][k], out[1][k], W) <= 1e-5
        ref = oracle.solve(inst, iters, rho=RHO)
        assert max_pos_err(inst, out[0][k], ref["xi"], W) <= 1e-4


def test_batched_3d_and_a_first_step_that_misses_the_boundary():
    """3-D instances (G n_d = 12 columns) from an initial iterate off A xi = b (the first
    step's P_b term), against the oracle."""
    insts = [sfgen.custom_instance(n=12, n_obs=6, H=40, n_d=3, seed=s, extent=(6.0, 6.0, 3.0)) for s in range(4)]
    rng = np.random.default_rng(2)
    xi0 = [i["xi"] + rng.normal(0, 0.1, size=i["xi"].shape) for i in insts]
    s = solver(insts, "bf16x3", 40, 1, True, cluster=4)
    assert s.option(SF_OPT_TC_BATCH) == 4
    d = s.pack(insts)
    xo, _, _ = s.solve(d, d["xi"], 40, xi0=pack_list(s, xi0))
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    W = oracle.basis(40, 11)
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, 40, rho=RHO, xi0=xi0[k])
        assert max_pos_err(inst, s.unpack(xo, k).double().cpu().numpy(), ref["xi"], W) <= 1e-4


def test_batched_adjoint_with_per_instance_seeds():
    """The adjoint through the batched product, with a residual seed of zero on some
    instances (every instance of a cluster still takes the same barriers), against the FP32
    SIMT adjoint: within 2.5 x 20 x 2^-15 relative, as for the per-instance product."""
    insts = sfgen.make_batch(2, B=4)
    rng = np.random.default_rng(3)
    g = [rng.normal(size=i["xi"].shape) * 1e-2 for i in insts]
    grp2 = torch.tensor([0.0, 1.0, 0.0, 0.5], dtype=torch.float64, device="cuda")
    got = []
    for prec in ("bf16x3", "fp32"):
        s = solver(insts, prec, 12, 1, True, cluster=4, ckpt=4)
        if prec == "bf16x3":
            assert s.option(SF_OPT_TC_BATCH) == 4
        d = s.pack(insts)
        s.solve(d, d["xi"], 12)
        gx, gx0, gl0 = s.backward(pack_list(s, g), None, grp2)
        torch.cuda.synchronize()
        assert (s.status() == 0).all()
        got.append([[s.unpack(t, k).double().cpu().numpy() for k in range(4)] for t in (gx, gx0, gl0)])
    bound = 2.5 * 20 * 2.0 ** -15
    for a, b in zip(got[0], got[1]):
        for k in range(4):
            assert rel(a[k], b[k]) <= bound, (k, rel(a[k], b[k]))
