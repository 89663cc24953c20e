"""The projection of eq. batch_comp on the tensor cores (tcgen05.mma, TMEM accumulator):
TF32, BF16, and BF16 x3 (hi*hi + hi*lo + lo*hi of a two-term BF16 split), all with FP32
accumulation, against the FP32 SIMT projection and the FP64 oracle.

One iteration from a fixed state isolates the projection: xi_bar^1 - xi_bar^0 is
P_eta v, so its relative error is bounded by the operand format's precision
(TF32 2^-11, BF16 2^-8, BF16 x3 about 2^-15) times the cancellation factor
kappa = || |P_eta| |v| || / || P_eta v || of the product, with a factor 3 for rounding
both operands and the accumulation."""
import numpy as np
import pytest

import oracle
import sfgen
from gpu_util import gpu_solve, max_pos_err, rel

pytestmark = pytest.mark.gpu
RHO = 0.3
UNIT = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "bf16x3": 2.0 ** -15}
BOUND = {k: 20 * v for k, v in UNIT.items()}   # loose bound for multi-iteration comparisons


def projection_bound(solver, k, inst, xi0, lam0, lam1, precision):
    """3 u kappa for instance k, with v = xi - xi_bar^0 + 2 lambda^1 - lambda^0 (correction form)."""
    P = solver.operator(k, 1)
    v = inst["xi"] - xi0 + 2 * lam1 - lam0
    num = den = 0.0
    for ax in range(inst["n_d"]):
        va = v[ax].ravel()
        num += np.sum((np.abs(P) @ np.abs(va)) ** 2)
        den += np.sum((P @ va) ** 2)
    return 3 * UNIT[precision] * np.sqrt(num / den)


@pytest.mark.parametrize("precision", ["tf32", "bf16", "bf16x3"])
@pytest.mark.parametrize("cluster,threads", [(1, 512), (2, 256), (4, 128), (8, 1024)])
def test_one_step_projection_error_is_within_the_format_bound(precision, cluster, threads):
    insts = sfgen.make_batch(2, B=2)
    rng = np.random.default_rng(4)
    xi0 = [i["xi"] + rng.normal(0, 0.1, size=i["xi"].shape) for i in insts]
    for x, i in zip(xi0, insts):
        x[:, :, 0] = i["bnd"][:, :, 0]
        x[:, :, -1] = i["bnd"][:, :, 1]
    lam0 = [rng.normal(0, 0.2, size=i["xi"].shape) for i in insts]
    ref = gpu_solve(insts, 1, precision="fp32", proj="dense", xi0=xi0, lam0=lam0)
    got = gpu_solve(insts, 1, precision=precision, proj="dense", xi0=xi0, lam0=lam0, cluster=cluster, threads=threads)
    assert (got["status"] == 0).all()
    for k in range(2):
        d_ref = ref["xi"][k] - xi0[k]
        d_got = got["xi"][k] - xi0[k]
        bound = projection_bound(ref["solver"], k, insts[k], xi0[k], lam0[k], ref["lam"][k], precision)
        assert rel(d_got, d_ref) <= bound, (rel(d_got, d_ref), bound)
        np.testing.assert_allclose(got["lam"][k], ref["lam"][k], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("precision", ["tf32", "bf16x3"])
def test_tensor_core_3d_and_uneven(precision):
    insts = [sfgen.custom_instance(n=20, n_obs=10, H=60, n_d=3, seed=3, extent=(8.0, 8.0, 3.0)),
             sfgen.custom_instance(n=7, n_obs=4, H=33, n_d=3, seed=4, extent=(6.0, 6.0, 3.0))]
    rng = np.random.default_rng(8)
    xi0 = [i["xi"] + rng.normal(0, 0.1, size=i["xi"].shape) for i in insts]
    for x, i in zip(xi0, insts):
        x[:, :, 0] = i["bnd"][:, :, 0]
        x[:, :, -1] = i["bnd"][:, :, 1]
    lam0 = [rng.normal(0, 0.2, size=i["xi"].shape) for i in insts]
    ref = gpu_solve(insts, 1, precision="fp32", proj="dense", xi0=xi0, lam0=lam0)
    got = gpu_solve(insts, 1, precision=precision, proj="dense", xi0=xi0, lam0=lam0)
    for k, inst in enumerate(insts):
        bound = projection_bound(ref["solver"], k, inst, xi0[k], lam0[k], ref["lam"][k], precision)
        assert rel(got["xi"][k] - xi0[k], ref["xi"][k] - xi0[k]) <= bound


@pytest.mark.parametrize("precision,n_refine", [("bf16x3", 1), ("tf32", 2), ("bf16", 5)])
def test_tensor_core_run_error_against_the_oracle(precision, n_refine):
    """200 iterations of config 2 (3 instances) with refinement: the maximum position error
    and the final residual difference against the FP64 oracle within the reduced-precision
    tolerances (1e-4 m, 1e-3 m).  Unrefined products are held to their format's one-step
    bound above; over 200 iterations they drift by 2e-3 to 9e-2 m and carry no tolerance."""
    insts = sfgen.make_batch(2, B=3)
    out = gpu_solve(insts, 200, precision=precision, proj="dense", n_refine=n_refine)
    W = oracle.basis(100, 11)
    errs, rdiff = [], []
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, 200, rho=RHO)
        errs.append(max_pos_err(inst, out["xi"][k], ref["xi"], W))
        rdiff.append(abs(out["resid"][k, 1] - oracle.residual(inst, ref["xi"])[1]))
    print("\nTCRUN %s refine %d: max position error %.3e m, max final-residual difference %.3e m"
          % (precision, n_refine, max(errs), max(rdiff)))
    assert max(errs) <= 1e-4 and max(rdiff) <= 1e-3


@pytest.mark.parametrize("precision", ["tf32", "bf16x3"])
def test_adjoint_through_the_tensor_core_projection(precision):
    import torch
    from test_gpu_backward import gpu_grad, seeds
    insts = sfgen.make_batch(2, B=2)
    gxo, glo, grp2 = seeds(insts, 2)
    ref = gpu_grad(insts, 10, gxo, glo, grp2, precision="fp32", ckpt=4)
    got = gpu_grad(insts, 10, gxo, glo, grp2, precision=precision, ckpt=4)
    for a, b in zip(got, ref):
        for k in range(2):
            assert rel(a[k], b[k]) <= 2.5 * BOUND[precision], rel(a[k], b[k])
