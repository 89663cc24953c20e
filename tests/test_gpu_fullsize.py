"""Full-size workloads in the launch configuration the benchmark times (autotuned cluster
and CTA size), checked on sampled instances against the oracle and, at any size,
through properties that need no oracle run.

Configurations: 64 uneven instances (200 iterations); 128 instances of 32 robots through
the differentiable solve (50 unrolled iterations, checkpoints every 10, loss
||r_p||^2 + 0.1 ||out - candidate||^2); 16 instances of 64 robots in 3D (300 iterations;
the oracle takes minutes per instance there, so it checks 30 iterations of the same
launch, and FP32 is held to FP64 over the whole run).  Tolerances as in the parity
tests: FP64 1e-10 relative, FP32 1e-4 m in position and 1e-3 m in the final residual.
"""
import numpy as np
import pytest
import torch

import oracle
import sfgen
from gpu_util import (SENS_DRAWS, SENS_ULPS, check_adjoint_per_instance, check_positions_per_instance, max_pos_err,
                      rel, ulp_perturbed)
from paper_2510_09204_b300 import SFSolve, SFSolver

pytestmark = pytest.mark.gpu
RHO = 0.3


def tuned(insts, precision, proj, iters, ckpt=0):
    cfg_nd = insts[0]["n_d"]
    s = SFSolver(insts, cfg_nd, 11, rho=RHO, precision=precision, proj=proj, max_iters=iters, ckpt_every=ckpt)
    d = s.pack(insts)
    s.autotune(d, d["xi"], iters, reps=1)
    return s, d


def rounded32(inst):
    """The instance as an FP32 handle holds it: every array and shape parameter rounded to
    float32 (an FP32 solve cannot see finer input than that)."""
    p = dict(inst)
    for key in ("xi", "bnd", "obs_c", "obs_ab", "pmin", "pmax"):
        p[key] = np.asarray(inst[key], dtype=np.float32).astype(np.float64)
    for key in ("a", "b"):
        p[key] = float(np.float32(inst[key]))
    return p


def unpack_all(s, flat, B):
    return [s.unpack(flat, k).double().cpu().numpy() for k in range(B)]


def boundary_exact(s, xo, insts):
    for k, inst in enumerate(insts):
        x = s.unpack(xo, k).cpu().numpy()
        b = inst["bnd"].astype(x.dtype)
        assert np.array_equal(x[:, :, 0], b[:, :, 0]) and np.array_equal(x[:, :, -1], b[:, :, 1])


def test_uneven_64_instances_fp32_structured():
    insts = sfgen.make_batch(3)
    iters = sfgen.CONFIGS[3].iters
    s, d = tuned(insts, "fp32", "structured", iters)
    xo, _, res = s.solve(d, d["xi"], iters)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    boundary_exact(s, xo, insts)
    xs = unpack_all(s, xo, len(insts))
    r = res.cpu().numpy()
    cost = [i["n"] * (i["n"] + i["n_obs"]) * i["H"] for i in insts]
    order = np.argsort(cost)
    for k in (int(order[0]), int(order[len(order) // 4])):   # the cheapest and a lower-quartile instance
        inst = insts[k]
        ref = oracle.solve(inst, iters, rho=RHO)
        W = oracle.basis(inst["H"], 11)
        assert max_pos_err(inst, xs[k], ref["xi"], W) <= 1e-4
        assert abs(r[k, 1] - oracle.residual(inst, ref["xi"], rho=RHO)[1]) <= 1e-3
    # the FP64 residual kernel on the GPU's own output (and the data as the FP32 handle
    # holds it), any instance
    k = int(order[-1])
    rr = oracle.residual(rounded32(insts[k]), xs[k], rho=RHO)
    np.testing.assert_allclose(r[k, :2], rr[:2], rtol=1e-9, atol=1e-12)
    # the two largest instances (up to 64 robots, 120 timesteps) against the oracle, 40
    # iterations of the same launch (the oracle takes seconds per iteration there)
    x40, _, r40 = s.solve(d, d["xi"], 40)
    torch.cuda.synchronize()
    for k in (int(order[-1]), int(order[-2])):
        inst = rounded32(insts[k])
        ref = oracle.solve(inst, 40, rho=RHO)
        W = oracle.basis(inst["H"], 11)
        err = max_pos_err(inst, s.unpack(x40, k).double().cpu().numpy(), ref["xi"], W)
        print("\nconfig 3 instance %d (n %d, n_obs %d, H %d), 40 iterations: FP32 vs oracle %.2e m"
              % (k, inst["n"], inst["n_obs"], inst["H"], err))
        assert err <= 1e-4
        assert abs(r40[k, 1].item() - oracle.residual(inst, ref["xi"], rho=RHO)[1]) <= 1e-3


def test_uneven_64_instances_fp32_against_fp64_per_instance():
    """Every instance of the uneven batch (200 iterations, the benchmark's launch) against the
    FP64 GPU solve of the same input as FP32 holds it (FP64 is pinned to the oracle
    elsewhere), with the per-instance exception rule of check_positions_per_instance."""
    insts = [rounded32(i) for i in sfgen.make_batch(3)]
    iters = sfgen.CONFIGS[3].iters

    def run(batch, prec):
        s, d = tuned(batch, prec, "structured", iters)
        xo, _, res = s.solve(d, d["xi"], iters)
        torch.cuda.synchronize()
        assert (s.status() == 0).all()
        out = unpack_all(s, xo, len(batch)), res.cpu().numpy()
        s.close()
        return out

    x32, r32 = run(insts, "fp32")
    x64, r64 = run(insts, "fp64")
    pert = [run([ulp_perturbed(i, 100 * s + k, SENS_ULPS) for k, i in enumerate(insts)], "fp64")[0]
            for s in range(SENS_DRAWS)]
    err, sens = [], []
    for k, inst in enumerate(insts):
        W = oracle.basis(inst["H"], 11)
        err.append(max_pos_err(inst, x32[k], x64[k], W))
        sens.append(max(max_pos_err(inst, p[k], x64[k], W) for p in pert))
    check_positions_per_instance(err, sens, what="config 3")
    assert np.abs(r32[:, 1] - r64[:, 1]).max() <= 1e-3


def test_differentiable_128_instances_fp64_autograd():
    insts = sfgen.make_batch(4)
    iters = sfgen.CONFIGS[4].iters
    s, d = tuned(insts, "fp64", "structured", iters, ckpt=10)
    xc = d["xi"].clone().requires_grad_(True)
    x0 = xc.detach().clone().requires_grad_(True)
    l0 = torch.zeros_like(xc, requires_grad=True)
    xo, lo, rp2, _ = SFSolve.apply(xc, x0, l0, s, d, iters)
    loss = rp2.sum() + 0.1 * ((xo - xc) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    for k in (0, 77):
        inst = insts[k]
        ref = oracle.solve(inst, iters, rho=RHO)
        out = s.unpack(xo.detach(), k).cpu().numpy()
        assert rel(out, ref["xi"]) <= 1e-10
        gx, gx0, gl0 = oracle.solve_backward(inst, iters, 0.2 * (out - inst["xi"]), None, 1.0, rho=RHO,
                                             xi0=inst["xi"], lam0=np.zeros_like(inst["xi"]))
        ref_xc = gx - 0.2 * (out - inst["xi"])
        assert rel(s.unpack(xc.grad, k).cpu().numpy(), ref_xc) <= 1e-9
        assert rel(s.unpack(x0.grad, k).cpu().numpy(), gx0) <= 1e-9
        assert rel(s.unpack(l0.grad, k).cpu().numpy(), gl0) <= 1e-9


def adjoint_run(insts, prec, iters, ckpt, seed):
    s, d = tuned(insts, prec, "structured", iters, ckpt=ckpt)
    xo, _, res = s.solve(d, d["xi"], iters)
    g = torch.as_tensor(np.random.default_rng(seed).normal(size=xo.numel()) * 1e-2, dtype=xo.dtype, device="cuda")
    gx, _, _ = s.backward(g, None, torch.ones(len(insts), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    out = (unpack_all(s, xo, len(insts)), res.cpu().numpy(), unpack_all(s, gx, len(insts)))
    s.close()
    return out


def test_differentiable_128_instances_fp32_against_fp64():
    """The FP32 differentiable step on the whole batch against the FP64 GPU step (itself
    pinned to the oracle above) on the same input as FP32 holds it: outputs within the
    FP32 tolerance, gradients per instance within the bound of check_adjoint_per_instance.
    (Some instances here amplify input perturbations by ~300 in 50 iterations even in
    exact arithmetic: rounding the candidate to float32 alone moves the oracle's answer by
    up to 8e-5 m, which is why the reference takes the rounded input.)"""
    insts = [rounded32(i) for i in sfgen.make_batch(4)]
    iters = sfgen.CONFIGS[4].iters
    outs = {p: adjoint_run(insts, p, iters, 10, 4) for p in ("fp64", "fp32")}
    outs["fp64p"] = [adjoint_run([ulp_perturbed(i, 100 * s + k, SENS_ULPS) for k, i in enumerate(insts)], "fp64",
                                 iters, 10, 4)[2] for s in range(SENS_DRAWS)]
    W = oracle.basis(100, 11)
    errs = [max_pos_err(i, a, b, W) for i, a, b in zip(insts, outs["fp32"][0], outs["fp64"][0])]
    print("\nconfig 4 FP32 vs FP64 (rounded input): max position error %.2e m (median %.2e)"
          % (max(errs), np.median(errs)))
    assert max(errs) <= 1e-4
    assert np.abs(outs["fp32"][1][:, 1] - outs["fp64"][1][:, 1]).max() <= 1e-3
    check_adjoint_per_instance(outs["fp32"][2], outs["fp64"][2], outs["fp64p"], what="config 4")


def test_benchmark_step_config2():
    """The benchmark's step exactly: all 32 instances of the 16-robot 2-D config, FP32,
    structured projection, autotuned geometry, a checkpoint every iteration, forward,
    FP64 residual check and adjoint of the 200 iterations.  Forward: sampled instances
    against the oracle on the input as FP32 holds it.  Adjoint: per instance against the
    FP64 GPU step (pinned to the oracle's reverse pass elsewhere) on the same input, within
    the bound of check_adjoint_per_instance."""
    insts = [rounded32(i) for i in sfgen.make_batch(2)]
    iters = sfgen.CONFIGS[2].iters
    outs = {p: adjoint_run(insts, p, iters, 1, 2) for p in ("fp64", "fp32")}
    outs["fp64p"] = [adjoint_run([ulp_perturbed(i, 100 * s + k, SENS_ULPS) for k, i in enumerate(insts)], "fp64",
                                 iters, 1, 2)[2] for s in range(SENS_DRAWS)]
    s = SFSolver(insts, 2, 11, rho=RHO, precision="fp32", proj="structured", max_iters=iters)
    d = s.pack(insts)
    xo, _, _ = s.solve(d, d["xi"], iters)
    torch.cuda.synchronize()
    boundary_exact(s, xo, insts)
    W = oracle.basis(100, 11)
    for k in (0, 13, 31):
        ref = oracle.solve(insts[k], iters, rho=RHO)
        assert max_pos_err(insts[k], outs["fp32"][0][k], ref["xi"], W) <= 1e-4
        assert abs(outs["fp32"][1][k, 1] - oracle.residual(insts[k], ref["xi"], rho=RHO)[1]) <= 1e-3
    errs = [max_pos_err(i, a, b, W) for i, a, b in zip(insts, outs["fp32"][0], outs["fp64"][0])]
    assert max(errs) <= 1e-4
    check_adjoint_per_instance(outs["fp32"][2], outs["fp64"][2], outs["fp64p"], what="config 2")


@pytest.mark.parametrize("proj", ["structured", "dense"])
def test_3d_64_robots_fp32(proj):
    insts = sfgen.make_batch(5)
    iters = sfgen.CONFIGS[5].iters
    W = oracle.basis(100, 11)
    s64, d64 = tuned(insts, "fp64", proj, iters)
    s32, d32 = tuned(insts, "fp32", proj, iters)
    # 30 iterations of the full batch against the oracle on one sampled instance
    x64, _, _ = s64.solve(d64, d64["xi"], 30)
    x32, _, _ = s32.solve(d32, d32["xi"], 30)
    torch.cuda.synchronize()
    ref = oracle.solve(insts[5], 30, rho=RHO)
    assert rel(s64.unpack(x64, 5).cpu().numpy(), ref["xi"]) <= 1e-10
    assert max_pos_err(insts[5], s32.unpack(x32, 5).double().cpu().numpy(), ref["xi"], W) <= 1e-4
    # the whole run: FP32 against FP64 on every instance
    x64, _, r64 = s64.solve(d64, d64["xi"], iters)
    x32, _, r32 = s32.solve(d32, d32["xi"], iters)
    torch.cuda.synchronize()
    assert (s32.status() == 0).all() and (s64.status() == 0).all()
    boundary_exact(s32, x32, insts)
    a, b = unpack_all(s32, x32, len(insts)), unpack_all(s64, x64, len(insts))
    errs = [max_pos_err(i, u, v, W) for i, u, v in zip(insts, a, b)]
    print("\nconfig 5 %s: FP32 vs FP64 max position error %.2e m" % (proj, max(errs)))
    assert max(errs) <= 1e-4
    assert np.abs(r32.cpu().numpy()[:, 1] - r64.cpu().numpy()[:, 1]).max() <= 1e-3


@pytest.mark.parametrize("precision,n_refine", [("bf16x3", 1), ("tf32", 3), ("bf16", 5)])
def test_3d_64_robots_tensor_core_meets_the_fp32_tolerance(precision, n_refine):
    """The mixed-precision configuration: the projection on tensor cores with refinement
    against FP64 on the whole batch, every instance within the reduced-precision
    tolerance (1e-4 m in position, 1e-3 m in the final residual).  The pass counts are the
    ones each format needs here: BF16 gains about a factor 5-10 per pass (3 passes leave
    4e-4 m, 4 leave 5e-5 m, 5 leave 2.5e-5 m), TF32 a factor 3, BF16 x3 is at FP32 accuracy
    after one."""
    insts = sfgen.make_batch(5)
    iters = sfgen.CONFIGS[5].iters
    W = oracle.basis(100, 11)
    s64 = SFSolver(insts, 3, 11, rho=RHO, precision="fp64", proj="dense", max_iters=iters)
    d64 = s64.pack(insts)
    x64, _, r64 = s64.solve(d64, d64["xi"], iters)
    s = SFSolver(insts, 3, 11, rho=RHO, precision=precision, proj="dense", max_iters=iters, n_refine=n_refine)
    d = s.pack(insts)
    xt, _, rt = s.solve(d, d["xi"], iters)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    errs = [max_pos_err(i, u, v, W) for i, u, v in
            zip(insts, unpack_all(s, xt, len(insts)), unpack_all(s64, x64, len(insts)))]
    rdiff = np.abs(rt.cpu().numpy()[:, 1] - r64.cpu().numpy()[:, 1]).max()
    print("\nconfig 5 %s + %d refinement: max position error %.2e m, residual difference %.2e m"
          % (precision, n_refine, max(errs), rdiff))
    assert max(errs) <= 1e-4 and rdiff <= 1e-3
