"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 GPU vs oracle <= 1e-10 relative per iterate (||dz|| / ||z||);
FP32 paths <= 1e-4 m maximum position error and <= 1e-3 m difference in the final
maximum constraint residual.
"""
import numpy as np
import pytest

import oracle
import pinlib
import sfgen
from gpu_util import gpu_solve, max_pos_err, rel

pytestmark = pytest.mark.gpu
RHO = 0.3


def _sub(inst, n=None, n_obs=None):
    """A smaller instance cut from a generated one (first n robots / n_obs obstacles)."""
    out = dict(inst)
    if n is not None:
        out.update(n=n, xi=inst["xi"][:, :n].copy(), bnd=inst["bnd"][:, :n].copy())
    if n_obs is not None:
        out.update(n_obs=n_obs, obs_c=inst["obs_c"][:n_obs].copy(), obs_ab=inst["obs_ab"][:n_obs].copy())
    return out


@pytest.mark.parametrize("n,n_obs,H", [(4, 4, 50), (16, 20, 100), (1, 0, 10), (3, 2, 7), (64, 100, 100)])
def test_fp64_factorisation_matches_oracle(n, n_obs, H):
    inst = sfgen.custom_instance(n=min(n, 8), n_obs=min(n_obs, 4), H=H, seed=1)
    inst = dict(inst, n=n, n_obs=n_obs,
                xi=np.zeros((2, n, 11)), bnd=np.zeros((2, n, 2)),
                obs_c=np.zeros((n_obs, 2)), obs_ab=np.ones((n_obs, 2)))
    from paper_2510_09204_b300 import SFSolver
    s = SFSolver([inst], 2, 11, rho=RHO, precision="fp64", max_iters=1)
    np.testing.assert_allclose(s.operator(0, 0), oracle.basis(H, 11), atol=1e-14)
    if n * 11 <= 400:
        _, Pe, Pb = oracle.kkt(2, 11, RHO, n, n_obs, H)
        np.testing.assert_allclose(s.operator(0, 1), Pe, atol=1e-12)
        np.testing.assert_allclose(s.operator(0, 2), Pb, atol=1e-12)
    else:  # large shapes: the Kronecker closed form (pinned against the oracle on CPU)
        W = pinlib.bernstein(H, 11)
        A0 = np.vstack([W[0], W[-1]])

        def cinv(c):
            K = np.block([[np.eye(11) + RHO * c * W.T @ W, A0.T], [A0, np.zeros((2, 2))]])
            return np.linalg.inv(K)[:11, :11]

        Q = np.ones((n, n)) / n
        ref = np.kron(np.eye(n) - Q, cinv(n + n_obs + 2)) + np.kron(Q, cinv(n_obs + 2))
        np.testing.assert_allclose(s.operator(0, 1), ref, atol=1e-12)


def test_fp64_every_iterate_matches_oracle():
    """Iterate by iterate: one-iteration solves chained through (xi0, lam0)."""
    inst = sfgen.make_batch(1)[0]
    tr = oracle.solve(inst, 30, rho=RHO, traj=True)["traj"]
    x, l = inst["xi"], np.zeros_like(inst["xi"])
    for it in range(30):
        out = gpu_solve([inst], 1, xi0=[x], lam0=[l])
        x, l = out["xi"][0], out["lam"][0]
        z = np.concatenate([x.ravel(), l.ravel()])
        zr = np.concatenate([tr[it + 1, 0].ravel(), tr[it + 1, 1].ravel()])
        assert rel(z, zr) <= 1e-10, (it, rel(z, zr))


@pytest.mark.parametrize("cid,B,iters", [(1, 1, 100), (2, 3, 200)])
def test_fp64_run_matches_oracle(cid, B, iters):
    insts = sfgen.make_batch(cid, B=B)
    out = gpu_solve(insts, iters)
    assert (out["status"] == 0).all()
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, iters, rho=RHO)
        z = np.concatenate([out["xi"][k].ravel(), out["lam"][k].ravel()])
        zr = np.concatenate([ref["xi"].ravel(), ref["lam"].ravel()])
        assert rel(z, zr) <= 1e-10, rel(z, zr)


def test_fp64_boundary_mismatch_and_warm_start():
    """(xi0, lam0) from an initialisation network need not meet A xi = b: the first step's
    P_b (b - A xi_bar^0) term restores it."""
    inst = sfgen.make_batch(1)[0]
    rng = np.random.default_rng(3)
    xi0 = inst["xi"] + rng.normal(0, 0.2, size=inst["xi"].shape)
    lam0 = rng.normal(0, 0.1, size=inst["xi"].shape)
    ref = oracle.solve(inst, 5, rho=RHO, xi0=xi0, lam0=lam0)
    out = gpu_solve([inst], 5, xi0=[xi0], lam0=[lam0])
    assert rel(out["xi"][0], ref["xi"]) <= 1e-10
    assert rel(out["lam"][0], ref["lam"]) <= 1e-10


def test_fp64_residual_outputs_match_oracle():
    insts = sfgen.make_batch(2, B=3)
    out = gpu_solve(insts, 40)
    for k, inst in enumerate(insts):
        r = oracle.residual(inst, out["xi"][k])
        np.testing.assert_allclose(out["resid"][k, 0], r[0], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(out["resid"][k, 1], r[1], rtol=1e-10, atol=1e-12)
        h = oracle.solve(inst, 40, rho=RHO, hist=True)["hist"]
        np.testing.assert_allclose(out["resid"][k, 2], h[-1, 2], rtol=1e-8, atol=1e-12)


def test_structured_projection_equals_dense():
    insts = sfgen.make_batch(2, B=2)
    a = gpu_solve(insts, 60, proj="dense")
    b = gpu_solve(insts, 60, proj="structured")
    for k in range(2):
        assert rel(b["xi"][k], a["xi"][k]) <= 1e-11
        assert rel(b["lam"][k], a["lam"][k]) <= 1e-11


@pytest.mark.parametrize("aniso,dyn", [(False, False), (True, False), (False, True)])
def test_fp64_3d_anisotropic_dynamic(aniso, dyn):
    inst = sfgen.custom_instance(n=6, n_obs=5, H=30, n_d=3, seed=4, extent=(6.0, 6.0, 3.0), dyn_obs=dyn)
    if aniso:
        inst = dict(inst, b=0.3, obs_ab=inst["obs_ab"] * np.array([1.0, 0.7]))
    ref = oracle.solve(inst, 50, rho=RHO)
    out = gpu_solve([inst], 50)
    z = np.concatenate([out["xi"][0].ravel(), out["lam"][0].ravel()])
    zr = np.concatenate([ref["xi"].ravel(), ref["lam"].ravel()])
    assert rel(z, zr) <= 1e-10


def test_fp64_uneven_batch_and_edge_shapes():
    """One launch over uneven instances, including one robot (no pair rows), no obstacles,
    the shortest horizon H = 2 and a horizon that is not a multiple of the chunk."""
    base = sfgen.make_batch(3, B=3)
    insts = [_sub(base[0], n=1, n_obs=0),
             _sub(base[1], n=3, n_obs=4),
             dict(_sub(base[2], n=9, n_obs=0), H=2),
             sfgen.custom_instance(n=40, n_obs=7, H=117, seed=9)]
    out = gpu_solve(insts, 25)
    assert (out["status"] == 0).all()
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, 25, rho=RHO)
        z = np.concatenate([out["xi"][k].ravel(), out["lam"][k].ravel()])
        zr = np.concatenate([ref["xi"].ravel(), ref["lam"].ravel()])
        assert rel(z, zr) <= 1e-10, (k, rel(z, zr))


def test_zero_iterations_returns_the_initial_iterate():
    inst = sfgen.make_batch(1)[0]
    out = gpu_solve([inst], 0)
    np.testing.assert_array_equal(out["xi"][0], inst["xi"])
    np.testing.assert_array_equal(out["lam"][0], 0.0)
    r = oracle.residual(inst, inst["xi"])
    np.testing.assert_allclose(out["resid"][0, 1], r[1], rtol=1e-10)


@pytest.mark.parametrize("proj", ["dense", "structured"])
def test_fp32_within_tolerance(proj):
    insts = sfgen.make_batch(2, B=3)
    out = gpu_solve(insts, 200, precision="fp32", proj=proj)
    W = oracle.basis(insts[0]["H"], 11)
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, 200, rho=RHO)
        err = max_pos_err(inst, out["xi"][k], ref["xi"], W)
        assert err <= 1e-4, err
        r_ref = oracle.residual(inst, ref["xi"])[1]
        assert abs(out["resid"][k, 1] - r_ref) <= 1e-3


def test_fp32_full_config2_batch_sampled():
    """The benchmark's launch: all 32 instances of the 16-robot 2D config, 200 iterations,
    FP32; three sampled instances against the oracle."""
    insts = sfgen.make_batch(2)
    out = gpu_solve(insts, 200, precision="fp32")
    assert (out["status"] == 0).all()
    W = oracle.basis(100, 11)
    for k in (0, 13, 31):
        ref = oracle.solve(insts[k], 200, rho=RHO)
        assert max_pos_err(insts[k], out["xi"][k], ref["xi"], W) <= 1e-4
        assert np.all(out["xi"][k][:, :, 0] == np.float32(insts[k]["bnd"][:, :, 0]))


@pytest.mark.parametrize("proj", ["dense", "structured"])
@pytest.mark.parametrize("cluster,threads", [(1, 512), (2, 256), (3, 128), (5, 96), (8, 64)])
def test_fp64_every_cluster_geometry_matches_oracle(cluster, threads, proj):
    """The instance split over 1..8 CTAs of a cluster (shares of 100 timesteps that are
    not multiples of each other) gives the oracle's iterates whatever the geometry."""
    insts = sfgen.make_batch(2, B=2)
    out = gpu_solve(insts, 30, proj=proj, cluster=cluster, threads=threads)
    assert out["solver"].launch()[0] == cluster
    assert (out["status"] == 0).all()
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, 30, rho=RHO)
        z = np.concatenate([out["xi"][k].ravel(), out["lam"][k].ravel()])
        zr = np.concatenate([ref["xi"].ravel(), ref["lam"].ravel()])
        assert rel(z, zr) <= 1e-10, (cluster, threads, rel(z, zr))
        r = oracle.residual(inst, out["xi"][k])
        np.testing.assert_allclose(out["resid"][k, :2], r[:2], rtol=1e-9, atol=1e-12)


def test_set_launch_rejects_bad_geometry():
    from paper_2510_09204_b300 import SFError
    insts = sfgen.make_batch(1)
    out = gpu_solve(insts, 1)
    s = out["solver"]
    for bad in [(9, 0), (-1, 0), (1, 48), (1, 100), (1, 1024)]:
        with pytest.raises(SFError):
            s.set_launch(*bad)


def test_autotune_keeps_a_valid_geometry_and_results():
    insts = sfgen.make_batch(2, B=3)
    out = gpu_solve(insts, 20)
    s, data = out["solver"], out["data"]
    c, t, ms = s.autotune(data, data["xi"], 20, reps=1)
    assert 1 <= c <= 8 and t in (128, 256, 512) and ms > 0
    assert s.launch()[:2] == (c, t)
    xo, lo, res = s.solve(data, data["xi"], 20)
    import torch
    torch.cuda.synchronize()
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, 20, rho=RHO)
        assert rel(s.unpack(xo, k).cpu().numpy(), ref["xi"]) <= 1e-10


@pytest.mark.parametrize("cluster,threads", [(4, 1024), (1, 1024), (8, 1024)])
def test_fp32_large_ctas_within_tolerance(cluster, threads):
    insts = sfgen.make_batch(2, B=2)
    out = gpu_solve(insts, 100, precision="fp32", proj="structured", cluster=cluster, threads=threads)
    W = oracle.basis(insts[0]["H"], 11)
    for k, inst in enumerate(insts):
        ref = oracle.solve(inst, 100, rho=RHO)
        assert max_pos_err(inst, out["xi"][k], ref["xi"], W) <= 1e-4


@pytest.mark.parametrize("precision,proj", [("fp64", "dense"), ("fp32", "structured")])
def test_zero_iterations_pass_the_input_through(precision, proj):
    """iters = 0: the outputs are the initial iterate (xi_bar^0 = xi_cand, lambda^0 = 0) bit
    for bit, the residual is the candidate's, and the adjoint passes the seeds through
    (dL/dxi_cand = dL/dxi_bar^L and dL/dlambda^0 = dL/dlambda^L when ||r_p||^2 has no seed)."""
    import torch
    from paper_2510_09204_b300 import SFSolver
    insts = sfgen.make_batch(2, B=3)
    s = SFSolver(insts, 2, 11, rho=RHO, precision=precision, proj=proj, max_iters=5, ckpt_every=1)
    d = s.pack(insts)
    xo, lo, res = s.solve(d, d["xi"], 0)
    g = torch.randn_like(xo)
    gl = torch.randn_like(xo)
    gx, gx0, gl0 = s.backward(g, gl, None)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    assert torch.equal(xo, d["xi"])
    assert torch.equal(lo, torch.zeros_like(lo))
    assert torch.equal(gx, g)
    assert torch.equal(gl0, gl)
    for k, inst in enumerate(insts):
        if precision == "fp32":   # the instance as an FP32 handle holds it
            inst = dict(inst, **{key: np.asarray(inst[key], dtype=np.float32).astype(np.float64)
                                 for key in ("obs_c", "obs_ab", "pmin", "pmax")},
                        a=float(np.float32(inst["a"])), b=float(np.float32(inst["b"])))
        r = oracle.residual(inst, s.unpack(d["xi"], k).double().cpu().numpy())
        np.testing.assert_allclose(res.cpu().numpy()[k, :2], r[:2], rtol=1e-9, atol=1e-12)
    s.close()


def test_early_exit_stops_converged_instances_only():
    """SF_OPT_EARLY_EXIT: an instance whose iterate l met the tolerance returns the iterate
    of iteration l + 1, bit for bit the plain solve run for l + 1 iterations; instances that
    never meet it return the full run's bits; a handle with checkpoints refuses the option."""
    import torch
    from paper_2510_09204_b300 import SFError, SFSolver
    from paper_2510_09204_b300.sf import SF_OPT_EARLY_EXIT
    # three small instances that meet the tolerance within 15 iterations, three of the
    # 16-robot batch that do not meet it in 300
    insts = [sfgen.custom_instance(n=4, n_obs=2, H=30, seed=s, extent=8.0, sigma=0.3) for s in range(3)]
    insts += sfgen.make_batch(2, B=3)
    iters = 300

    def run(n_it, early):
        s = SFSolver(insts, 2, 11, rho=RHO, precision="fp32", proj="structured", max_iters=iters, tol=1e-3)
        if early:
            s.set_option(SF_OPT_EARLY_EXIT, 1)
            assert s.option(SF_OPT_EARLY_EXIT) == 1
        d = s.pack(insts)
        xo, _, res = s.solve(d, d["xi"], n_it)
        torch.cuda.synchronize()
        assert (s.status() == 0).all()
        return [s.unpack(xo, k).cpu().numpy().copy() for k in range(len(insts))], res.cpu().numpy()

    full, rf = run(iters, False)
    early, re = run(iters, True)
    its = rf[:, 3].astype(int)
    assert (re[:, 3].astype(int) == its).all()
    stopped = [k for k in range(len(insts)) if 0 <= its[k] < iters - 1]
    assert stopped == [0, 1, 2], its
    for k in range(len(insts)):
        if k in stopped:
            ref, _ = run(int(its[k]) + 1, False)
            assert np.array_equal(early[k], ref[k]), k
            assert re[k, 1] <= 1e-3 + 1e-6
        else:
            assert np.array_equal(early[k], full[k]), k
    s = SFSolver(insts, 2, 11, rho=RHO, precision="fp32", max_iters=10, ckpt_every=1)
    with pytest.raises(SFError):
        s.set_option(SF_OPT_EARLY_EXIT, 1)
