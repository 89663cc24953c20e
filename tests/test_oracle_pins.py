"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them re-types the oracle's own
formulas: the references are scipy/numpy library routines, brute-force searches,
closed forms, Kronecker-product constructions of the Appendix's matrices, and
invariances of the problem statement.
"""
import numpy as np
import pytest

import oracle
import pinlib
import sfgen


RHO = 0.3


# ---------------------------------------------------------------- basis (eq. poly)
def test_basis_is_bernstein():
    for H, nxi in [(2, 2), (7, 4), (50, 11), (101, 11), (120, 16)]:
        np.testing.assert_allclose(oracle.basis(H, nxi), pinlib.bernstein(H, nxi), rtol=0, atol=1e-13)


def test_basis_endpoint_and_linear_reproduction():
    W = oracle.basis(37, 9)
    np.testing.assert_allclose(W.sum(1), 1.0, atol=1e-14)           # partition of unity
    np.testing.assert_array_equal(W[0], np.eye(9)[0])               # start = coefficient 0
    np.testing.assert_array_equal(W[-1], np.eye(9)[-1])             # goal = last coefficient
    np.testing.assert_allclose(W @ (np.arange(9) / 8.0), np.linspace(0, 1, 37), atol=1e-14)


# ------------------------------------------------ alpha / beta / d steps (eqs. alpha..d_step)
@pytest.mark.parametrize("nd", [2, 3])
def test_estep_isotropic_is_exterior_ball_projection(nd):
    """For a = b the alpha, beta, d minimisers of rho/2 ||Delta - e||^2 over the spherical
    form with d >= 1 give the nearest point outside the radius-a ball (brute force)."""
    rng = np.random.default_rng(nd)
    a = 0.7
    for trial in range(12):
        D = rng.normal(size=nd) * (0.4 if trial % 2 else 1.5)
        e, _ = oracle.estep(D, a, a)
        ref = pinlib.exterior_projection_bruteforce(D, a)
        np.testing.assert_allclose(e, ref, atol=1e-9)


def test_estep_anisotropic_scaled_radial_projection():
    """Spheroid rows (a != b), reading of the beta/d steps: outside the spheroid e = Delta
    (d = the exact line-of-sight distance); inside, M^-1 e is the unit vector along M^-1 Delta."""
    rng = np.random.default_rng(7)
    a, b = 0.8, 0.5
    M = np.array([a, a, b])
    for trial in range(20):
        D = rng.normal(size=3)
        e, _ = oracle.estep(D, a, b)
        s = D / M
        if np.linalg.norm(s) > 1.0:
            np.testing.assert_allclose(e, D, atol=1e-13)
        else:
            np.testing.assert_allclose(e / M, s / np.linalg.norm(s), atol=1e-13)


@pytest.mark.parametrize("nd,a,b", [(2, 0.6, 0.6), (3, 0.6, 0.6), (3, 0.8, 0.5)])
def test_estep_jacobian_central_difference(nd, a, b):
    rng = np.random.default_rng(3)
    for trial in range(10):
        D = rng.normal(size=nd) * (0.3 if trial % 2 else 1.2)
        _, J = oracle.estep(D, a, b)
        eps = 1e-6
        Jfd = np.empty((nd, nd))
        for q in range(nd):
            dp, dm = D.copy(), D.copy()
            dp[q] += eps
            dm[q] -= eps
            Jfd[:, q] = (oracle.estep(dp, a, b)[0] - oracle.estep(dm, a, b)[0]) / (2 * eps)
        np.testing.assert_allclose(J, Jfd, atol=1e-7)


# ---------------------------------------------- xi_bar step matrices (Appendix, M and eta)
@pytest.mark.parametrize("n,n_obs,H,nxi", [(1, 0, 10, 5), (3, 2, 12, 6), (5, 4, 30, 11)])
def test_kkt_hessian_matches_appendix_matrices(n, n_obs, H, nxi):
    """H = I + rho F'F + rho G'G with F, G assembled as Kronecker products."""
    rho = 0.7
    _, F, G, A = pinlib.dense_mats(n, n_obs, H, nxi)
    Hm, Pe, Pb = oracle.kkt(2, nxi, rho, n, n_obs, H)
    ref = np.eye(n * nxi) + rho * F.T @ F + rho * G.T @ G
    np.testing.assert_allclose(Hm, ref, atol=1e-11 * np.abs(ref).max())
    # P_eta, P_b solve the KKT system [[H, A'], [A, 0]] (numpy dense solve)
    K = np.block([[ref, A.T], [A, np.zeros((2 * n, 2 * n))]])
    Kinv = np.linalg.inv(K)
    np.testing.assert_allclose(Pe, Kinv[:n * nxi, :n * nxi], atol=1e-11)
    np.testing.assert_allclose(Pb, Kinv[:n * nxi, n * nxi:], atol=1e-11)


@pytest.mark.parametrize("n,n_obs,H,nxi,rho", [(2, 0, 20, 7, 1.0), (6, 3, 25, 8, 0.3), (16, 20, 100, 11, 0.1)])
def test_kkt_kronecker_closed_form(n, n_obs, H, nxi, rho):
    """F'F + G'G = ((n + n_obs + 2) I - 11') (x) W'W, so with Q = 11'/n
    P_eta = (I - Q) (x) P_dev + Q (x) P_mean, P_dev / P_mean the n_xi x n_xi constrained
    inverses of I + rho (n + n_obs + 2) W'W and I + rho (n_obs + 2) W'W."""
    W = pinlib.bernstein(H, nxi)
    A0 = np.vstack([W[0], W[-1]])

    def cinv(c):
        K = np.block([[np.eye(nxi) + rho * c * W.T @ W, A0.T], [A0, np.zeros((2, 2))]])
        Ki = np.linalg.inv(K)
        return Ki[:nxi, :nxi], Ki[:nxi, nxi:]

    Pdev, Bdev = cinv(n + n_obs + 2)
    Pmean, Bmean = cinv(n_obs + 2)
    Q = np.ones((n, n)) / n
    ref_e = np.kron(np.eye(n) - Q, Pdev) + np.kron(Q, Pmean)
    ref_b = np.kron(np.eye(n) - Q, Bdev) + np.kron(Q, Bmean)
    _, Pe, Pb = oracle.kkt(2, nxi, rho, n, n_obs, H)
    np.testing.assert_allclose(Pe, ref_e, atol=1e-12)
    np.testing.assert_allclose(Pb, ref_b, atol=1e-12)


# ---------------------------------------------------- one AM sweep (eqs. alpha_step..xi_step)
@pytest.mark.parametrize("nd,H,seed,scale", [(2, 8, 0, 1.0), (2, 8, 1, 1.0), (3, 5, 2, 1.0), (2, 6, 3, 1.6)])
def test_one_sweep_is_block_argmin_of_augmented_lagrangian(nd, H, seed, scale):
    """From a random state (xi_bar, lambda), one oracle sweep equals the block minimisers of
    eq. aug_lag built independently: brute-force e, closed-form slack, lambda step, and a
    dense KKT solve of the equality-constrained xi_bar step."""
    inst = pinlib.small_instance(n=3, n_obs=2, H=H, n_d=nd, n_xi=6, seed=seed)
    rng = np.random.default_rng(100 + seed)
    xib = scale * inst["xi"] + rng.normal(0, 0.3, size=inst["xi"].shape)
    lam = rng.normal(0, 0.2, size=inst["xi"].shape)
    if scale > 1.0:  # the state leaves the workspace box: the slack clamp is exercised
        assert oracle.residual(inst, xib)[1] > 0.3
    got = oracle.solve(inst, 1, rho=RHO, xi0=xib, lam0=lam)
    ref_x, ref_l = pinlib.one_step_reference(inst, xib, lam, RHO)
    np.testing.assert_allclose(got["lam"], ref_l, atol=1e-8)
    np.testing.assert_allclose(got["xi"], ref_x, atol=1e-8)


# ------------------------------------------------------------------ invariants
def test_boundary_equality_every_iterate():
    """A xi_bar = b after every xi_bar step (eqs. boundary_con, xi_step)."""
    inst = sfgen.make_batch(1)[0]
    tr = oracle.solve(inst, 60, rho=RHO, traj=True)["traj"]
    xs = tr[1:, 0]
    np.testing.assert_allclose(xs[:, :, :, 0], np.broadcast_to(inst["bnd"][:, :, 0], xs[:, :, :, 0].shape), atol=1e-12)
    np.testing.assert_allclose(xs[:, :, :, -1], np.broadcast_to(inst["bnd"][:, :, 1], xs[:, :, :, -1].shape), atol=1e-12)


def _feasible_instance(nd=2):
    """Robots on parallel lanes 2 m apart, far from two obstacles, inside the box."""
    n, nxi, H = 4, 11, 40
    ramp = np.arange(nxi) / (nxi - 1)
    starts = np.array([[-3.0, -3.0 + 2.0 * i] + [0.0] * (nd - 2) for i in range(n)])
    goals = starts + np.array([6.0, 0.0] + [0.0] * (nd - 2))
    xi = starts.T[:, :, None] * (1 - ramp) + goals.T[:, :, None] * ramp
    xi[1, :, 1:-1] += 0.3 * np.sin(np.pi * ramp[1:-1])  # a gentle bend, still clear
    obs = np.array([[4.5, 4.5] + [0.0] * (nd - 2), [-4.5, 4.5] + [0.0] * (nd - 2)])
    return dict(n=n, n_obs=2, H=H, n_d=nd, n_xi=nxi, dyn_obs=False, a=0.5, b=0.5,
                pmin=np.full(nd, -5.0), pmax=np.full(nd, 5.0), obs_c=obs,
                obs_ab=np.array([[0.6, 0.6], [0.5, 0.5]]),
                bnd=np.stack([starts.T, goals.T], axis=-1).copy(), xi=np.ascontiguousarray(xi))


@pytest.mark.parametrize("nd", [2, 3])
def test_feasible_candidate_is_fixed_point(nd):
    """A candidate meeting every constraint, with lambda^0 = 0: e = F xi, s = h - G xi,
    r = 0, lambda stays 0 and xi_bar = xi in every iteration (Sec. IV-B, eq. fixed_point)."""
    inst = _feasible_instance(nd)
    out = oracle.residual(inst, inst["xi"])
    assert out[1] < 1e-12
    tr = oracle.solve(inst, 25, rho=RHO, traj=True)["traj"]
    np.testing.assert_allclose(tr[:, 0], np.broadcast_to(inst["xi"], tr[:, 0].shape), atol=1e-12)
    np.testing.assert_allclose(tr[:, 1], 0.0, atol=1e-12)


def test_single_robot_converges_to_affine_projection():
    """1 robot, no obstacles, inside the box: the projection is the textbook affine one,
    xi_bar = xi - A'(AA')^-1 (A xi - b)."""
    nxi, H = 9, 30
    rng = np.random.default_rng(5)
    xi = np.cumsum(rng.normal(0, 0.3, size=(2, 1, nxi)), axis=-1)
    bnd = np.stack([xi[:, :, 0] + 0.4, xi[:, :, -1] - 0.3], axis=-1)  # candidate violates A xi = b
    inst = dict(n=1, n_obs=0, H=H, n_d=2, n_xi=nxi, dyn_obs=False, a=0.5, b=0.5,
                pmin=np.full(2, -10.0), pmax=np.full(2, 10.0), obs_c=np.zeros((0, 2)),
                obs_ab=np.zeros((0, 2)), bnd=bnd, xi=xi)
    _, _, _, A = pinlib.dense_mats(1, 0, H, nxi)
    ref = np.empty_like(xi)
    for ax in range(2):
        x = xi[ax].ravel()
        ref[ax] = (x - A.T @ np.linalg.solve(A @ A.T, A @ x - bnd[ax].ravel())).reshape(1, nxi)
    got = oracle.solve(inst, 400, rho=RHO)["xi"]
    np.testing.assert_allclose(got, ref, atol=1e-10)


def test_permutation_equivariance():
    inst = sfgen.make_batch(2, B=1)[0]
    inst = dict(inst, n=6, xi=inst["xi"][:, :6].copy(), bnd=inst["bnd"][:, :6].copy())
    perm = np.array([3, 0, 5, 1, 4, 2])
    pinst = dict(inst, xi=inst["xi"][:, perm].copy(), bnd=inst["bnd"][:, perm].copy())
    a = oracle.solve(inst, 30, rho=RHO)
    b = oracle.solve(pinst, 30, rho=RHO)
    np.testing.assert_allclose(b["xi"], a["xi"][:, perm], atol=1e-10)
    np.testing.assert_allclose(b["lam"], a["lam"][:, perm], atol=1e-10)


def test_translation_equivariance():
    """Bernstein partition of unity: translating every position input by c translates
    xi_bar by c and leaves lambda unchanged."""
    inst = sfgen.make_batch(1)[0]
    c = np.array([1.25, -0.75])
    tinst = dict(inst, xi=inst["xi"] + c[:, None, None], bnd=inst["bnd"] + c[:, None, None],
                 obs_c=inst["obs_c"] + c, pmin=inst["pmin"] + c, pmax=inst["pmax"] + c)
    a = oracle.solve(inst, 40, rho=RHO)
    b = oracle.solve(tinst, 40, rho=RHO)
    np.testing.assert_allclose(b["xi"], a["xi"] + c[:, None, None], atol=1e-10)
    np.testing.assert_allclose(b["lam"], a["lam"], atol=1e-10)


def test_flat_3d_reproduces_2d():
    inst = sfgen.make_batch(1)[0]
    z = lambda arr, val=0.0: np.concatenate([arr, np.full((1,) + arr.shape[1:], val)], axis=0)
    i3 = dict(inst, n_d=3, xi=z(inst["xi"]), bnd=z(inst["bnd"]),
              obs_c=np.concatenate([inst["obs_c"], np.zeros((inst["n_obs"], 1))], axis=1),
              pmin=np.append(inst["pmin"], -5.0), pmax=np.append(inst["pmax"], 5.0))
    a = oracle.solve(inst, 40, rho=RHO)
    b = oracle.solve(i3, 40, rho=RHO)
    np.testing.assert_allclose(b["xi"][:2], a["xi"], atol=1e-10)
    np.testing.assert_allclose(b["xi"][2], 0.0, atol=1e-10)


def test_residual_decreases_over_the_run():
    """Reading: AM on a non-convex set is not monotone per iteration.  Pinned: the smallest
    primal residual reached is far below the initial one and the final one is below it."""
    for inst in sfgen.make_batch(2, B=3):
        h = oracle.solve(inst, 150, rho=RHO, hist=True)["hist"]
        assert h[:, 0].min() < 0.2 * h[0, 0]
        assert h[-1, 0] < h[0, 0]
        win = np.convolve(h[:, 0], np.ones(10) / 10, mode="valid")
        assert win[-1] < win[0]


# -------------------------------------------- brute-force projection (eqs. proj_cost..proj_robot)
def _one_obstacle_instance(H, oy, nxi=5):
    ramp = np.arange(nxi) / (nxi - 1)
    s, g = np.array([-2.0, 0.0]), np.array([2.0, 0.0])
    xi = (s[:, None] * (1 - ramp) + g[:, None] * ramp)[:, None, :].copy()
    return dict(n=1, n_obs=1, H=H, n_d=2, n_xi=nxi, dyn_obs=False, a=0.5, b=0.5,
                pmin=np.full(2, -5.0), pmax=np.full(2, 5.0), obs_c=np.array([[0.0, oy]]),
                obs_ab=np.array([[0.6, 0.6]]), bnd=np.stack([s, g], axis=-1)[:, None, :].copy(), xi=xi)


def _two_robot_instance(H, nxi=5, offset=0.3):
    ramp = np.arange(nxi) / (nxi - 1)
    s = np.array([[-2.0, offset / 2], [2.0, -offset / 2]])
    g = np.array([[2.0, offset / 2], [-2.0, -offset / 2]])
    xi = s.T[:, :, None] * (1 - ramp) + g.T[:, :, None] * ramp
    return dict(n=2, n_obs=0, H=H, n_d=2, n_xi=nxi, dyn_obs=False, a=0.5, b=0.5,
                pmin=np.full(2, -5.0), pmax=np.full(2, 5.0), obs_c=np.zeros((0, 2)),
                obs_ab=np.zeros((0, 2)), bnd=np.stack([s.T, g.T], axis=-1).copy(), xi=xi.copy())


def _box_instance(H=5, nxi=5):
    """One robot whose straight candidate bulges out of the box at a single timestep."""
    inst = _one_obstacle_instance(H, 0.0, nxi)
    xi = inst["xi"].copy()
    xi[1, 0, 1:-1] += np.array([1.0, 2.5, 1.0])[: nxi - 2]
    return dict(inst, n_obs=0, obs_c=np.zeros((0, 2)), obs_ab=np.zeros((0, 2)), xi=xi,
                pmax=np.array([5.0, 1.0]))


@pytest.mark.parametrize("make", [lambda: _box_instance(),
                                  lambda: _one_obstacle_instance(5, 0.3),
                                  lambda: _one_obstacle_instance(5, -0.2),
                                  lambda: _two_robot_instance(5)])
def test_single_row_conflict_converges_to_bruteforce_projection(make):
    """When a single constraint row is ever violated, the AM fixed point is the projection
    of eqs. proj_cost..proj_robot: compared with an SLSQP solve of the original problem."""
    inst = make()
    ref, res = pinlib.projection_bruteforce(inst)
    assert res.success
    got = oracle.solve(inst, 20000, rho=0.1, hist=True)
    assert got["hist"][-1, 2] < 1e-13          # converged
    W = pinlib.bernstein(inst["H"], inst["n_xi"])
    P1 = np.einsum("kc,dic->dik", W, got["xi"])
    P2 = np.einsum("kc,dic->dik", W, ref)
    assert np.abs(P1 - P2).max() < 1e-6


def test_multi_row_conflict_lands_on_feasible_point_near_projection():
    """Reading (reported): with several violated rows the AM fixed point is feasible but not
    the Euclidean projection, because lambda never decays on rows that became inactive and
    the small-rho limit follows the flow of F'r_1, whose metric is F'F.  Pinned: the fixed
    point is feasible, its distance to the candidate is at least the projection's, and the
    gap is a few millimetres at rho = 0.1."""
    inst = _two_robot_instance(30, nxi=7)
    ref, res = pinlib.projection_bruteforce(inst)
    assert res.success
    got = oracle.solve(inst, 20000, rho=0.1, hist=True)
    assert got["hist"][-1, 2] < 1e-12 and oracle.residual(inst, got["xi"])[1] < 1e-12
    d_am = np.linalg.norm(got["xi"] - inst["xi"])
    d_bf = np.linalg.norm(ref - inst["xi"])
    assert d_am >= d_bf - 1e-9
    W = pinlib.bernstein(inst["H"], inst["n_xi"])
    gap = np.abs(np.einsum("kc,dic->dik", W, got["xi"] - ref)).max()
    assert 1e-4 < gap < 2e-2


# ------------------------------------------------------------ gradients (Sec. IV-B, Fig. unroll)
def _grad_instance(nd, seed, iters, aniso=False):
    """A small conflicting instance whose rows stay clear of every kink during the run."""
    for s in range(seed, seed + 200):
        inst = pinlib.small_instance(n=3, n_obs=2, H=10, n_d=nd, n_xi=6, seed=s, aniso=aniso)
        h = oracle.solve(inst, iters, rho=RHO, hist=True)["hist"]
        fin = oracle.residual(inst, oracle.solve(inst, iters, rho=RHO)["xi"])
        if h[:, 3].min() > 1e-3 and fin[2] > 1e-3 and h[0, 1] > 0.05:
            return inst
    raise RuntimeError("no kink-free instance found")


@pytest.mark.parametrize("nd,aniso", [(2, False), (3, False), (3, True)])
def test_backward_matches_torch_autograd(nd, aniso):
    import torch
    iters = 6
    inst = _grad_instance(nd, 10 * nd + aniso, iters, aniso)
    W, F, G, A = pinlib.dense_mats(inst["n"], inst["n_obs"], inst["H"], inst["n_xi"])
    T, rsq = pinlib.torch_T(inst, RHO, W, F, G, A)
    rng = np.random.default_rng(1)
    gx_out = rng.normal(size=inst["xi"].shape)
    gl_out = rng.normal(size=inst["xi"].shape)
    xi_c = torch.tensor(inst["xi"], requires_grad=True)
    lam0 = torch.tensor(rng.normal(0, 0.1, size=inst["xi"].shape), requires_grad=True)
    xi0 = torch.tensor(inst["xi"] + rng.normal(0, 0.05, size=inst["xi"].shape), requires_grad=True)
    x, l = xi0, lam0
    for _ in range(iters):
        x, l = T(x, l, xi_c)
    loss = (x * torch.tensor(gx_out)).sum() + (l * torch.tensor(gl_out)).sum() + 0.7 * rsq(x)
    loss.backward()
    gx, gx0, gl0 = oracle.solve_backward(inst, iters, gx_out, gl_out, 0.7, rho=RHO,
                                         xi0=xi0.detach().numpy(), lam0=lam0.detach().numpy())
    for got, ref in [(gx, xi_c.grad), (gx0, xi0.grad), (gl0, lam0.grad)]:
        ref = ref.numpy()
        np.testing.assert_allclose(got, ref, atol=1e-10 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("nd", [2, 3])
def test_backward_central_finite_differences(nd):
    """FP64 central differences, eps = 1e-6, along random directions (dot-product test:
    <J v, w> from differences of the forward map equals <v, J'w> from the reverse pass)."""
    iters = 8
    inst = _grad_instance(nd, 40 * nd, iters)
    rng = np.random.default_rng(2)
    w = rng.normal(size=inst["xi"].shape)
    gx, gx0, gl0 = oracle.solve_backward(inst, iters, w, None, 0.0, rho=RHO)
    eps = 1e-6
    for trial in range(3):
        v = rng.normal(size=inst["xi"].shape)
        v[:, :, 0] = 0.0
        v[:, :, -1] = 0.0
        fp = oracle.solve(dict(inst, xi=inst["xi"] + eps * v), iters, rho=RHO)["xi"]
        fm = oracle.solve(dict(inst, xi=inst["xi"] - eps * v), iters, rho=RHO)["xi"]
        jv = (fp - fm) / (2 * eps)
        lhs, rhs = float(np.sum(jv * w)), float(np.sum(v * gx))
        assert abs(lhs - rhs) <= 1e-6 * max(1.0, abs(rhs)), (lhs, rhs)
        # lambda^0 direction
        fp = oracle.solve(inst, iters, rho=RHO, lam0=eps * v)["xi"]
        fm = oracle.solve(inst, iters, rho=RHO, lam0=-eps * v)["xi"]
        lhs, rhs = float(np.sum((fp - fm) / (2 * eps) * w)), float(np.sum(v * gl0))
        assert abs(lhs - rhs) <= 1e-6 * max(1.0, abs(rhs)), (lhs, rhs)


def test_residual_gradient_is_twice_g():
    """||r_p||^2 is the squared distance of (F xi, G xi) to the constraint set in row space,
    so its gradient is 2 (F'r_1 + G'r_2); the reverse pass through the residual seed agrees."""
    inst = _grad_instance(2, 7, 1)
    _, g = oracle.residual(inst, inst["xi"], want_g=True)
    gx, gx0, _ = oracle.solve_backward(inst, 0, None, None, 1.0, rho=RHO)
    np.testing.assert_allclose(gx0, 2 * g, atol=1e-12)


def test_batch_matches_single_instances():
    insts = sfgen.make_batch(2, B=3)
    xs, res = oracle.solve_batch(insts, 20, rho=RHO)
    for inst, x, r in zip(insts, xs, res):
        ref = oracle.solve(inst, 20, rho=RHO)["xi"]
        np.testing.assert_array_equal(x, ref)
        np.testing.assert_allclose(r, oracle.residual(inst, ref)[:2], rtol=0, atol=0)


# ---- endpoint-pinned least-squares fit (candidate helper) -----------------------------

@pytest.mark.parametrize("H,nxi", [(11, 11), (40, 11), (200, 7), (9, 9)])
def test_fit_recovers_representable_curves(H, nxi):
    """Samples of a polynomial of the basis are fitted exactly (zero residual), endpoints included."""
    rng = np.random.default_rng(H + nxi)
    xi = rng.normal(size=(2, 5, nxi)) * 3.0
    pos = np.einsum("kc,dic->dik", oracle.basis(H, nxi), xi)
    assert np.abs(oracle.fit_positions(pos, nxi) - xi).max() <= 1e-9


def test_fit_pins_endpoints_and_is_optimal():
    """Endpoints equal the first and last samples exactly; no interior perturbation lowers
    the squared error (brute force over random directions)."""
    rng = np.random.default_rng(3)
    H, nxi = 50, 11
    pos = rng.normal(size=(3, 4, H)) * 2.0
    xi = oracle.fit_positions(pos, nxi)
    assert np.array_equal(xi[..., 0], pos[..., 0]) and np.array_equal(xi[..., -1], pos[..., -1])
    W = oracle.basis(H, nxi)
    err = lambda x: ((np.einsum("kc,dic->dik", W, x) - pos) ** 2).sum()
    e0 = err(xi)
    for _ in range(200):
        d = np.zeros_like(xi)
        d[..., 1:-1] = rng.normal(size=xi[..., 1:-1].shape) * 10 ** rng.uniform(-6, -1)
        assert err(xi + d) >= e0 - 1e-12 * max(e0, 1.0)


# ---- trajectory optimiser: smoothness cost (eq. cost, eq. eq::form) ------------------------

DT = 0.05


def _q1(H, nxi, dt=DT):
    Wdd = pinlib.bernstein_dd(H, nxi, dt)
    return Wdd.T @ Wdd


@pytest.mark.parametrize("H,nxi,dt", [(20, 6, 0.1), (100, 11, 0.05), (7, 3, 1.0)])
def test_smooth_basis_is_bernstein_second_derivative(H, nxi, dt):
    ref = pinlib.bernstein_dd(H, nxi, dt)
    np.testing.assert_allclose(oracle.basis_dd(H, nxi, dt), ref, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("n,n_obs,H,nxi", [(1, 0, 10, 5), (3, 2, 12, 6), (4, 3, 30, 11)])
def test_smooth_kkt_matches_dense_and_kronecker(n, n_obs, H, nxi):
    """H = (I (x) Wdd'Wdd) + rho F'F + rho G'G; the Kronecker form keeps P_dev / P_mean with
    Q1 + rho c W'W in place of I + rho c W'W."""
    rho = 0.7
    W, F, G, A = pinlib.dense_mats(n, n_obs, H, nxi)
    Q1 = _q1(H, nxi)
    Hm, Pe, Pb = oracle.kkt(2, nxi, rho, n, n_obs, H, cost="smoothness", dt=DT)
    ref = np.kron(np.eye(n), Q1) + rho * F.T @ F + rho * G.T @ G
    np.testing.assert_allclose(Hm, ref, atol=1e-10 * np.abs(ref).max())
    Kinv = np.linalg.inv(np.block([[ref, A.T], [A, np.zeros((2 * n, 2 * n))]]))
    np.testing.assert_allclose(Pe, Kinv[:n * nxi, :n * nxi], atol=1e-9 * np.abs(Kinv).max())
    A0 = np.vstack([W[0], W[-1]])

    def cinv(c):
        Ki = np.linalg.inv(np.block([[Q1 + rho * c * W.T @ W, A0.T], [A0, np.zeros((2, 2))]]))
        return Ki[:nxi, :nxi], Ki[:nxi, nxi:]

    Qn = np.ones((n, n)) / n
    (Pd, Bd), (Pm, Bm) = cinv(n + n_obs + 2), cinv(n_obs + 2)
    np.testing.assert_allclose(Pe, np.kron(np.eye(n) - Qn, Pd) + np.kron(Qn, Pm), atol=1e-9 * np.abs(Pe).max())
    np.testing.assert_allclose(Pb, np.kron(np.eye(n) - Qn, Bd) + np.kron(Qn, Bm), atol=1e-9 * np.abs(Pb).max())


@pytest.mark.parametrize("nd,seed", [(2, 0), (3, 2)])
def test_smooth_one_sweep_is_block_argmin(nd, seed):
    """One sweep of the optimiser equals the independently built block minimisers, with the
    smoothness cost in the xi_bar step and no candidate term."""
    H = 8
    inst = pinlib.small_instance(n=3, n_obs=2, H=H, n_d=nd, n_xi=6, seed=seed)
    rng = np.random.default_rng(200 + seed)
    xib = inst["xi"] + rng.normal(0, 0.3, size=inst["xi"].shape)
    lam = rng.normal(0, 0.2, size=inst["xi"].shape)
    got = oracle.solve(inst, 1, rho=RHO, xi0=xib, lam0=lam, cost="smoothness", dt=DT)
    ref_x, ref_l = pinlib.one_step_reference(inst, xib, lam, RHO, Q1=_q1(H, 6))
    np.testing.assert_allclose(got["lam"], ref_l, atol=1e-8)
    np.testing.assert_allclose(got["xi"], ref_x, atol=1e-8 * max(1.0, np.abs(ref_x).max()))


def test_smooth_unconstrained_optimum_is_the_straight_line():
    """One robot, no obstacles, a box it never touches: the minimum-acceleration trajectory
    between fixed endpoints is the straight line at constant speed, which the basis holds
    exactly as the linear ramp of coefficients."""
    inst = pinlib.small_instance(n=1, n_obs=0, H=30, n_d=2, n_xi=8, seed=5, sigma=0.4, extent=40.0)
    out = oracle.solve(inst, 3000, rho=1.0, cost="smoothness", dt=0.02)
    b = inst["bnd"]
    ramp = b[..., :1] + (b[..., 1:] - b[..., :1]) * np.linspace(0.0, 1.0, 8)
    assert oracle.residual(inst, out["xi"], rho=1.0)[1] == 0.0
    np.testing.assert_allclose(out["xi"], ramp, atol=1e-8)


def test_smooth_backward_matches_torch_autograd():
    import torch
    iters = 5
    inst = _grad_instance(2, 77, iters, False)
    W, F, G, A = pinlib.dense_mats(inst["n"], inst["n_obs"], inst["H"], inst["n_xi"])
    T, rsq = pinlib.torch_T(inst, RHO, W, F, G, A, Q1=_q1(inst["H"], inst["n_xi"]))
    rng = np.random.default_rng(2)
    gx_out = rng.normal(size=inst["xi"].shape)
    gl_out = rng.normal(size=inst["xi"].shape)
    xi_c = torch.tensor(inst["xi"], requires_grad=True)
    lam0 = torch.tensor(rng.normal(0, 0.1, size=inst["xi"].shape), requires_grad=True)
    xi0 = torch.tensor(inst["xi"] + rng.normal(0, 0.05, size=inst["xi"].shape), requires_grad=True)
    x, l = xi0, lam0
    for _ in range(iters):
        x, l = T(x, l, xi_c)
    loss = (x * torch.tensor(gx_out)).sum() + (l * torch.tensor(gl_out)).sum() + 0.7 * rsq(x)
    loss.backward()
    gx, gx0, gl0 = oracle.solve_backward(inst, iters, gx_out, gl_out, 0.7, rho=RHO, xi0=xi0.detach().numpy(),
                                         lam0=lam0.detach().numpy(), cost="smoothness", dt=DT)
    assert xi_c.grad is None or np.abs(xi_c.grad.numpy()).max() == 0.0   # the candidate does not enter
    assert np.abs(gx).max() == 0.0
    for got, ref in [(gx0, xi0.grad), (gl0, lam0.grad)]:
        ref = ref.numpy()
        np.testing.assert_allclose(got, ref, atol=1e-10 * max(1.0, np.abs(ref).max()))


# ---- candidate metrics and selection (the ranking stages of the pipeline) -------------------

def test_metrics_of_a_straight_line_and_a_parabola():
    """A straight line at constant speed has zero smoothness cost and path length
    ||goal - start||; the parabola s + (g - s) tau + c tau (1 - tau) has the constant
    acceleration -2 c / T^2, so its smoothness cost is H 4 ||c||^2 / T^4."""
    H, nxi, dt = 40, 11, 0.05
    T = (H - 1) * dt
    rng = np.random.default_rng(8)
    inst = pinlib.small_instance(n=3, n_obs=0, H=H, n_d=2, n_xi=nxi, seed=3, extent=50.0)
    b = inst["bnd"]
    ramp = b[..., :1] + (b[..., 1:] - b[..., :1]) * np.linspace(0.0, 1.0, nxi)
    m = oracle.metrics(inst, ramp, dt=dt)
    assert abs(m[2]) <= 1e-18 * H
    np.testing.assert_allclose(m[3], np.linalg.norm(b[..., 1] - b[..., 0], axis=0).mean(), rtol=1e-12)
    tau = np.linspace(0.0, 1.0, H)
    c = rng.normal(size=(2, 3)) * 0.5
    pos = b[..., :1] + (b[..., 1:] - b[..., :1]) * tau + c[..., None] * tau * (1.0 - tau)
    xi = oracle.fit_positions(pos, nxi)
    m = oracle.metrics(inst, xi, dt=dt)
    np.testing.assert_allclose(m[2], (H * 4.0 * (c ** 2).sum(axis=0) / T ** 4).mean(), rtol=1e-9)


def test_select_orders_feasible_by_secondary_then_the_rest():
    p = [0.5, 1e-4, np.nan, 2e-4, 3.0, 1e-4]
    q = [9.0, 5.0, 1.0, 4.0, 0.0, 5.0]
    assert oracle.select(p, q, 1e-3, 6) == [3, 1, 5, 0, 4, 2]
    assert oracle.select(p, None, -np.inf, 3) == [1, 5, 3]
    assert oracle.select([1.0, 0.5], None, -np.inf, 4) == [1, 0, -1, -1]


# ------------------------------------------- initial-velocity boundary rows (Sec. V, hardware)
VDT = 0.1   # time step of the velocity rows' time scale


def _vel_instance(cid=1, idx=0, seed=0):
    return sfgen.with_initial_velocity(sfgen.make_batch(cid, B=idx + 1)[idx], seed)


@pytest.mark.parametrize("H,nxi,dt", [(20, 6, 0.1), (50, 11, 0.05)])
def test_velocity_basis_is_bernstein_first_derivative(H, nxi, dt):
    np.testing.assert_allclose(oracle.basis_d(H, nxi, dt), pinlib.bernstein_d(H, nxi, dt), atol=1e-11)


@pytest.mark.parametrize("n,n_obs,H,nxi", [(3, 2, 12, 6), (2, 0, 9, 5)])
def test_velocity_kkt_matches_dense_kkt(n, n_obs, H, nxi):
    """P_eta and P_b with the velocity rows against numpy's solve of the KKT system built
    from the Appendix's matrices with A = I (x) [W_0; W_{H-1}; W'_0]."""
    _, F, G, A = pinlib.dense_mats(n, n_obs, H, nxi, n_bc=3, dt=VDT)
    Hm = np.eye(n * nxi) + RHO * (F.T @ F + G.T @ G)
    K = np.block([[Hm, A.T], [A, np.zeros((A.shape[0], A.shape[0]))]])
    Kinv = np.linalg.inv(K)
    _, Pe, Pb = oracle.kkt(2, nxi, RHO, n, n_obs, H, dt=VDT, n_bc=3)
    N = n * nxi
    np.testing.assert_allclose(Pe, Kinv[:N, :N], atol=1e-11)
    np.testing.assert_allclose(Pb, Kinv[:N, N:], atol=1e-11)


def test_velocity_rows_hold_every_iterate():
    """A xi_bar = b for all three rows per robot and axis after every xi_bar step, the
    velocity row evaluated with scipy's derivative of the basis."""
    inst = _vel_instance()
    tr = oracle.solve(inst, 40, rho=RHO, dt=VDT, traj=True)["traj"]
    wd0 = pinlib.bernstein_d(inst["H"], inst["n_xi"], VDT)[0]
    for x in tr[1:, 0]:
        np.testing.assert_allclose(x[..., 0], inst["bnd"][..., 0], atol=1e-12)
        np.testing.assert_allclose(x[..., -1], inst["bnd"][..., 1], atol=1e-12)
        np.testing.assert_allclose(x @ wd0, inst["bnd"][..., 2], atol=1e-10)


@pytest.mark.parametrize("nd,seed", [(2, 3), (3, 4)])
def test_velocity_one_sweep_is_block_argmin(nd, seed):
    inst = pinlib.small_instance(n=3, n_obs=2, H=12, n_d=nd, n_xi=6, seed=seed)
    inst = sfgen.with_initial_velocity(inst, seed)
    rng = np.random.default_rng(seed)
    xib = inst["xi"] + rng.normal(0, 0.2, size=inst["xi"].shape)
    lam = rng.normal(0, 0.1, size=inst["xi"].shape)
    got = oracle.solve(inst, 1, rho=RHO, xi0=xib, lam0=lam, dt=VDT)
    ref_x, ref_l = pinlib.one_step_reference(inst, xib, lam, RHO, dt=VDT)
    np.testing.assert_allclose(got["lam"], ref_l, atol=1e-8)
    np.testing.assert_allclose(got["xi"], ref_x, atol=1e-8)


def test_velocity_single_robot_affine_projection():
    """1 robot, no obstacles, inside the box: the textbook affine projection onto the three
    boundary rows, xi_bar = xi - A'(AA')^-1 (A xi - b)."""
    nxi, H = 9, 30
    rng = np.random.default_rng(6)
    xi = np.cumsum(rng.normal(0, 0.3, size=(2, 1, nxi)), axis=-1)
    bnd = np.stack([xi[:, :, 0] + 0.4, xi[:, :, -1] - 0.3, np.array([[0.7], [-0.4]])], axis=-1)
    inst = dict(n=1, n_obs=0, H=H, n_d=2, n_xi=nxi, dyn_obs=False, a=0.5, b=0.5,
                pmin=np.full(2, -10.0), pmax=np.full(2, 10.0), obs_c=np.zeros((0, 2)),
                obs_ab=np.zeros((0, 2)), bnd=bnd, xi=xi)
    _, _, _, A = pinlib.dense_mats(1, 0, H, nxi, n_bc=3, dt=VDT)
    ref = np.empty_like(xi)
    for ax in range(2):
        x = xi[ax].ravel()
        ref[ax] = (x - A.T @ np.linalg.solve(A @ A.T, A @ x - bnd[ax].ravel())).reshape(1, nxi)
    got = oracle.solve(inst, 400, rho=RHO, dt=VDT)["xi"]
    np.testing.assert_allclose(got, ref, atol=1e-10)


def _torch_unroll(inst, iters, xi0, lam0, n_bc=2):
    import torch
    W, F, G, A = pinlib.dense_mats(inst["n"], inst["n_obs"], inst["H"], inst["n_xi"], n_bc=n_bc, dt=VDT)
    T, rsq = pinlib.torch_T(inst, RHO, W, F, G, A)
    xi_c = torch.tensor(inst["xi"], requires_grad=True)
    x0 = torch.tensor(xi0, requires_grad=True)
    l0 = torch.tensor(lam0, requires_grad=True)
    zs = [(x0, l0)]
    for _ in range(iters):
        zs.append(T(zs[-1][0], zs[-1][1], xi_c))
    return xi_c, x0, l0, zs, rsq


def test_velocity_backward_matches_torch_autograd():
    import torch
    iters = 5
    base = pinlib.small_instance(n=3, n_obs=2, H=10, n_d=2, n_xi=6, seed=21)
    inst = sfgen.with_initial_velocity(base, 21)
    rng = np.random.default_rng(3)
    g_out = rng.normal(size=inst["xi"].shape)
    xi0 = inst["xi"] + rng.normal(0, 0.05, size=inst["xi"].shape)
    lam0 = rng.normal(0, 0.1, size=inst["xi"].shape)
    xi_c, x0, l0, zs, rsq = _torch_unroll(inst, iters, xi0, lam0, n_bc=3)
    loss = (zs[-1][0] * torch.tensor(g_out)).sum() + 0.4 * rsq(zs[-1][0])
    loss.backward()
    gx, gx0, gl0 = oracle.solve_backward(inst, iters, g_out, None, 0.4, rho=RHO, xi0=xi0, lam0=lam0, dt=VDT)
    for got, ref in [(gx, xi_c.grad), (gx0, x0.grad), (gl0, l0.grad)]:
        ref = ref.numpy()
        np.testing.assert_allclose(got, ref, atol=1e-10 * max(1.0, np.abs(ref).max()))


# ------------------------------------------- self-supervised loss (eq. NN_loss, Fig. unroll)
@pytest.mark.parametrize("nd", [2, 3])
def test_fixed_point_loss_gradient_matches_torch_autograd(nd):
    """The loss of eq. NN_loss, sum_{l<L} ||z^{l+1} - z^l||^2 + ||xi_bar^L - xi||^2 (the
    fixed-point residual read as the step of z = (xi_bar, lambda)), differentiated by
    torch autograd through the unrolled restatement, against the reverse pass with
    g_fp = 1 and g_xi_out = 2 (xi_bar^L - xi) (the candidate's own share of the last term
    added by the caller)."""
    import torch
    iters = 6
    inst = _grad_instance(nd, 70 + nd, iters)
    rng = np.random.default_rng(9)
    xi0 = inst["xi"] + rng.normal(0, 0.05, size=inst["xi"].shape)
    lam0 = rng.normal(0, 0.1, size=inst["xi"].shape)
    xi_c, x0, l0, zs, _ = _torch_unroll(inst, iters, xi0, lam0)
    loss = sum(((zs[l + 1][0] - zs[l][0]) ** 2).sum() + ((zs[l + 1][1] - zs[l][1]) ** 2).sum()
               for l in range(iters))
    loss = loss + ((zs[-1][0] - xi_c) ** 2).sum()
    loss.backward()
    xL = oracle.solve(inst, iters, rho=RHO, xi0=xi0, lam0=lam0)["xi"]
    gx, gx0, gl0 = oracle.solve_backward(inst, iters, 2 * (xL - inst["xi"]), None, 0.0, rho=RHO, xi0=xi0,
                                         lam0=lam0, g_fp=1.0)
    gx = gx - 2 * (xL - inst["xi"])
    for got, ref in [(gx, xi_c.grad), (gx0, x0.grad), (gl0, l0.grad)]:
        ref = ref.numpy()
        np.testing.assert_allclose(got, ref, atol=1e-10 * max(1.0, np.abs(ref).max()))


def test_fixed_point_loss_central_differences():
    """Dot-product test of the fixed-point term alone: <grad, v> against central
    differences (eps = 1e-6) of sum_l ||z^{l+1} - z^l||^2 along lambda^0 and xi_bar^0."""
    iters = 7
    inst = _grad_instance(2, 90, iters)
    rng = np.random.default_rng(4)

    def loss(xi0, lam0):
        tr = oracle.solve(inst, iters, rho=RHO, xi0=xi0, lam0=lam0, traj=True)["traj"]
        return float(np.sum(np.diff(tr, axis=0) ** 2))

    xi0 = inst["xi"].copy()
    lam0 = np.zeros_like(xi0)
    _, gx0, gl0 = oracle.solve_backward(inst, iters, None, None, 0.0, rho=RHO, xi0=xi0, lam0=lam0, g_fp=1.0)
    eps = 1e-6
    for _ in range(2):
        v = rng.normal(size=xi0.shape)
        lhs = (loss(xi0 + eps * v, lam0) - loss(xi0 - eps * v, lam0)) / (2 * eps)
        assert abs(lhs - float(np.sum(v * gx0))) <= 1e-6 * max(1.0, abs(lhs))
        lhs = (loss(xi0, lam0 + eps * v) - loss(xi0, lam0 - eps * v)) / (2 * eps)
        assert abs(lhs - float(np.sum(v * gl0))) <= 1e-6 * max(1.0, abs(lhs))
