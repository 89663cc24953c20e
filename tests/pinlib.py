"""Independent constructions used to pin the oracle (and, through it, the CUDA path).

Nothing here calls the oracle's arithmetic: the basis comes from scipy's
Bernstein evaluator, the constraint matrices are assembled with Kronecker
products exactly as the paper's Appendix writes them (F_r = [F_r,1; ...] (x) W,
F_o = blockdiag(stack W)), row projections come from brute-force search, and
linear systems are solved with numpy's dense solver.
"""
from __future__ import annotations

import numpy as np
import scipy.interpolate as si
import scipy.optimize as so


def bernstein(H, n_xi):
    """W[k, c] = c-th Bernstein polynomial of degree n_xi-1 at k/(H-1), via scipy.BPoly."""
    tau = np.linspace(0.0, 1.0, H)
    cols = [si.BPoly(np.eye(n_xi)[c][:, None], [0.0, 1.0])(tau) for c in range(n_xi)]
    return np.stack(cols, axis=1)


def bernstein_dd(H, n_xi, dt):
    """Second time derivative of the Bernstein basis at t_k = k dt on [0, (H-1) dt], via
    scipy.BPoly.derivative (smoothness cost of the trajectory optimiser)."""
    T = (H - 1) * dt
    t = np.linspace(0.0, T, H)
    cols = [si.BPoly(np.eye(n_xi)[c][:, None], [0.0, T]).derivative(2)(t) for c in range(n_xi)]
    return np.stack(cols, axis=1)


def bernstein_d(H, n_xi, dt):
    """First time derivative of the Bernstein basis at t_k = k dt on [0, (H-1) dt], via
    scipy.BPoly.derivative (initial-velocity boundary rows)."""
    T = (H - 1) * dt
    t = np.linspace(0.0, T, H)
    cols = [si.BPoly(np.eye(n_xi)[c][:, None], [0.0, T]).derivative(1)(t) for c in range(n_xi)]
    return np.stack(cols, axis=1)


def incidence(n):
    """Stacked F_{r,i} = [F_i, -I] of the Appendix: row (i, j>i) is e_i - e_j."""
    rows = []
    for i in range(n):
        Fi = np.zeros((n - i - 1, i + 1))
        Fi[:, i] = 1.0
        rows.append(np.hstack([Fi, -np.eye(n - i - 1)]))
    return np.vstack(rows) if rows else np.zeros((0, n))


def dense_mats(n, n_obs, H, n_xi, n_bc=2, dt=0.1):
    """Per-axis F (pair rows then obstacle rows), G, A for one instance.  A's rows per robot:
    start W[0], goal W[H-1] and, with n_bc = 3, the initial velocity p'(0) (time t = tau (H-1) dt)."""
    W = bernstein(H, n_xi)
    Fr = np.kron(incidence(n), W)
    Fo = np.kron(np.eye(n), np.vstack([W] * n_obs)) if n_obs else np.zeros((0, n * n_xi))
    F = np.vstack([Fr, Fo])
    G = np.vstack([np.kron(np.eye(n), W), -np.kron(np.eye(n), W)])
    rows = [W[0], W[-1]] + ([bernstein_d(H, n_xi, dt)[0]] if n_bc == 3 else [])
    A = np.kron(np.eye(n), np.vstack(rows))
    return W, F, G, A


def row_centres(inst):
    """Per-axis offsets of every F row: 0 for pair rows, the obstacle centre for obstacle rows."""
    n, n_obs, H, nd = inst["n"], inst["n_obs"], inst["H"], inst["n_d"]
    npair = n * (n - 1) // 2
    c = np.zeros((nd, npair * H + n * n_obs * H))
    radius = np.full(c.shape[1], inst["a"])
    for i in range(n):
        for m in range(n_obs):
            base = npair * H + (i * n_obs + m) * H
            for k in range(H):
                oc = inst["obs_c"][m, k] if inst.get("dyn_obs") else inst["obs_c"][m]
                c[:, base + k] = oc
            radius[base:base + H] = inst["obs_ab"][m, 0]
    return c, radius


def exterior_projection_bruteforce(delta, a):
    """argmin_{||e|| >= a} ||delta - e|| by a direction search (grid, then local refinement).

    For a fixed unit direction u the best admissible length is max(a, <delta, u>);
    the search runs over u only.
    """
    delta = np.asarray(delta, dtype=np.float64)
    nd = delta.size

    def cost_dir(ang):
        if nd == 2:
            u = np.array([np.cos(ang[0]), np.sin(ang[0])])
        else:
            u = np.array([np.cos(ang[0]) * np.sin(ang[1]), np.sin(ang[0]) * np.sin(ang[1]), np.cos(ang[1])])
        r = max(a, float(delta @ u))
        return float(np.sum((delta - r * u) ** 2)), r * u

    if nd == 2:
        grid = [(t,) for t in np.linspace(-np.pi, np.pi, 721)]
    else:
        grid = [(t, p) for t in np.linspace(-np.pi, np.pi, 121) for p in np.linspace(0, np.pi, 61)]
    best = min(grid, key=lambda g: cost_dir(g)[0])
    res = so.minimize(lambda g: cost_dir(g)[0], np.array(best), method="Nelder-Mead",
                      options=dict(xatol=1e-13, fatol=1e-26, maxiter=4000))
    return cost_dir(res.x)[1]


def one_step_reference(inst, xib, lam, rho, ws_hess=True, Q1=None, dt=0.1):
    """One AM sweep (alpha, beta, d, s, lambda, xi_bar) built from the augmented Lagrangian.

    Isotropic robots and obstacles only: the joint (alpha, beta, d) minimiser of
    rho/2 ||F xi_bar - e||^2 over the spherical form is then the projection onto the
    exterior of the ball, found by brute force row by row.
    """
    n, n_obs, H, nd, n_xi = inst["n"], inst["n_obs"], inst["H"], inst["n_d"], inst["n_xi"]
    W, F, G, A = dense_mats(n, n_obs, H, n_xi, inst["bnd"].shape[-1], dt)
    cen, rad = row_centres(inst)
    y = np.stack([F @ xib[ax].ravel() for ax in range(nd)])
    e = np.empty_like(y)
    for r in range(y.shape[1]):
        e[:, r] = cen[:, r] + exterior_projection_bruteforce(y[:, r] - cen[:, r], rad[r])
    xi_new = np.empty_like(xib)
    lam_new = np.empty_like(lam)
    for ax in range(nd):
        q = G @ xib[ax].ravel()
        h = np.concatenate([np.full(n * H, inst["pmax"][ax]), np.full(n * H, -inst["pmin"][ax])])
        s = np.maximum(0.0, h - q)  # argmin_{s>=0} (q - h + s)^2
        r1 = y[ax] - e[ax]
        r2 = q - h + s
        lam_new[ax] = (lam[ax].ravel() - rho * F.T @ r1 - rho * G.T @ r2).reshape(n, n_xi)
        # cost: 1/2 ||xi_bar - xi||^2, or with Q1 the smoothness cost 1/2 xi_bar' (I (x) Q1) xi_bar
        C = np.eye(n * n_xi) if Q1 is None else np.kron(np.eye(n), Q1)
        Hm = C + rho * F.T @ F + (rho * G.T @ G if ws_hess else 0.0)
        lin = (inst["xi"][ax].ravel() if Q1 is None else 0.0) + lam_new[ax].ravel() + rho * F.T @ e[ax]
        if ws_hess:
            lin = lin + rho * G.T @ (h - s)
        b = inst["bnd"][ax].reshape(-1)  # (start, goal[, v_0]) per robot, robot-major
        K = np.block([[Hm, A.T], [A, np.zeros((A.shape[0], A.shape[0]))]])
        sol = np.linalg.solve(K, np.concatenate([lin, b]))
        xi_new[ax] = sol[:n * n_xi].reshape(n, n_xi)
    return xi_new, lam_new


def projection_bruteforce(inst):
    """min 1/2 ||xi_bar - xi||^2 s.t. A xi_bar = b, box, pair and obstacle separations,
    by SLSQP on the interior coefficients (the equalities fix the end coefficients)."""
    n, n_obs, H, nd, n_xi = inst["n"], inst["n_obs"], inst["H"], inst["n_d"], inst["n_xi"]
    W = bernstein(H, n_xi)
    xi = inst["xi"]

    def full(z):
        X = xi.copy()
        X[:, :, 1:-1] = z.reshape(nd, n, n_xi - 2)
        X[:, :, 0] = inst["bnd"][:, :, 0]
        X[:, :, -1] = inst["bnd"][:, :, 1]
        return X

    def f(z):
        return 0.5 * np.sum((full(z) - xi) ** 2)

    def cons(z):
        P = np.einsum("kc,dic->dik", W, full(z))
        out = []
        for i in range(n):
            for j in range(i + 1, n):
                out.append(np.sum((P[:, i] - P[:, j]) ** 2, axis=0) - inst["a"] ** 2)
            for m in range(n_obs):
                out.append(np.sum((P[:, i] - inst["obs_c"][m][:, None]) ** 2, axis=0)
                           - inst["obs_ab"][m, 0] ** 2)
            out.append((inst["pmax"][:, None] - P[:, i]).ravel())
            out.append((P[:, i] - inst["pmin"][:, None]).ravel())
        return np.concatenate(out)

    res = so.minimize(f, xi[:, :, 1:-1].ravel(), method="SLSQP",
                      constraints=[dict(type="ineq", fun=cons)],
                      options=dict(ftol=1e-15, maxiter=3000))
    return full(res.x), res


def torch_T(inst, rho, W, F, G, A, Q1=None):
    """Differentiable float64 PyTorch restatement of T (trig closed forms), for gradient pins.
    Q1: the per-robot smoothness Hessian block (trajectory-optimiser cost) instead of the
    projection cost."""
    import torch

    n, n_obs, H, nd, n_xi = inst["n"], inst["n_obs"], inst["H"], inst["n_d"], inst["n_xi"]
    cen, _ = row_centres(inst)
    tt = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64)
    Ft, Gt, At = tt(F), tt(G), tt(A)
    cen_t = tt(cen)
    npair = n * (n - 1) // 2
    Arad = np.full(F.shape[0], inst["a"])
    Brad = np.full(F.shape[0], inst["b"])
    for i in range(n):
        for m in range(n_obs):
            base = npair * H + (i * n_obs + m) * H
            Arad[base:base + H] = inst["obs_ab"][m, 0]
            Brad[base:base + H] = inst["obs_ab"][m, 1]
    Ar, Br = tt(Arad), tt(Brad)
    h = [torch.cat([torch.full((n * H,), float(inst["pmax"][ax]), dtype=torch.float64),
                    torch.full((n * H,), float(-inst["pmin"][ax]), dtype=torch.float64)]) for ax in range(nd)]
    Cm = torch.eye(n * n_xi, dtype=torch.float64) if Q1 is None else tt(np.kron(np.eye(n), Q1))
    Hm = Cm + rho * Ft.T @ Ft + rho * Gt.T @ Gt
    K = torch.cat([torch.cat([Hm, At.T], 1), torch.cat([At, torch.zeros(A.shape[0], A.shape[0], dtype=torch.float64)], 1)], 0)

    def estep(D):
        dx, dy = D[0], D[1]
        al = torch.atan2(dy, dx)
        w = dx * torch.cos(al) + dy * torch.sin(al)
        if nd == 3:
            dz = D[2]
            be = torch.atan2(w / Ar, dz / Br)
            sb, cb = torch.sin(be), torch.cos(be)
            t = (Ar * sb * w + Br * cb * dz) / (Ar ** 2 * sb ** 2 + Br ** 2 * cb ** 2)
        else:
            sb, cb = torch.ones_like(w), torch.zeros_like(w)
            t = w / Ar
        d = torch.clamp(t, min=1.0)
        out = [d * Ar * torch.cos(al) * sb, d * Ar * torch.sin(al) * sb]
        if nd == 3:
            out.append(d * Br * cb)
        return torch.stack(out)

    def residual_sq(xib):
        y = torch.stack([Ft @ xib[ax].reshape(-1) for ax in range(nd)])
        e = cen_t + estep(y - cen_t)
        tot = ((y - e) ** 2).sum()
        for ax in range(nd):
            q = Gt @ xib[ax].reshape(-1)
            tot = tot + (torch.clamp(q - h[ax], min=0.0) ** 2).sum()
        return tot

    def T(xib, lam, xi_c):
        y = torch.stack([Ft @ xib[ax].reshape(-1) for ax in range(nd)])
        e = cen_t + estep(y - cen_t)
        xs, ls = [], []
        for ax in range(nd):
            q = Gt @ xib[ax].reshape(-1)
            s = torch.clamp(h[ax] - q, min=0.0)
            r1 = y[ax] - e[ax]
            r2 = q - h[ax] + s
            ln = lam[ax].reshape(-1) - rho * Ft.T @ r1 - rho * Gt.T @ r2
            lin = xi_c[ax].reshape(-1) if Q1 is None else 0.0
            eta = lin + ln + rho * Ft.T @ e[ax] + rho * Gt.T @ (h[ax] - s)
            bb = tt(inst["bnd"][ax].reshape(-1))
            sol = torch.linalg.solve(K, torch.cat([eta, bb]))
            xs.append(sol[:n * n_xi].reshape(n, n_xi))
            ls.append(ln.reshape(n, n_xi))
        return torch.stack(xs), torch.stack(ls)

    return T, residual_sq


def small_instance(n=3, n_obs=2, H=12, n_d=2, n_xi=6, seed=0, sigma=0.6, extent=4.0, aniso=False):
    """A small random instance with conflicts, for gradient and step pins."""
    rng = np.random.default_rng(seed)
    half = extent / 2
    r = 0.3
    pmin, pmax = np.full(n_d, -half + r), np.full(n_d, half - r)
    starts = rng.uniform(pmin, pmax, size=(n, n_d))
    goals = rng.uniform(pmin, pmax, size=(n, n_d))
    ramp = np.arange(n_xi) / (n_xi - 1)
    xi = starts.T[:, :, None] * (1 - ramp) + goals.T[:, :, None] * ramp
    xi[:, :, 1:-1] += rng.normal(0, sigma, size=(n_d, n, n_xi - 2))
    obs_c = rng.uniform(-half, half, size=(n_obs, n_d))
    ro = rng.uniform(0.3, 0.6, size=n_obs)
    ab = np.stack([ro + r, (ro + r) * (1.3 if aniso else 1.0)], axis=1)
    return dict(n=n, n_obs=n_obs, H=H, n_d=n_d, n_xi=n_xi, dyn_obs=False, a=2 * r,
                b=2 * r * (0.7 if aniso else 1.0), pmin=pmin, pmax=pmax, obs_c=obs_c, obs_ab=ab,
                bnd=np.stack([starts.T, goals.T], axis=-1).copy(), xi=np.ascontiguousarray(xi))
