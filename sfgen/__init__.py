"""Seeded synthetic Safety-Filter (SF) instances.

This module is shared by the CPU oracle's tests, the CUDA path's tests and the
benchmark.  It draws random numbers and lays out geometry; it holds none of the
SF method's arithmetic (no basis evaluation, no constraint rows, no solver step).

Every instance is a dict of float64 numpy arrays:

  n, n_obs, H, n_d, n_xi        sizes (robots, obstacles, timesteps K+1, workspace
                                dimension, polynomial coefficients per robot per axis)
  a, b                          robot spheroid axes: M_r = diag(a, a, b)  (Sec. III-A)
  pmin, pmax  [n_d]             workspace box, already inset by the robot radius
  obs_c       [n_obs][n_d]      static obstacle centres
              or [n_obs][H][n_d] when dyn_obs is true (per-timestep centres)
  obs_ab      [n_obs][2]        obstacle axes (a_o, b_o), inflated by the robot radius
  bnd         [n_d][n][2]       boundary values (start, goal) per axis and robot, or
              [n_d][n][3]       (start, goal, initial velocity in m/s) with initial-velocity rows
  xi          [n_d][n][n_xi]    candidate coefficients, axis-major (Sec. III-A, coefficient stacking)

Candidates are written directly in coefficient space.  The trajectory basis is
the Bernstein basis, whose coefficients form a control polygon: the straight
start->goal line is the linear ramp of control points, and the first and last
coefficients are the start and goal.  Noise is added to the interior control
points only, so every candidate meets the boundary equalities exactly.

Seeds: numpy PCG64 with seed = 1000 * config_id + instance_index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

N_XI_DEFAULT = 11


@dataclass(frozen=True)
class SFConfig:
    """One benchmark configuration (map, robots, obstacles, candidate noise)."""
    cid: int
    name: str
    B: int
    n: tuple            # robot count: (lo, hi) inclusive, uniform integer
    n_obs: tuple        # obstacle count: (lo, hi) inclusive
    H: tuple            # horizon choices
    n_d: int
    r_robot: float
    extent: tuple       # map size per axis, metres (box centred at the origin)
    r_obs: tuple        # obstacle radius U[lo, hi]
    noise: str          # "iid" or "gp"
    sigma: float
    ell: float = 10.0   # GP lengthscale in timesteps
    iters: int = 100
    min_sep: float = 0.8
    precision: str = "fp32"
    extra: dict = field(default_factory=dict)


def _load_configs():
    """The workloads of configs.json as SFConfig records, keyed by config id."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs.json")) as f:
        spec = json.load(f)
    out = {}
    for c in spec["configs"]:
        out[c["cid"]] = SFConfig(c["cid"], c["name"], c["B"], tuple(c["n"]), tuple(c["n_obs"]), tuple(c["H"]),
                                 c["n_d"], c["r_robot"], tuple(c["extent"]), tuple(c["r_obs"]), c["noise"],
                                 c["sigma"], ell=c.get("ell", 10.0), iters=c["iters"],
                                 precision=c.get("precision", "fp32"), extra=dict(c.get("extra", {})))
    return out, spec["solver"]


CONFIGS, SOLVER_DEFAULTS = _load_configs()


def rng_for(cid: int, idx: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * cid + idx))


def _sample_separated(rng, n, lo, hi, min_sep, max_tries=200000):
    """n points uniform in the box [lo, hi] with pairwise distance >= min_sep."""
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d separated points" % n)
        q = rng.uniform(lo, hi)
        if all(np.linalg.norm(q - p) >= min_sep for p in pts):
            pts.append(q)
    return np.array(pts)


def _gp_noise(rng, n_xi, H, sigma, ell_steps, n_series):
    """Squared-exponential GP samples over the interior control points.

    Control point c sits at time fraction c/(n_xi-1), i.e. at timestep
    c (H-1)/(n_xi-1); the lengthscale in timesteps is converted accordingly.
    The linear interpolant of the two endpoint values is subtracted so the
    endpoints carry no noise.  Returns [n_series][n_xi].
    """
    t = np.arange(n_xi) * (H - 1) / (n_xi - 1)
    K = sigma ** 2 * np.exp(-0.5 * (t[:, None] - t[None, :]) ** 2 / ell_steps ** 2)
    L = np.linalg.cholesky(K + 1e-10 * np.eye(n_xi))
    z = rng.standard_normal((n_series, n_xi)) @ L.T
    ramp = np.arange(n_xi) / (n_xi - 1)
    z = z - (z[:, :1] * (1 - ramp) + z[:, -1:] * ramp)
    z[:, 0] = 0.0
    z[:, -1] = 0.0
    return z


def make_instance(cfg: SFConfig, idx: int, n_xi: int = N_XI_DEFAULT, dyn_obs: bool = False):
    rng = rng_for(cfg.cid, idx)
    n = int(rng.integers(cfg.n[0], cfg.n[1] + 1))
    n_obs = int(rng.integers(cfg.n_obs[0], cfg.n_obs[1] + 1))
    H = int(cfg.H[int(rng.integers(0, len(cfg.H)))])
    nd = cfg.n_d
    half = np.array(cfg.extent[:nd]) / 2.0
    r = cfg.r_robot
    pmin = -half + r
    pmax = half - r
    starts = _sample_separated(rng, n, pmin, pmax, cfg.min_sep)
    goals = _sample_separated(rng, n, pmin, pmax, cfg.min_sep)
    ends = np.concatenate([starts, goals])
    obs_c, obs_r = [], []
    while len(obs_c) < n_obs:
        c = rng.uniform(-half, half)
        ro = rng.uniform(cfg.r_obs[0], cfg.r_obs[1])
        if np.all(np.linalg.norm(ends - c, axis=1) > ro + r):
            obs_c.append(c)
            obs_r.append(ro)
    obs_c = np.array(obs_c).reshape(n_obs, nd)
    obs_r = np.array(obs_r)
    ramp = np.arange(n_xi) / (n_xi - 1)
    xi = np.empty((nd, n, n_xi))
    for ax in range(nd):
        xi[ax] = starts[:, ax:ax + 1] * (1 - ramp) + goals[:, ax:ax + 1] * ramp
    if cfg.noise == "iid":
        noise = rng.normal(0.0, cfg.sigma, size=(nd, n, n_xi))
        noise[:, :, 0] = 0.0
        noise[:, :, -1] = 0.0
    else:
        noise = _gp_noise(rng, n_xi, H, cfg.sigma, cfg.ell, nd * n).reshape(nd, n, n_xi)
    xi = xi + noise
    bnd = np.stack([starts.T, goals.T], axis=-1)  # [nd][n][2]
    if dyn_obs:
        # straight-line obstacle motion, constant velocity up to 0.5 m over the horizon
        vel = rng.uniform(-0.5, 0.5, size=(n_obs, nd))
        frac = np.arange(H) / max(H - 1, 1)
        obs_c = obs_c[:, None, :] + frac[None, :, None] * vel[:, None, :]
    return dict(
        n=n, n_obs=n_obs, H=H, n_d=nd, n_xi=n_xi, dyn_obs=bool(dyn_obs),
        a=2.0 * r, b=2.0 * r, pmin=pmin, pmax=pmax,
        obs_c=np.ascontiguousarray(obs_c, dtype=np.float64),
        obs_ab=np.stack([obs_r + r, obs_r + r], axis=1),
        bnd=np.ascontiguousarray(bnd), xi=np.ascontiguousarray(xi),
    )


def make_batch(cid: int, B: int | None = None, n_xi: int = N_XI_DEFAULT, start: int = 0,
               dyn_obs: bool = False):
    cfg = CONFIGS[cid]
    B = cfg.B if B is None else B
    return [make_instance(cfg, start + i, n_xi=n_xi, dyn_obs=dyn_obs) for i in range(B)]


def custom_instance(n, n_obs, H, n_d=2, n_xi=N_XI_DEFAULT, seed=0, extent=10.0, r_robot=0.25,
                    r_obs=(0.3, 0.6), noise="iid", sigma=0.5, ell=10.0, dyn_obs=False,
                    min_sep=0.8):
    """An instance of arbitrary size drawn with the config-1 style generators."""
    cfg = SFConfig(900 + seed, "custom", 1, (n, n), (n_obs, n_obs), (H,), n_d, r_robot,
                   (extent,) * n_d if np.isscalar(extent) else tuple(extent), r_obs, noise,
                   sigma, ell=ell, min_sep=min_sep)
    return make_instance(cfg, 0, n_xi=n_xi, dyn_obs=dyn_obs)


def with_initial_velocity(inst, seed, vmax=0.5):
    """A copy of ``inst`` with an initial velocity per robot and axis, uniform in
    [-vmax, vmax] m/s (seeded), appended to the boundary values: bnd becomes
    [n_d][n][3] = (start, goal, v_0).  The candidate is left as it is."""
    rng = np.random.Generator(np.random.PCG64(7919 + seed))
    v0 = rng.uniform(-vmax, vmax, size=inst["bnd"].shape[:2])
    out = dict(inst)
    out["bnd"] = np.ascontiguousarray(np.concatenate([inst["bnd"][..., :2], v0[..., None]], axis=-1))
    return out


def batch_stats(insts):
    """Counts of pair-timestep and robot-obstacle-timestep rows per iteration."""
    pairs = sum(i["n"] * (i["n"] - 1) // 2 * i["H"] for i in insts)
    obs = sum(i["n"] * i["n_obs"] * i["H"] for i in insts)
    return pairs, obs


__all__ = ["CONFIGS", "SFConfig", "make_instance", "make_batch", "custom_instance",
           "with_initial_velocity", "batch_stats", "rng_for", "N_XI_DEFAULT"]
