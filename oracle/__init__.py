"""Python access to the plain FP64 SF oracle (``sf_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product package never imports
it.  It shares no code with the CUDA path; both sides read the same seeded
instances from ``sfgen``.

Instances are the dicts produced by ``sfgen`` (see its docstring for the layout).
All arrays are float64, axis-major ``[n_d][n][n_xi]`` for coefficients.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sf_oracle.c")
_LIB = os.path.join(_HERE, "libsforacle.so")
_lock = threading.Lock()
_lib = None

NHIST = 4  # per-iteration history columns: ||r_p||, max residual, FP residual, kink margin
DEFAULT_RHO = 1.0


def build(force: bool = False, src: str = _SRC, out: str = _LIB, extra=()):
    """Compile the oracle with gcc (plain -O2, OpenMP over instances)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o", out, src, "-lm",
               *extra]
        subprocess.check_call(cmd)
    return out


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` selects another build."""
    global _lib
    if path is not None:
        return _declare(ct.CDLL(path))
    with _lock:
        if _lib is None:
            alt = os.environ.get("SF_ORACLE_LIB")  # a mutant build, planted by the pin tests
            if alt:
                _lib = _declare(ct.CDLL(alt))
            else:
                build()
                _lib = _declare(ct.CDLL(_LIB))
    return _lib


_D = ct.POINTER(ct.c_double)
_I = ct.POINTER(ct.c_int)
_LL = ct.POINTER(ct.c_longlong)


def _declare(lib):
    i, d = ct.c_int, ct.c_double
    lib.sfo_basis.argtypes = [i, i, _D]
    lib.sfo_basis_dd.argtypes = [i, i, d, _D]
    lib.sfo_basis_d.argtypes = [i, i, d, _D]
    lib.sfo_estep.argtypes = [i, _D, d, d, _D, _D]
    lib.sfo_kkt.argtypes = [i, i, d, i, i, i, i, i, d, i, _D, _D, _D]
    lib.sfo_residual.argtypes = [i, i, d, i, i, i, i, d, d, _D, _D, _D, _D, _D, _D, _D]
    lib.sfo_solve.argtypes = [i, i, d, i, i, i, i, d, d, _D, _D, _D, _D, _D, _D, _D, _D, i, i, i, d, i,
                              _D, _D, _D, _D]
    lib.sfo_solve_backward.argtypes = [i, i, d, i, i, i, i, d, d, _D, _D, _D, _D, _D, _D, _D, _D,
                                       i, i, i, d, i, _D, _D, d, d, _D, _D, _D]
    lib.sfo_solve_batch.argtypes = [i, i, i, d, _I, _D, _D, _D, _LL, _D, _LL, _D, _LL, _D, _LL,
                                    i, i, i, d, i, _D, _D, _D]
    for f in ("sfo_basis", "sfo_basis_dd", "sfo_basis_d", "sfo_estep", "sfo_kkt", "sfo_residual", "sfo_solve",
              "sfo_solve_backward", "sfo_solve_batch"):
        getattr(lib, f).restype = ct.c_int
    return lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _c(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def basis(H, n_xi, lib=None):
    lib = lib or load()
    W = np.empty((H, n_xi))
    _check(lib.sfo_basis(H, n_xi, _p(W)), "basis")
    return W


def estep(delta, A, Bz, lib=None):
    """Closed-form alpha/beta/d step of one row: (e, J = de/d delta)."""
    lib = lib or load()
    delta = _c(delta)
    nd = delta.shape[0]
    e = np.empty(nd)
    J = np.empty((nd, nd))
    _check(lib.sfo_estep(nd, _p(delta), A, Bz, _p(e), _p(J)), "estep")
    return e, J


COSTS = {"projection": 0, "smoothness": 1}
DEFAULT_DT = 0.1   # time step of the smoothness cost (reading R13)


def basis_dd(H, n_xi, dt=DEFAULT_DT, lib=None):
    """Second time derivative of the basis, t = tau (H - 1) dt (smoothness cost)."""
    lib = lib or load()
    W = np.empty((H, n_xi))
    _check(lib.sfo_basis_dd(H, n_xi, float(dt), _p(W)), "basis_dd")
    return W


def basis_d(H, n_xi, dt=DEFAULT_DT, lib=None):
    """First time derivative of the basis, t = tau (H - 1) dt (initial-velocity rows)."""
    lib = lib or load()
    W = np.empty((H, n_xi))
    _check(lib.sfo_basis_d(H, n_xi, float(dt), _p(W)), "basis_d")
    return W


def kkt(n_d, n_xi, rho, n, n_obs, H, ws_hess=True, cost="projection", dt=DEFAULT_DT, n_bc=2, lib=None):
    """Explicit per-axis Hessian, P_eta and P_b of the xi_bar step (P_b columns robot-major:
    start, goal[, initial velocity])."""
    lib = lib or load()
    N = n * n_xi
    Hm = np.empty((N, N))
    Pe = np.empty((N, N))
    Pb = np.empty((N, n_bc * n))
    _check(lib.sfo_kkt(n_d, n_xi, rho, n, n_obs, H, int(ws_hess), COSTS[cost], float(dt), int(n_bc), _p(Hm),
                       _p(Pe), _p(Pb)), "kkt")
    return Hm, Pe, Pb


def n_bc(inst):
    """Boundary rows per robot and axis: 2 (start, goal) or 3 (with the initial velocity),
    the last extent of the instance's boundary array."""
    return int(np.shape(inst["bnd"])[-1])


def _inst_args(inst, rho):
    return (int(inst["n_d"]), int(inst["n_xi"]), float(rho), int(inst["n"]), int(inst["n_obs"]),
            int(inst["H"]), int(bool(inst.get("dyn_obs", False))), float(inst["a"]), float(inst["b"]))


def _geom(inst):
    pmin, pmax = _c(inst["pmin"]), _c(inst["pmax"])
    obs_c = _c(inst["obs_c"]) if inst["n_obs"] else np.zeros(1)
    obs_ab = _c(inst["obs_ab"]) if inst["n_obs"] else np.zeros(2)
    return pmin, pmax, obs_c, obs_ab


def residual(inst, xi_bar, rho=DEFAULT_RHO, want_g=False, lib=None):
    """(||r_p||, max residual in m, kink margin) of xi_bar, and optionally F'r1 + G'r2."""
    lib = lib or load()
    pmin, pmax, obs_c, obs_ab = _geom(inst)
    xi_bar = _c(xi_bar)
    out = np.empty(3)
    g = np.empty_like(xi_bar) if want_g else None
    _check(lib.sfo_residual(*_inst_args(inst, rho), _p(pmin), _p(pmax), _p(obs_c), _p(obs_ab),
                            _p(xi_bar), _p(out), _p(g)), "residual")
    return (out, g) if want_g else out


def solve(inst, iters, rho=DEFAULT_RHO, xi0=None, lam0=None, ws_hess=True, hist=False,
          traj=False, cost="projection", dt=DEFAULT_DT, lib=None):
    """Run ``iters`` SF iterations; returns dict(xi, lam[, hist][, traj]).  cost="smoothness"
    runs the trajectory optimiser (smoothness cost) instead of the projection."""
    lib = lib or load()
    pmin, pmax, obs_c, obs_ab = _geom(inst)
    xi = _c(inst["xi"])
    xi0, lam0 = _c(xi0), _c(lam0)
    xo = np.empty_like(xi)
    lo = np.empty_like(xi)
    h = np.empty((iters, NHIST)) if hist else None
    tr = np.empty((iters + 1, 2) + xi.shape) if traj else None
    _check(lib.sfo_solve(*_inst_args(inst, rho), _p(pmin), _p(pmax), _p(obs_c), _p(obs_ab),
                         _p(_c(inst["bnd"])), _p(xi), _p(xi0), _p(lam0), int(iters), int(ws_hess),
                         COSTS[cost], float(dt), n_bc(inst), _p(xo), _p(lo), _p(h), _p(tr)), "solve")
    out = dict(xi=xo, lam=lo)
    if hist:
        out["hist"] = h
    if traj:
        out["traj"] = tr
    return out


def solve_backward(inst, iters, g_xi_out=None, g_lam_out=None, g_rp2=0.0, rho=DEFAULT_RHO,
                   xi0=None, lam0=None, ws_hess=True, cost="projection", dt=DEFAULT_DT, g_fp=0.0, lib=None):
    """Reverse mode through ``iters`` SF iterations: (g_xi_cand, g_xi0, g_lam0).  Seeds: the
    outputs' cotangents, g_rp2 (weight of ||r_p(xi_out)||^2) and g_fp (weight of the
    self-supervised fixed-point term sum_l ||z^{l+1} - z^l||^2 of eq. NN_loss)."""
    lib = lib or load()
    pmin, pmax, obs_c, obs_ab = _geom(inst)
    xi = _c(inst["xi"])
    gx, gx0, gl0 = np.empty_like(xi), np.empty_like(xi), np.empty_like(xi)
    _check(lib.sfo_solve_backward(*_inst_args(inst, rho), _p(pmin), _p(pmax), _p(obs_c),
                                  _p(obs_ab), _p(_c(inst["bnd"])), _p(xi), _p(_c(xi0)),
                                  _p(_c(lam0)), int(iters), int(ws_hess), COSTS[cost], float(dt),
                                  n_bc(inst), _p(_c(g_xi_out)),
                                  _p(_c(g_lam_out)), float(g_rp2), float(g_fp), _p(gx), _p(gx0), _p(gl0)),
           "solve_backward")
    return gx, gx0, gl0


def solve_batch(insts, iters, rho=DEFAULT_RHO, ws_hess=True, threads=None, cost="projection",
                dt=DEFAULT_DT, lib=None):
    """All instances at once (OpenMP over instances).  Returns (xi list, resid [B,2])."""
    lib = lib or load()
    if threads is not None:
        os.environ["OMP_NUM_THREADS"] = str(threads)
    B = len(insts)
    nd, nxi = int(insts[0]["n_d"]), int(insts[0]["n_xi"])
    shp = np.array([[i["n"], i["n_obs"], i["H"], int(bool(i.get("dyn_obs", False)))] for i in insts],
                   dtype=np.int32)
    ab = np.array([[i["a"], i["b"]] for i in insts], dtype=np.float64)
    box = np.zeros((B, 6))
    for k, i in enumerate(insts):
        box[k, :nd] = i["pmin"]
        box[k, 3:3 + nd] = i["pmax"]

    def pack(key, fallback):
        parts = [(_c(i[key]).ravel() if i["n_obs"] or key not in ("obs_c", "obs_ab")
                  else np.zeros(fallback)) for i in insts]
        off = np.zeros(B, dtype=np.int64)
        off[1:] = np.cumsum([p.size for p in parts])[:-1]
        return np.ascontiguousarray(np.concatenate(parts)), off

    obs_c, o_obs = pack("obs_c", 1)
    obs_ab, o_oab = pack("obs_ab", 2)
    bnd, o_bnd = pack("bnd", 0)
    xi, o_xi = pack("xi", 0)
    xo = np.empty_like(xi)
    resid = np.empty((B, 2))
    ll = lambda a: a.ctypes.data_as(_LL)
    _check(lib.sfo_solve_batch(B, nd, nxi, float(rho), shp.ctypes.data_as(_I), _p(ab), _p(box),
                               _p(obs_c), ll(o_obs), _p(obs_ab), ll(o_oab), _p(bnd), ll(o_bnd),
                               _p(xi), ll(o_xi), int(iters), int(ws_hess), COSTS[cost], float(dt),
                               n_bc(insts[0]), _p(xo), None,
                               _p(resid)), "solve_batch")
    outs = [xo[o_xi[k]:o_xi[k] + insts[k]["xi"].size].reshape(insts[k]["xi"].shape)
            for k in range(B)]
    return outs, resid


def fit_positions(pos, n_xi, lib=None):
    """Endpoint-pinned least-squares coefficients of sampled trajectories (eq. poly, p = W xi,
    with the boundary rows fixing coefficients 0 and n_xi - 1): pos [n_d][n][H] ->
    xi [n_d][n][n_xi] with xi_0 = p_0, xi_last = p_{H-1} and the interior the least-squares
    solution (numpy lstsq) against the samples minus the two endpoint columns."""
    pos = np.asarray(pos, dtype=np.float64)
    nd, n, H = pos.shape
    W = basis(H, n_xi, lib)
    p0, p1 = pos[..., 0], pos[..., -1]
    r = pos - W[:, 0] * p0[..., None] - W[:, -1] * p1[..., None]
    sol = np.linalg.lstsq(W[:, 1:-1], r.reshape(-1, H).T, rcond=None)[0]   # [n_xi - 2][rows]
    xi = np.empty((nd, n, n_xi))
    xi[..., 0] = p0
    xi[..., -1] = p1
    xi[..., 1:-1] = sol.T.reshape(nd, n, n_xi - 2)
    return xi


def metrics(inst, xi_bar, rho=DEFAULT_RHO, dt=DEFAULT_DT, lib=None):
    """(||r_p||, max residual in m, smoothness cost, path length) of xi_bar: the residuals of
    ``residual``; the smoothness cost sum_k ||p''_{i|k}||^2 and the path length
    sum_k ||p_{i|k+1} - p_{i|k}|| averaged over robots (the paper's quality metrics)."""
    xi_bar = np.asarray(xi_bar, dtype=np.float64)
    H, nxi = int(inst["H"]), int(inst["n_xi"])
    r = residual(inst, xi_bar, rho=rho, lib=lib)
    acc = np.einsum("kc,dic->dik", basis_dd(H, nxi, dt, lib), xi_bar)
    pos = np.einsum("kc,dic->dik", basis(H, nxi, lib), xi_bar)
    smooth = (acc ** 2).sum(axis=(0, 2)).mean()
    path = np.sqrt((np.diff(pos, axis=2) ** 2).sum(axis=0)).sum(axis=1).mean()
    return np.array([r[0], r[1], smooth, path])


def select(scores_primary, scores_secondary=None, threshold=-np.inf, k=1):
    """Indices of the k best candidates of one group: feasible ones (primary <= threshold)
    first by secondary (or primary), then the rest by primary, NaN last, ties to the lower
    index; -1 past the group's size."""
    p = np.asarray(scores_primary, dtype=np.float64)
    q = p if scores_secondary is None else np.asarray(scores_secondary, dtype=np.float64)

    def key(j):
        feas = p[j] <= threshold
        v = q[j] if feas else p[j]
        if np.isnan(v):
            return (2, 0.0, j)
        return (0 if feas else 1, v, j)

    order = sorted(range(len(p)), key=key)[:k]
    return order + [-1] * (k - len(order))


def positions(xi_bar, H, lib=None):
    """p = W xi_bar for every axis and robot: [n_d][n][H]."""
    W = basis(H, xi_bar.shape[-1], lib)
    return np.einsum("kc,dic->dik", W, xi_bar)
