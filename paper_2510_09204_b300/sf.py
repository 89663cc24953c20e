"""Thin Python binding of the C ABI in ``include/sf.h`` (argument marshalling only).

Every step of the solver runs in ``libsf.so``'s CUDA kernels; this module packs
tensors, passes device pointers and streams, and raises on any non-zero status.
There is no CPU fallback: if the library or a CUDA device is missing, calls fail.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np
import torch

from . import build as _build

(SF_OK, SF_EINVAL, SF_ESHAPE, SF_ECUDA, SF_ENOMEM, SF_ETIMEOUT, SF_ENONFINITE, SF_ESTATE, SF_EUNSUPPORTED,
 SF_ETOOBIG, SF_EBOUNDS) = range(11)
SF_NOALLOC_MAX_INST, SF_NOALLOC_MAX_H = 256, 1024
SF_FP64, SF_FP32, SF_TF32, SF_BF16X3, SF_BF16 = range(5)
SF_PROJ_DENSE, SF_PROJ_STRUCTURED = 0, 1
SF_LAYOUT_XI, SF_LAYOUT_BND, SF_LAYOUT_OBS, SF_LAYOUT_OBS_AB = range(4)
SF_RES_RP, SF_RES_MAX, SF_RES_FP, SF_RES_ITERS, SF_RES_FPSUM, SF_NRES = range(6)

PRECISIONS = {"fp64": SF_FP64, "fp32": SF_FP32, "tf32": SF_TF32, "bf16x3": SF_BF16X3, "bf16": SF_BF16}
PROJECTIONS = {"dense": SF_PROJ_DENSE, "structured": SF_PROJ_STRUCTURED}
COSTS = {"projection": 0, "smoothness": 1}

# every symbol declared in include/sf.h
EXPORTS = ("sf_create", "sf_destroy", "sf_layout", "sf_solve", "sf_solve_backward", "sf_get_status",
           "sf_shape_operator", "sf_profile", "sf_kernel_times", "sf_solve_noalloc", "sf_set_launch",
           "sf_get_launch", "sf_set_option", "sf_get_option", "sf_autotune", "sf_fit_positions", "sf_metrics",
           "sf_select", "sf_alu_peaks", "sf_strerror", "sf_version")
SF_OPT_CULL, SF_OPT_TEST_TIMEOUT, SF_OPT_TC_RESIDENT, SF_OPT_TC_BATCH, SF_OPT_EARLY_EXIT = 1, 2, 3, 4, 5
SF_KT_FORWARD, SF_KT_RESIDUAL, SF_KT_BACKWARD, SF_NKT = range(4)


class sf_shape(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("n_obs", ct.c_int32), ("H", ct.c_int32), ("dyn_obs", ct.c_int32),
                ("a", ct.c_double), ("b", ct.c_double), ("p_min", ct.c_double * 3), ("p_max", ct.c_double * 3)]


class sf_desc(ct.Structure):
    _fields_ = [("n_d", ct.c_int32), ("n_xi", ct.c_int32), ("rho", ct.c_double), ("precision", ct.c_int32),
                ("proj", ct.c_int32), ("n_refine", ct.c_int32), ("max_iters", ct.c_int32),
                ("ckpt_every", ct.c_int32), ("tol", ct.c_double), ("n_inst", ct.c_int32),
                ("shapes", ct.POINTER(sf_shape)), ("stream", ct.c_void_p), ("cost", ct.c_int32), ("dt", ct.c_double),
                ("n_bc", ct.c_int32)]


class sf_instance_data(ct.Structure):
    _fields_ = [("bnd", ct.c_void_p), ("obs_c", ct.c_void_p), ("obs_ab", ct.c_void_p)]


_lib = None


class SFError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s failed: %s (status %d)" % (what, lib().sf_strerror(code).decode(), code))


def lib(path: str | None = None):
    """Load libsf.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        p = path or _build.LIB
        if path is None and _build.stale():
            _build.build()
        L = ct.CDLL(p)
        vp, i32, i64p = ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_int64)
        L.sf_create.argtypes = [ct.POINTER(sf_desc), ct.POINTER(vp)]
        L.sf_destroy.argtypes = [vp]
        L.sf_layout.argtypes = [vp, i32, i64p]
        L.sf_solve.argtypes = [vp, ct.POINTER(sf_instance_data), vp, vp, vp, i32, vp, vp, vp, vp, vp]
        L.sf_solve_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.sf_get_status.argtypes = [vp, ct.POINTER(ct.c_int32)]
        L.sf_shape_operator.argtypes = [vp, i32, i32, ct.POINTER(ct.c_double)]
        L.sf_profile.argtypes = [vp, i32]
        L.sf_kernel_times.argtypes = [vp, ct.POINTER(ct.c_float)]
        L.sf_solve_noalloc.argtypes = [i32, i32, ct.c_double, ct.POINTER(sf_shape), i32, vp, vp, vp, vp, i32, vp,
                                       vp, vp, vp]
        L.sf_set_launch.argtypes = [vp, i32, i32]
        L.sf_autotune.argtypes = [vp, ct.POINTER(sf_instance_data), vp, i32, i32, vp, ct.POINTER(i32),
                                  ct.POINTER(i32), ct.POINTER(ct.c_float)]
        L.sf_get_launch.argtypes = [vp, ct.POINTER(i32), ct.POINTER(i32), ct.POINTER(i32)]
        L.sf_set_option.argtypes = [vp, i32, i32]
        L.sf_fit_positions.argtypes = [i32, i32, i32, ct.POINTER(i32), ct.POINTER(i32), vp, vp, vp]
        L.sf_metrics.argtypes = [vp, ct.POINTER(sf_instance_data), vp, vp, vp]
        L.sf_select.argtypes = [i32, ct.POINTER(i32), vp, vp, ct.c_double, i32, vp, vp]
        L.sf_get_option.argtypes = [vp, i32, ct.POINTER(i32)]
        L.sf_alu_peaks.argtypes = [ct.c_double, ct.POINTER(ct.c_double), vp]
        L.sf_strerror.argtypes = [i32]
        L.sf_strerror.restype = ct.c_char_p
        L.sf_version.restype = i32
        for f in ("sf_create", "sf_destroy", "sf_layout", "sf_solve", "sf_solve_backward", "sf_get_status",
                  "sf_shape_operator", "sf_profile", "sf_kernel_times", "sf_solve_noalloc", "sf_set_launch",
                  "sf_get_launch", "sf_set_option", "sf_get_option", "sf_autotune", "sf_fit_positions", "sf_metrics",
                  "sf_select", "sf_alu_peaks"):
            getattr(L, f).restype = ct.c_int
        _lib = L
    return _lib


def _check(rc, what):
    if rc != SF_OK:
        raise SFError(rc, what)


def _ptr(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ct.c_void_p(stream.cuda_stream)


class SFSolver:
    """A handle over a fixed batch of instance shapes (``sf_create`` .. ``sf_destroy``).

    ``shapes``: list of dicts with keys n, n_obs, H, a, b, pmin, pmax and optional dyn_obs
    (the instance dicts of ``sfgen`` qualify).  ``n_bc``: boundary rows per robot and axis,
    2 (start, goal) or 3 (with the initial velocity, time step ``dt``); None takes it from
    the first shape's ``bnd`` array when it has one, else 2.
    """

    def __init__(self, shapes, n_d, n_xi=11, rho=0.3, precision="fp32", proj="dense", max_iters=1000,
                 ckpt_every=0, tol=1e-3, n_refine=0, stream=None, cost="projection", dt=0.1, n_bc=None):
        if not torch.cuda.is_available():
            raise RuntimeError("SFSolver needs a CUDA device; there is no CPU path")
        L = lib()
        self.n_d, self.n_xi, self.rho = int(n_d), int(n_xi), float(rho)
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.B = len(shapes)
        arr = (sf_shape * self.B)()
        for k, s in enumerate(shapes):
            arr[k].n, arr[k].n_obs, arr[k].H = int(s["n"]), int(s["n_obs"]), int(s["H"])
            arr[k].dyn_obs = int(bool(s.get("dyn_obs", False)))
            arr[k].a, arr[k].b = float(s["a"]), float(s["b"])
            for ax in range(self.n_d):
                arr[k].p_min[ax] = float(s["pmin"][ax])
                arr[k].p_max[ax] = float(s["pmax"][ax])
        self._shapes = [dict(n=int(s["n"]), n_obs=int(s["n_obs"]), H=int(s["H"]),
                             dyn_obs=bool(s.get("dyn_obs", False))) for s in shapes]
        if n_bc is None:
            n_bc = int(np.shape(shapes[0]["bnd"])[-1]) if "bnd" in shapes[0] else 2
        self.n_bc = int(n_bc)
        d = sf_desc(self.n_d, self.n_xi, self.rho, PRECISIONS[precision], PROJECTIONS[proj], int(n_refine),
                    int(max_iters), int(ckpt_every), float(tol), self.B, arr, _stream(stream), COSTS[cost],
                    float(dt), self.n_bc)
        self.cost = cost
        h = ct.c_void_p()
        _check(L.sf_create(ct.byref(d), ct.byref(h)), "sf_create")
        self.h = h
        self.max_iters, self.ckpt_every = int(max_iters), int(ckpt_every)
        self.offsets = {}
        for kind in range(4):
            o = (ct.c_int64 * (self.B + 1))()
            _check(L.sf_layout(h, kind, o), "sf_layout")
            self.offsets[kind] = np.array(o[:], dtype=np.int64)

    # ---- packing -----------------------------------------------------------
    def pack(self, insts, device="cuda"):
        """Pack per-instance arrays: returns dict(bnd, obs_c, obs_ab, xi) device tensors."""
        def cat(key, kind):
            parts = []
            for k, i in enumerate(insts):
                want = self.offsets[kind][k + 1] - self.offsets[kind][k]
                a = np.asarray(i[key], dtype=np.float64).ravel() if want else np.zeros(0)
                if a.size != want:
                    raise ValueError("instance %d: %s has %d values, layout wants %d" % (k, key, a.size, want))
                parts.append(a)
            flat = np.concatenate(parts) if parts else np.zeros(0)
            return torch.as_tensor(flat, dtype=self.dtype, device=device)

        return dict(bnd=cat("bnd", SF_LAYOUT_BND), obs_c=cat("obs_c", SF_LAYOUT_OBS),
                    obs_ab=cat("obs_ab", SF_LAYOUT_OBS_AB), xi=cat("xi", SF_LAYOUT_XI))

    def unpack(self, flat, k):
        """Instance k's [n_d][n][n_xi] view of a packed coefficient tensor."""
        o = self.offsets[SF_LAYOUT_XI]
        s = self._shapes[k]
        return flat[o[k]:o[k + 1]].view(self.n_d, s["n"], self.n_xi)

    def _data(self, data):
        return sf_instance_data(data["bnd"].data_ptr(),
                                data["obs_c"].data_ptr() if data["obs_c"].numel() else None,
                                data["obs_ab"].data_ptr() if data["obs_ab"].numel() else None)

    # ---- calls ---------------------------------------------------------------
    def solve(self, data, xi_cand, iters, xi0=None, lam0=None, xi_out=None, lam_out=None, resid=None,
              want_resid=True, stream=None):
        """sf_solve: returns (xi_out, lam_out, resid [B, SF_NRES] float64 or None)."""
        for t in (xi_cand, xi0, lam0, data["bnd"]):
            if t is not None and (t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous()):
                raise TypeError("arrays must be contiguous CUDA tensors of %s" % self.dtype)
        if xi_out is None:
            xi_out = torch.empty_like(xi_cand)
        if lam_out is None:
            lam_out = torch.empty_like(xi_cand)
        if want_resid and resid is None:
            resid = torch.empty((self.B, SF_NRES), dtype=torch.float64, device=xi_cand.device)
        dd = self._data(data)
        _check(lib().sf_solve(self.h, ct.byref(dd), _ptr(xi_cand), _ptr(xi0), _ptr(lam0), int(iters),
                              _ptr(xi_out), _ptr(lam_out), _ptr(resid) if want_resid else None, None,
                              _stream(stream)), "sf_solve")
        self._keep = (data, xi_cand, xi0, lam0)
        return xi_out, lam_out, (resid if want_resid else None)

    def backward(self, g_xi_out, g_lam_out=None, g_rp2=None, want_xi0=True, want_lam0=True, out=None, stream=None,
                 g_fp=None):
        """sf_solve_backward: returns (g_xi_cand, g_xi0, g_lam0).  ``out``: optional
        preallocated (g_xi_cand, g_xi0, g_lam0) tensors (None entries are skipped).
        g_rp2, g_fp: per-instance float64 weights of ||r_p(xi_out)||^2 and of the fixed-point
        sum resid[:, SF_RES_FPSUM] (None = 0)."""
        ref = g_xi_out
        if out is not None:
            g_xc, g_x0, g_l0 = out
        else:
            g_xc = torch.empty_like(ref)
            g_x0 = torch.empty_like(ref) if want_xi0 else None
            g_l0 = torch.empty_like(ref) if want_lam0 else None
        _check(lib().sf_solve_backward(self.h, _ptr(g_xi_out), _ptr(g_lam_out), _ptr(g_rp2), _ptr(g_fp),
                                       _ptr(g_xc), _ptr(g_x0), _ptr(g_l0), _stream(stream)), "sf_solve_backward")
        return g_xc, g_x0, g_l0

    def metrics(self, data, xi, stream=None):
        """sf_metrics: FP64 [B, 4] device tensor of (||r_p||, max residual in m, smoothness
        cost, path length) per instance of the coefficients ``xi``."""
        out = torch.empty((self.B, 4), dtype=torch.float64, device=xi.device)   # sf_metrics: 4 columns
        dd = self._data(data)
        _check(lib().sf_metrics(self.h, ct.byref(dd), _ptr(xi), _ptr(out), _stream(stream)), "sf_metrics")
        return out

    def set_launch(self, cluster=0, threads=0):
        """sf_set_launch: CTAs per instance (0 = automatic) and threads per CTA (0 = 512)."""
        _check(lib().sf_set_launch(self.h, int(cluster), int(threads)), "sf_set_launch")

    def autotune(self, data, xi_cand, iters, reps=2, stream=None):
        """sf_autotune: returns (cluster, threads, best ms) and keeps that geometry."""
        c, t, ms = ct.c_int32(), ct.c_int32(), ct.c_float()
        dd = self._data(data)
        _check(lib().sf_autotune(self.h, ct.byref(dd), _ptr(xi_cand), int(iters), int(reps), _stream(stream),
                                 ct.byref(c), ct.byref(t), ct.byref(ms)), "sf_autotune")
        return c.value, t.value, ms.value

    def set_option(self, option, value):
        """sf_set_option (re-plans with the current geometry)."""
        _check(lib().sf_set_option(self.h, int(option), int(value)), "sf_set_option")

    def option(self, option):
        """sf_get_option: the option's effective value in the current plan."""
        v = ct.c_int32()
        _check(lib().sf_get_option(self.h, int(option), ct.byref(v)), "sf_get_option")
        return v.value

    def launch(self):
        """(cluster, threads, staged projection rows) in use."""
        c, t, p = ct.c_int32(), ct.c_int32(), ct.c_int32()
        _check(lib().sf_get_launch(self.h, ct.byref(c), ct.byref(t), ct.byref(p)), "sf_get_launch")
        return c.value, t.value, p.value

    def profile(self, enable=True):
        _check(lib().sf_profile(self.h, int(bool(enable))), "sf_profile")

    def kernel_times(self):
        """Milliseconds of (forward, residual, backward) kernels of the last profiled calls."""
        out = (ct.c_float * SF_NKT)()
        _check(lib().sf_kernel_times(self.h, out), "sf_kernel_times")
        return list(out)

    def solve_host(self, host, iters, pinned_out=None, stream=None):
        """End-to-end call from host memory: copy the packed inputs (dict of pinned CPU
        tensors bnd, obs_c, obs_ab, xi) to the device, solve, copy xi_out and the residuals
        back.  Returns (xi_out, resid) host tensors after synchronising the stream."""
        st = stream or torch.cuda.current_stream()
        with torch.cuda.stream(st):
            dev = {k: v.to("cuda", non_blocking=True) for k, v in host.items()}
            xo, lo, res = self.solve(dev, dev["xi"], iters, stream=st)
            if pinned_out is None:
                pinned_out = (torch.empty(xo.shape, dtype=xo.dtype, pin_memory=True),
                              torch.empty(res.shape, dtype=res.dtype, pin_memory=True))
            pinned_out[0].copy_(xo, non_blocking=True)
            pinned_out[1].copy_(res, non_blocking=True)
        st.synchronize()
        return pinned_out

    def status(self):
        out = (ct.c_int32 * self.B)()
        _check(lib().sf_get_status(self.h, out), "sf_get_status")
        return np.array(out[:], dtype=np.int32)

    def operator(self, k, which):
        s = self._shapes[k]
        N = s["n"] * self.n_xi
        nb = self.n_bc
        size = {0: s["H"] * self.n_xi, 1: N * N, 2: N * nb * s["n"],
                3: 3 * self.n_xi ** 2 + 2 * nb * self.n_xi}[which]
        out = np.empty(size)
        _check(lib().sf_shape_operator(self.h, k, which, out.ctypes.data_as(ct.POINTER(ct.c_double))),
               "sf_shape_operator")
        shape = {0: (s["H"], self.n_xi), 1: (N, N), 2: (N, nb * s["n"]), 3: (size,)}[which]
        return out.reshape(shape)

    def close(self):
        if getattr(self, "h", None):
            lib().sf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alu_peaks(seconds=1.0, stream=None):
    """sf_alu_peaks: measured (FP32 flop/s, FP64 flop/s, MUFU rsqrt/s) of the current device."""
    out = (ct.c_double * 3)()
    _check(lib().sf_alu_peaks(float(seconds), out, _stream(stream)), "sf_alu_peaks")
    return tuple(out)


def fit_positions(positions, n_xi=11, stream=None):
    """sf_fit_positions: endpoint-pinned least-squares coefficients of sampled trajectories.
    positions: list of [n_d][n][H] arrays (one per instance, any H >= n_xi); returns the
    list of [n_d][n][n_xi] float64 arrays."""
    if not torch.cuda.is_available():
        raise RuntimeError("fit_positions needs a CUDA device; there is no CPU path")
    arrs = [np.asarray(p, dtype=np.float64) for p in positions]
    nd = arrs[0].shape[0]
    ns = (ct.c_int32 * len(arrs))(*[a.shape[1] for a in arrs])
    Hs = (ct.c_int32 * len(arrs))(*[a.shape[2] for a in arrs])
    pos = torch.as_tensor(np.concatenate([a.ravel() for a in arrs]), device="cuda")
    out = torch.empty(sum(nd * a.shape[1] * n_xi for a in arrs), dtype=torch.float64, device="cuda")
    _check(lib().sf_fit_positions(nd, int(n_xi), len(arrs), ns, Hs, _ptr(pos), _ptr(out), _stream(stream)),
           "sf_fit_positions")
    flat = out.cpu().numpy()
    res, o = [], 0
    for a in arrs:
        m = nd * a.shape[1] * n_xi
        res.append(flat[o:o + m].reshape(nd, a.shape[1], n_xi))
        o += m
    return res


def select(group_sizes, primary, secondary=None, threshold=float("-inf"), k=1, stream=None):
    """sf_select: [groups, k] int32 device tensor of the k best candidates of each group of
    consecutive candidates (feasible = primary <= threshold first, by secondary; then the
    rest by primary; -1 past a group's size)."""
    sizes = (ct.c_int32 * len(group_sizes))(*[int(g) for g in group_sizes])
    out = torch.empty((len(group_sizes), int(k)), dtype=torch.int32, device=primary.device)
    _check(lib().sf_select(len(group_sizes), sizes, _ptr(primary.contiguous()),
                           _ptr(None if secondary is None else secondary.contiguous()), float(threshold), int(k),
                           _ptr(out), _stream(stream)), "sf_select")
    return out


class SFSolve(torch.autograd.Function):
    """(xi_cand, xi0, lam0) -> (xi_out, lam_out, rp2, fp_sum) through ``iters`` SF iterations.

    rp2 is ||r_p(xi_out)||^2 per instance (FP64), fp_sum the sum over the iterations of
    ||z^{l+1} - z^l||^2 per instance (FP64; the fixed-point term of the self-supervised loss
    of eq. NN_loss); both differentiable.  Gradients come from ``sf_solve_backward`` (the
    handle must have been created with ckpt_every > 0).
    """

    @staticmethod
    def forward(ctx, xi_cand, xi0, lam0, solver, data, iters):
        xo, lo, res = solver.solve(data, xi_cand.contiguous(), iters, xi0=xi0.contiguous(),
                                   lam0=lam0.contiguous())
        ctx.solver = solver
        rp2 = res[:, SF_RES_RP] ** 2
        return xo, lo, rp2, res[:, SF_RES_FPSUM].clone()

    @staticmethod
    def backward(ctx, g_xo, g_lo, g_rp2, g_fp):
        s = ctx.solver
        g_xo = torch.zeros_like(s._keep[1]) if g_xo is None else g_xo.contiguous()
        g_lo = None if g_lo is None else g_lo.contiguous()
        g_rp2 = None if g_rp2 is None else g_rp2.contiguous().to(torch.float64)
        g_fp = None if g_fp is None else g_fp.contiguous().to(torch.float64)
        gx, gx0, gl0 = s.backward(g_xo, g_lo, g_rp2, g_fp=g_fp)
        return gx, gx0, gl0, None, None, None
