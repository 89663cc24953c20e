#!/usr/bin/env python
"""Benchmark of the batched, differentiable Safety-Filter solve.

One step = the whole hot path on one batch: sf_solve (every iteration of T on every
instance, checkpoints every c iterations), the FP64 residual check of the result and
sf_solve_backward (the adjoint of all the iterations, seeded with a fixed cotangent).
Default workload: 32 instances of 16 disc robots in a 15 x 15 m 2D map with 20
obstacles, horizon 100, 200 iterations (seeded synthetic instances from ``sfgen``).
Beside it: the plain FP64 GPU path and the other precisions / projections on the same
batch (time and error against FP64), a CUDA-graph replay of the step, the end-to-end
call from pinned host memory and the FP64 oracle on the host cores.  Prints one JSON
line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config C] [--precision P] [--proj dense|structured] [--forward-only]

Under torchrun each rank solves its own batch (seeds offset by rank): weak scaling,
no collective on the data path; the step time is the max over ranks.  --shard-batch
instead splits the one batch over the ranks with shard.balance (strong scaling).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sfgen  # noqa: E402

SF_NRES = 5   # columns of sf_solve's residual output (include/sf.h)

RHO = 0.3
FP32_LANES_PER_SM = 128   # only for the fallback peak when the measurement fails


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", type=int, default=2)
    p.add_argument("--batch", type=int, default=0, help="instances of the config's shape (0: the config's own count)")
    p.add_argument("--precision", default="fp32")
    p.add_argument("--proj", default="structured")
    p.add_argument("--n-refine", type=int, default=0)
    p.add_argument("--ckpt-every", type=int, default=1,
                   help="checkpoint interval of the differentiable step (1: the adjoint recomputes nothing)")
    p.add_argument("--forward-only", action="store_true", help="time sf_solve + residual check without the adjoint")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-compare", action="store_true", help="skip the FP64 and tensor-core comparison solves")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--cluster", type=int, default=0, help="CTAs per instance (with --threads: a fixed geometry, no autotune)")
    p.add_argument("--threads", type=int, default=0)
    p.add_argument("--no-configs", action="store_true", help="skip the other workloads' summary (configs 3, 4, 5)")
    p.add_argument("--shard-batch", action="store_true",
                   help="under torchrun: split the one batch over the ranks (shard.balance) instead of one batch per rank")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(cid, rank=0, world=1, shard_batch=False, batch=0):
    """The config's batch: one batch per rank (seeds offset by rank), or with shard_batch
    this rank's share of the one batch (shard.balance by rows per iteration).  batch > 0
    replaces the config's instance count (the workload is then named for it)."""
    cfg = sfgen.CONFIGS[cid]
    if batch and batch != cfg.B:
        cfg = dataclasses.replace(cfg, B=batch, name=re.sub(r"b\d+", "b%d" % batch, cfg.name, count=1))
    if shard_batch:
        from paper_2510_09204_b300.shard import shard
        _, insts = shard(sfgen.make_batch(cid, B=cfg.B), rank, world)
    else:
        insts = sfgen.make_batch(cid, B=cfg.B, start=rank * cfg.B)
    pairs, obs = sfgen.batch_stats(insts)
    return cfg, insts, pairs, obs


# Algorithmic work per pair or obstacle row in the algebraic form of the alpha/beta/d
# closed forms (line of sight, scaled squared norm, activity test, r_1 = Delta (1 - s)
# and its accumulation): 14 FP operations and one reciprocal square root in 2-D, 19 and
# one in 3-D.
ROW_FLOPS = {2: 14, 3: 19}


def _per_iter(i, proj):
    """Algorithmic FP operations of one forward iteration of one instance: ROW_FLOPS per
    pair or obstacle row, 2 n_d per (robot, timestep) box test, positions W xi_bar once and
    the W' aggregation twice (of e and of r_1) at 2 n_d n H n_xi each, lambda and the
    right-hand side 6 n_d N, projection 2 n_d N^2 (dense) or 4 n_d n n_xi^2 (Kronecker
    form).  Returns (flops, rows, projection flops); rows is also the count of reciprocal
    square roots."""
    nd, n, H, nxi, no = i["n_d"], i["n"], i["H"], i["n_xi"], i["n_obs"]
    N = n * nxi
    rows = (n * (n - 1) // 2 + n * no) * H
    per = rows * ROW_FLOPS[nd] + 2 * nd * n * H + 3 * (2 * nd * n * H * nxi) + 6 * nd * N
    proj_f = 2 * nd * N * N if proj == "dense" else 4 * nd * n * nxi * nxi
    return per + proj_f, rows, proj_f


def algorithmic_flops(insts, iters, proj, kernel="k_forward", ckpt_every=1):
    """(FP operations, reciprocal square roots) of one launch of ``kernel`` at the
    algorithmic minimum.  k_forward: iters forward iterations.  k_backward: the
    recomputation inside the checkpoint segments (c - 1 forward iterations per segment of
    c) plus the reverse sweep, per iteration ROW_FLOPS per row (the line of sight,
    activity test and the active row's Jacobian product), 2 n_d per box entry, positions,
    R* = W g* and W' p* (2 n_d n H n_xi each), the projection and 8 n_d N elementwise.
    k_residual: one FP64 pass over the rows and the positions."""
    c = max(1, ckpt_every)
    recompute = iters - (iters + c - 1) // c
    tot, mufu = 0.0, 0.0
    for i in insts:
        fwd, rows, proj_f = _per_iter(i, proj)
        nd, n, H, nxi = i["n_d"], i["n"], i["H"], i["n_xi"]
        if kernel == "k_forward":
            tot += fwd * iters
            mufu += rows * iters
        elif kernel == "k_backward":
            rev = rows * ROW_FLOPS[nd] + 2 * nd * n * H + 6 * nd * n * H * nxi + proj_f + 8 * nd * n * nxi
            tot += fwd * recompute + rev * iters
            mufu += rows * (recompute + iters)
        else:
            tot += rows * ROW_FLOPS[nd] + 2 * nd * n * H + 2 * nd * n * H * nxi
            mufu += rows
    return tot, mufu


def alu_peaks(dev, seconds=1.0):
    """Measured pipe throughputs of this GPU (sf_alu_peaks: FP32 FMA, FP64 FMA, MUFU rsqrt,
    each a timed loop of about a second), and the SM count; falls back to the FP32 lanes x
    clock product when the measurement fails."""
    import torch

    from paper_2510_09204_b300.sf import alu_peaks as measure
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    try:
        f32, f64, mufu = measure(seconds)
        return {"fp32_tflops": f32 / 1e12, "fp64_tflops": f64 / 1e12, "mufu_tops": mufu / 1e12, "sms": sms,
                "source": "measured on this GPU by sf_alu_peaks (FMA / rsqrt dependency chains on every SM, "
                          "CUDA events, best of 3 launches of ~%.2f s)" % (seconds / 3)}
    except Exception as e:  # reported, never hidden
        sm_max = float(measured_peaks().get("sm_max_mhz", 2032.0))
        return {"fp32_tflops": sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12, "fp64_tflops": None,
                "mufu_tops": None, "sms": sms,
                "source": "derived (%d SMs x 128 FP32 lanes x 2 x %.0f MHz): measurement failed: %s"
                          % (sms, sm_max, str(e)[:120])}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, timestamped, sampled every 20 ms from before
    the warm-up until after the timed region; only samples inside the timed window count."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_sel):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_sel), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        self.t0 = self.t1 = None

    def wait_first(self, timeout=5.0):
        end = time.time() + timeout
        while self.p is not None and time.time() < end:
            if os.path.getsize(self.f.name) > 0:
                return
            time.sleep(0.02)

    def window(self, t0, t1):
        self.t0, self.t1 = t0, t1

    def stop(self):
        import datetime
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        with open(self.f.name) as fh:
            lines = fh.read().splitlines()
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]), float(parts[3]),
                             [nm for nm, val in zip(names, parts[5:9]) if val.lower().startswith("active")]))
            except ValueError:
                continue
        inside = [r for r in rows if self.t0 is not None and self.t0 - 0.01 <= r[0] <= self.t1 + 0.01]
        how = "samples inside the timed region"
        if not inside and rows and self.t0 is not None:
            mid = 0.5 * (self.t0 + self.t1)
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
            how = "nearest sample (timed region shorter than the 20 ms sampling interval)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = sorted({x for r in inside for x in r[4]})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "power_w_max": max(r[3] for r in inside), "reasons": reasons, "samples": len(inside),
                "sampling": how}


def profiled_traffic(kernel, workload, precision, proj):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary of this workload,
    or None when there is none or the kernel sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "%s_%s_%s_%s.md" % (kernel, workload, precision, proj))
    try:
        with open(path) as f:
            kv = dict(line.split(":", 1) for line in f.read().splitlines()
                      if line.startswith(("traffic_bytes_per_launch:", "source_sha256:")))
    except OSError:
        return None, None
    sys.path.insert(0, os.path.join(ROOT, "paper_2510_09204_b300"))
    import build as _build
    if kv.get("source_sha256", "").strip() != _build.source_digest():
        return None, os.path.relpath(path, ROOT) + " (stale: kernel sources changed since the capture)"
    return int(kv["traffic_bytes_per_launch"]), os.path.relpath(path, ROOT)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _oracle_step(sample, iters, seeds, forward_only, pool):
    """One step of the oracle on ``sample``: the FP64 solve (OpenMP over instances) or,
    for the differentiable step, per instance (threads over instances) the solve, the
    residual check and the reverse pass (which recomputes the forward, as the adjoint
    kernel does)."""
    import oracle
    if forward_only:
        oracle.solve_batch(sample, iters, rho=RHO)
        return

    def one(k):
        inst = sample[k]
        xo = oracle.solve(inst, iters, rho=RHO)["xi"]
        oracle.residual(inst, xo, rho=RHO)
        oracle.solve_backward(inst, iters, g_xi_out=seeds[k], g_rp2=1.0, rho=RHO)

    list(pool.map(one, range(len(sample))))


def _oracle_sample(insts, iters, forward_only, budget_s):
    """A bounded sample of the batch sized to about ``budget_s`` of host work per step."""
    import concurrent.futures
    import oracle
    oracle.load()
    cores = os.cpu_count() or 1
    pool = concurrent.futures.ThreadPoolExecutor(max_workers=cores)
    seeds = [np.random.default_rng(100 + k).normal(size=i["xi"].shape) * 1e-2 for k, i in enumerate(insts)]
    t0 = time.perf_counter()
    _oracle_step(insts[:1], iters, seeds, forward_only, pool)
    one = max(time.perf_counter() - t0, 1e-3)
    k = int(max(1, min(len(insts), budget_s / one * cores * 0.7)))
    return insts[:k], seeds[:k], pool, cores


def _oracle_desc(k, B, iters, forward_only, dt=None):
    what = ("FP64 solve, OpenMP over instances" if forward_only else
            "FP64 solve + residual + reverse pass per instance, threads over instances")
    d = "%d of %d instances x %d iterations, %s" % (k, B, iters, what)
    return d + (" (%.1f s)" % dt if dt is not None else "")


def cpu_baseline(insts, iters, forward_only, budget_s=15.0):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample of the batch,
    and on one core (one instance's step)."""
    sample, seeds, pool, cores = _oracle_sample(insts, iters, forward_only, budget_s)
    t0 = time.perf_counter()
    _oracle_step(sample, iters, seeds, forward_only, pool)
    dt = time.perf_counter() - t0
    pairs, _ = sfgen.batch_stats(sample)
    import concurrent.futures
    one = concurrent.futures.ThreadPoolExecutor(max_workers=1)
    t1 = time.perf_counter()
    _oracle_step(insts[:1], iters, seeds[:1], forward_only, one)   # one instance: one thread either way
    dt1 = time.perf_counter() - t1
    p1, _ = sfgen.batch_stats(insts[:1])
    return {"value": pairs * iters / dt, "unit": "pair-timestep updates/s", "cores": cores, "kind": "oracle",
            "sample": _oracle_desc(len(sample), len(insts), iters, forward_only, dt),
            "single_thread": {"value": p1 * iters / dt1, "sample": "1 instance on one thread (%.2f s)" % dt1}}


METRIC = "SF ms/batch & pair-timestep updates/s, chosen vs plain FP64, residual≤1e-3 m"


def _config(cfg, insts, iters, a, extra=None):
    c = {"workload": cfg.name, "instances": len(insts), "robots": cfg.n[0], "obstacles": cfg.n_obs[0],
         "horizon": cfg.H[0], "iterations": iters, "n_d": cfg.n_d, "n_xi": 11, "rho": RHO,
         "step": ("sf_solve + FP64 residual check" if a.forward_only else
                  "sf_solve (checkpoints every %d) + FP64 residual check + sf_solve_backward" % a.ckpt_every)}
    c.update(extra or {})
    return c


def run_reference(a):
    """The oracle as the reference arm: rank 0 only, host cores, bounded sample per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg, insts, _, _ = workload(a.config, batch=a.batch)
    iters = cfg.iters
    sample, seeds, pool, cores = _oracle_sample(insts, iters, a.forward_only, 2.0)   # ~2 s of host work per step
    pairs, _ = sfgen.batch_stats(sample)
    for _ in range(a.warmup):
        _oracle_step(sample, iters, seeds, a.forward_only, pool)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        _oracle_step(sample, iters, seeds, a.forward_only, pool)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = pairs * iters * a.steps / tot
    desc = _oracle_desc(len(sample), len(insts), iters, a.forward_only) + " per step"
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "pair-timestep updates/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(cfg, insts, iters, a, {"precision": "fp64 (oracle)",
                                                     "instances_timed_per_step": len(sample)}),
            "cpu_baseline": {"value": value, "unit": "pair-timestep updates/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "pair-timestep updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Step:
    """Buffers and calls of one bench step on one solver: the solve with the FP64 residual
    check and, unless forward-only, the adjoint seeded with a fixed cotangent on xi_out
    and d/d||r_p||^2 = 1 (the work of the reverse pass does not depend on the seed values)."""

    def __init__(self, solver, data, iters, forward_only, stream):
        import torch
        self.s, self.data, self.iters, self.fo, self.stream = solver, data, iters, forward_only, stream
        x = data["xi"]
        self.xo, self.lo = torch.empty_like(x), torch.empty_like(x)
        self.res = torch.empty((solver.B, SF_NRES), dtype=torch.float64, device=x.device)
        g = np.random.default_rng(7).normal(size=x.numel()) * 1e-2
        self.gxo = torch.as_tensor(g, dtype=x.dtype, device=x.device)
        self.grp2 = torch.ones(solver.B, dtype=torch.float64, device=x.device)
        self.g = (torch.empty_like(x), torch.empty_like(x), torch.empty_like(x))

    def __call__(self):
        self.s.solve(self.data, self.data["xi"], self.iters, xi_out=self.xo, lam_out=self.lo, resid=self.res,
                     stream=self.stream)
        if not self.fo:
            self.s.backward(self.gxo, None, self.grp2, out=self.g, stream=self.stream)

    def launches(self):
        return 2 if self.fo else 3


def _time_steps(step, n, stream, flush=None, per_kernel=None):
    import torch
    times, kt = [], []
    for _ in range(n):
        if flush is not None:
            flush.zero_()  # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        if per_kernel is not None:
            kt.append(per_kernel())
    return times, kt


def _positions(solver, flat, insts):
    import torch
    out = []
    for k in range(len(insts)):
        W = torch.as_tensor(solver.operator(k, 0), device=flat.device, dtype=torch.float64)
        out.append(torch.einsum("hc,anc->anh", W, solver.unpack(flat, k).double()))
    return out


def _max_pos_err(pa, pb):
    return max(float((a - b).norm(dim=0).max()) for a, b in zip(pa, pb))


def _pos_errs(pa, pb):
    """Per instance: the largest Euclidean position difference over robots and timesteps."""
    return [float((a - b).norm(dim=0).max()) for a, b in zip(pa, pb)]


# The per-instance rule of the parity tests: FP32 positions within POS_TOL of FP64 on the
# same input, or, for at most 15% of a batch, within 10 times the instance's own FP64
# sensitivity (the largest position change over SENS_DRAWS draws of a SENS_ULPS-ulp
# candidate perturbation: ill-conditioned instances move that much in exact arithmetic).
POS_TOL, SENS_ULPS, SENS_DRAWS, SENS_FACTOR, SENS_MAX_FRAC = 1e-4, 16, 3, 10.0, 0.15


def ulp_perturbed(inst, seed, ulps):
    """The instance with its candidate moved by ``ulps`` float32 ulps (random sign per
    coefficient)."""
    rng = np.random.default_rng(seed)
    xi = np.asarray(inst["xi"], dtype=np.float64)
    step = np.abs(np.spacing(xi.astype(np.float32))).astype(np.float64)
    return dict(inst, xi=xi + ulps * step * rng.choice([-1.0, 1.0], size=xi.shape))


def _variant(insts, nd, iters, a, precision, proj, n_refine, dev, stream, flush, ref_pos, ref_res, reps=10):
    """Times the step of another precision / projection and reports its error against
    the FP64 GPU solve of the same batch."""
    import torch

    from paper_2510_09204_b300 import SFSolver
    s = SFSolver(insts, nd, 11, rho=RHO, precision=precision, proj=proj, max_iters=iters,
                 ckpt_every=0 if a.forward_only else a.ckpt_every, n_refine=n_refine)
    d = s.pack(insts, device=dev)
    if not a.no_autotune:
        s.autotune(d, d["xi"], iters, reps=1, stream=stream)
    st = Step(s, d, iters, a.forward_only, stream)
    for _ in range(2):
        st()
    torch.cuda.synchronize()
    times, _ = _time_steps(st, reps, stream, flush)
    r = st.res.cpu().numpy()
    out = {"precision": precision, "projection": proj, "n_refine": n_refine, "ms_per_step": statistics.median(times),
           "launch": list(s.launch()[:2]), "status_ok": bool((s.status() == 0).all())}
    if precision in ("tf32", "bf16", "bf16x3"):
        # the dense projection's tensor-core work (eq. batch_comp): 2 n_d N^2 per instance per
        # projection, one projection per iteration forward and one per reverse step, each
        # applied 1 + n_refine times, with three products per BF16 x3 product; its rate over the
        # whole step is a lower bound on the tensor kernels' rate
        pk = measured_peaks()
        prods = (3 if precision == "bf16x3" else 1) * (1 + n_refine) * (1 if a.forward_only else 2)
        flops = sum(2.0 * nd * (i["n"] * 11) ** 2 for i in insts) * iters * prods
        tf = flops / (out["ms_per_step"] * 1e-3) / 1e12
        peak = pk.get("bf16_tflops")
        if peak and precision == "tf32":
            peak = peak * 1.1 / 2.25   # the nominal TF32 : BF16 dense ratio
        out["tensor"] = {"algorithmic_tflop_per_step": flops / 1e12, "achieved_tflops_over_step": tf,
                         "peak_tflops": peak, "frac_of_measured": (tf / peak) if peak else None,
                         "note": "tcgen05 products of the dense projection only; the step is bound by "
                                 "the iteration's other phases"}
    if ref_pos is not None:
        out["max_position_error_vs_fp64_m"] = _max_pos_err(_positions(s, st.xo, insts), ref_pos)
        out["max_final_residual_diff_vs_fp64_m"] = float(np.abs(r[:, 1] - ref_res[:, 1]).max())
    out["_pos"], out["_res"] = _positions(s, st.xo, insts), r
    s.close()
    return out


def _optimizer(insts, nd, iters, a, dev, stream, flush, pairs, dt=0.05, reps=10):
    """The trajectory optimiser (smoothness cost, eq. eq::form) on the same batch and
    iteration count: forward solve with the FP64 residual check, ms per batch, the final
    residual and the smoothness cost 1/2 sum xi' Q1 xi from the library's cost block."""
    import torch

    from paper_2510_09204_b300 import SFSolver
    s = SFSolver(insts, nd, 11, rho=RHO, precision=a.precision, proj=a.proj, max_iters=iters,
                 cost="smoothness", dt=dt)
    d = s.pack(insts, device=dev)
    if not a.no_autotune:
        s.autotune(d, d["xi"], iters, reps=1, stream=stream)
    st = Step(s, d, iters, True, stream)
    for _ in range(2):
        st()
    torch.cuda.synchronize()
    times, _ = _time_steps(st, reps, stream, flush)
    ms = statistics.median(times)
    r = st.res.cpu().numpy()
    costs = []
    for k in range(len(insts)):
        q1 = torch.as_tensor(s.operator(k, 3)[2 * 121 + 44:].reshape(11, 11), device=dev)
        x = s.unpack(st.xo, k).double()
        costs.append(0.5 * float(torch.einsum("anc,cd,and->", x, q1, x)))
    out = {"cost": "smoothness", "dt": dt, "precision": a.precision, "projection": a.proj, "iterations": iters,
           "ms_per_batch": ms, "value": pairs * iters / (ms * 1e-3), "unit": "pair-timestep updates/s",
           "final_max_residual_m_median": float(np.median(r[:, 1])),
           "smoothness_cost_median": float(np.median(costs)), "launch": list(s.launch()[:2])}
    s.close()
    return out


def _convergence(insts, nd, a, dev, stream, iters=4000, tol=1e-3):
    """Time to the paper's residual threshold: the chosen path run for up to ``iters``
    iterations on the same batch (forward only), with each instance's first iteration whose
    max residual is <= tol (the solver's iterations-to-tolerance output)."""
    import torch

    from paper_2510_09204_b300 import SFSolver
    s = SFSolver(insts, nd, 11, rho=RHO, precision=a.precision, proj=a.proj, max_iters=iters, tol=tol)
    d = s.pack(insts, device=dev)
    s.solve(d, d["xi"], iters, stream=stream)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, _, res = s.solve(d, d["xi"], iters, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    its = res[:, 3].cpu().numpy()
    ok = its >= 0
    # the same with SF_OPT_EARLY_EXIT: converged instances stop and free their SMs; the batch
    # still waits for the instances that never meet the tolerance
    from paper_2510_09204_b300.sf import SF_OPT_EARLY_EXIT
    s.set_option(SF_OPT_EARLY_EXIT, 1)
    s.solve(d, d["xi"], iters, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    s.solve(d, d["xi"], iters, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms_early = e0.elapsed_time(e1)
    s.close()
    need = int(its[ok].max()) if ok.all() else None
    return {"iterations": iters, "tol_m": tol, "ms": ms, "ms_early_exit": ms_early, "frac_converged": float(ok.mean()),
            "iters_to_tol_median": float(np.median(its[ok])) if ok.any() else None,
            "iters_to_tol_max": int(its[ok].max()) if ok.any() else None,
            "ms_until_every_instance_converged": ms * need / iters if need is not None else None}


def _pipeline(a, dev, stream, problems=50, per=10, keep=5, iters=500):
    """The paper's throughput scenario for the pipeline: 50 problems of the 16-robot 2D
    shape, 10 candidates each (the problem's candidate plus smooth noise), keep the 5 least
    violating, refine them with `iters` SF iterations and pick the best per problem.
    Timed end to end through pipeline.refine_candidates (handles, packing, factorisation,
    every stage), and the 250-trajectory SF solve alone on a prepared handle."""
    import torch

    from paper_2510_09204_b300 import SFSolver
    from paper_2510_09204_b300.pipeline import refine_candidates
    probs = sfgen.make_batch(2, B=problems, start=1000)
    rng = np.random.default_rng(17)
    cands = []
    for p in probs:
        x = np.repeat(p["xi"][None], per, axis=0)
        x[..., 1:-1] += rng.normal(0, 0.3, size=x[..., 1:-1].shape)
        cands.append(x)
    from paper_2510_09204_b300.pipeline import HandleCache
    kw = dict(keep=keep, iters=iters, precision=a.precision, proj=a.proj, rho=RHO)
    refine_candidates(probs, cands, **kw)   # warm-up (kernels, allocator)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = refine_candidates(probs, cands, **kw)
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    # a planner that calls again with the same shapes keeps its handles (no sf_create)
    cache = HandleCache()
    refine_candidates(probs, cands, cache=cache, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    refine_candidates(probs, cands, cache=cache, **kw)
    torch.cuda.synchronize()
    total_cached = time.perf_counter() - t0
    cache.close()
    kept = [dict(probs[g], xi=cands[g][j]) for g in range(problems) for j in out[g]["refined"]]
    s = SFSolver(kept, 2, 11, rho=RHO, precision=a.precision, proj=a.proj, max_iters=iters)
    d = s.pack(kept, device=dev)
    if not a.no_autotune:
        s.autotune(d, d["xi"], iters, reps=1, stream=stream)
    st = Step(s, d, iters, True, stream)
    st()
    torch.cuda.synchronize()
    times, _ = _time_steps(st, 5, stream)
    s.close()
    return {"problems": problems, "candidates_per_problem": per, "kept": keep, "trajectories_refined": len(kept),
            "robots": 16, "iterations": iters, "precision": a.precision, "projection": a.proj,
            "ms_end_to_end": 1e3 * total, "ms_end_to_end_cached_handles": 1e3 * total_cached,
            "ms_sf_solve_250": statistics.median(times),
            "feasible_fraction": float(np.mean([o["feasible"] for o in out])),
            "paper": "< 300 ms to refine 250 trajectories (RTX 5090, JAX; robots and iterations not stated)"}


def rounded32(inst):
    """The instance as an FP32 handle holds it: every array and shape parameter rounded to
    float32 (an FP32 solve cannot see finer input than that)."""
    p = dict(inst)
    for key in ("xi", "bnd", "obs_c", "obs_ab", "pmin", "pmax"):
        p[key] = np.asarray(inst[key], dtype=np.float32).astype(np.float64)
    for key in ("a", "b"):
        p[key] = float(np.float32(inst[key]))
    return p


def _config_step(cid, precision, proj, n_refine, dev, stream, flush, reps=5, graph=False, round_input=False,
                 perturb=None):
    """One workload's step on the GPU (the config's own iteration count; the
    differentiable config 4 also runs the adjoint, checkpoints every 10): autotuned
    geometry, CUDA events, L2 flushed between steps; optionally replayed from a CUDA
    graph.  Returns (record, positions, residuals)."""
    import torch

    from paper_2510_09204_b300 import SFSolver
    cfg = sfgen.CONFIGS[cid]
    insts = sfgen.make_batch(cid)
    if round_input:
        insts = [rounded32(i) for i in insts]
    if perturb is not None:   # (seed, ulps): the sensitivity draws
        insts = [ulp_perturbed(i, perturb[0] * 1000 + k, perturb[1]) for k, i in enumerate(insts)]
    iters, nd = cfg.iters, cfg.n_d
    ck = int(cfg.extra.get("ckpt_every", 0))
    fwd_only = ck == 0
    s = SFSolver(insts, nd, 11, rho=RHO, precision=precision, proj=proj, max_iters=iters, ckpt_every=ck,
                 n_refine=n_refine)
    d = s.pack(insts, device=dev)
    s.autotune(d, d["xi"], iters, reps=1, stream=stream)
    st = Step(s, d, iters, fwd_only, stream)
    for _ in range(2):
        st()
    torch.cuda.synchronize()
    run = st
    if graph:
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            gst = Step(s, d, iters, fwd_only, side)
            gst()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            gst.stream = torch.cuda.current_stream()
            gst()
        run, st = g.replay, gst
    times, _ = _time_steps(run, reps, stream, flush)
    ok = bool((s.status() == 0).all())
    pos, res = _positions(s, st.xo, insts), st.res.cpu().numpy()
    rec = {"precision": precision, "projection": proj, "n_refine": n_refine, "ms_per_step": statistics.median(times),
           "launch": list(s.launch()[:2]), "status_ok": ok, "cuda_graph": graph}
    s.close()
    return rec, pos, res, insts, iters, fwd_only


def other_configs(dev, stream, flush, peaks):
    """The other workloads of the benchmark set, each against the plain FP64 GPU path (time
    on the same batch; max position error and final residual difference against FP64 on
    the same input as FP32 holds it, i.e. rounded to float32, and the position difference
    to FP64 on the unrounded input beside it) and against the measured FP32 peak
    (algorithmic flops of its step / time):
      3  64 uneven instances, FP32 structured, replayed from a CUDA graph
      4  128 x 32 robots, FP32 differentiable step (forward + adjoint, checkpoints every 10)
      5  16 x 64 robots in 3-D: FP32 (structured, dense SIMT) and the tensor-core projection
         in BF16 (+5 refinement passes), TF32 (+3) and BF16 x3 (+1)
    Positions are judged per instance by the parity tests' rule: each instance above 1e-4 m
    is listed with its FP64 sensitivity, and within_tolerance_rule says whether all of them
    stay within 10 times it (and at most 15% of the batch is above)."""
    out = {}
    plan = {3: [("fp32", "structured", 0, True)], 4: [("fp32", "structured", 0, False)],
            5: [("fp32", "structured", 0, False), ("fp32", "dense", 0, False), ("bf16", "dense", 5, False),
                ("tf32", "dense", 3, False), ("bf16x3", "dense", 1, False)]}
    for cid, runs in plan.items():
        ref, praw, _, insts, iters, fwd_only = _config_step(cid, "fp64", "structured", 0, dev, stream, flush, reps=3)
        _, pref, rref, _, _, _ = _config_step(cid, "fp64", "structured", 0, dev, stream, flush, reps=1,
                                              round_input=True)
        sens = None   # FP64 sensitivity per instance, computed when some instance needs it
        recs = []
        for prec, proj, nr, gr in runs:
            rec, pos, res, _, _, _ = _config_step(cid, prec, proj, nr, dev, stream, flush, graph=gr)
            fl = algorithmic_flops(insts, iters, proj, "k_forward")[0]
            if not fwd_only:
                fl += algorithmic_flops(insts, iters, proj, "k_backward", 10)[0]
            errs = _pos_errs(pos, pref)
            over = [k for k, e in enumerate(errs) if e > POS_TOL]
            if over and sens is None:
                draws = [_config_step(cid, "fp64", "structured", 0, dev, stream, flush, reps=1, round_input=True,
                                      perturb=(d + 1, SENS_ULPS))[1] for d in range(SENS_DRAWS)]
                sens = [max(e) for e in zip(*[_pos_errs(p, pref) for p in draws])]
            rec["max_position_error_vs_fp64_m"] = max(errs)
            rec["median_position_error_vs_fp64_m"] = float(np.median(errs))
            rec["instances_above_1e-4_m"] = [{"instance": k, "error_m": errs[k], "fp64_sensitivity_m": sens[k]}
                                             for k in over]
            rec["within_tolerance_rule"] = (all(errs[k] <= SENS_FACTOR * sens[k] for k in over) and
                                            len(over) <= SENS_MAX_FRAC * len(errs))
            rec["max_position_diff_vs_fp64_unrounded_input_m"] = _max_pos_err(pos, praw)
            rec["max_final_residual_diff_vs_fp64_m"] = float(np.abs(res[:, 1] - rref[:, 1]).max())
            rec["achieved_tflops"] = fl / (rec["ms_per_step"] * 1e-3) / 1e12
            rec["frac_of_measured_fp32"] = rec["achieved_tflops"] / peaks["fp32_tflops"]
            rec["speedup_vs_fp64"] = ref["ms_per_step"] / rec["ms_per_step"]
            recs.append(rec)
        cfg = sfgen.CONFIGS[cid]
        out[cfg.name] = {"iterations": iters, "step": "forward" if fwd_only else "forward + adjoint",
                         "fp64_gpu_ms": ref["ms_per_step"], "runs": recs}
    return out


def batch_sweep(dev, stream, flush, peaks, sizes=(32, 128, 512)):
    """The config-2 step (16 robots, 2-D, 200 iterations, forward + FP64 residual check +
    adjoint, checkpoints every iteration) at growing batch sizes: config 2's 32 instances
    leave SMs idle and its time is one instance's dependent chain, while larger batches
    fill the GPU.  Per size: autotuned geometry, median of 3 steps with the L2 flushed,
    throughput and the fraction of the measured FP32 peak over both step kernels."""
    import torch

    from paper_2510_09204_b300 import SFSolver
    cfg = sfgen.CONFIGS[2]
    out = []
    for B in sizes:
        insts = sfgen.make_batch(2, B=B)
        pairs, _ = sfgen.batch_stats(insts)
        s = SFSolver(insts, 2, 11, rho=RHO, precision="fp32", proj="structured", max_iters=cfg.iters, ckpt_every=1)
        d = s.pack(insts, device=dev)
        c, t, _ = s.autotune(d, d["xi"], cfg.iters, reps=1, stream=stream)
        st = Step(s, d, cfg.iters, False, stream)
        for _ in range(2):
            st()
        torch.cuda.synchronize()
        times, _ = _time_steps(st, 3, stream, flush)
        ms = statistics.median(times)
        fl = algorithmic_flops(insts, cfg.iters, "structured", "k_forward")[0] + \
            algorithmic_flops(insts, cfg.iters, "structured", "k_backward", 1)[0]
        out.append({"instances": B, "cluster": c, "threads": t, "ms_per_step": ms,
                    "pair_timestep_updates_per_s": pairs * cfg.iters / (ms * 1e-3),
                    "frac_of_measured_fp32": fl / (ms * 1e-3) / 1e12 / peaks["fp32_tflops"],
                    "status_ok": bool((s.status() == 0).all())})
        s.close()
    return out


def summary_of(line, configs):
    """The few numbers a reader needs, last in the line: the chosen step against plain
    FP64 on the GPU, and per other workload its fastest run's time, error and fraction."""
    s = {"chosen_ms": line["ms_per_step"], "roofline_frac": line["roofline"]["frac"]}
    if line.get("batch_sweep"):
        s["batch_sweep"] = {str(b["instances"]): {"ms": round(b["ms_per_step"], 3),
                                                  "frac": round(b["frac_of_measured_fp32"], 4)}
                            for b in line["batch_sweep"]}
    f = line.get("fp64_gpu")
    if f:
        s.update(fp64_gpu_ms=f["ms_per_step"], chosen_speedup_vs_fp64=f["chosen_speedup"],
                 chosen_max_position_error_vs_fp64_m=f["chosen_max_position_error_m"])
    for name, c in (configs or {}).items():
        best = min(c["runs"], key=lambda r: r["ms_per_step"])
        s[name] = {"fp64_gpu_ms": c["fp64_gpu_ms"],
                   "runs_ms": {"%s/%s+%d" % (r["precision"], r["projection"], r["n_refine"]): round(r["ms_per_step"], 3)
                               for r in c["runs"]},
                   "best": "%s/%s" % (best["precision"], best["projection"]), "best_ms": best["ms_per_step"],
                   "best_frac": best["frac_of_measured_fp32"],
                   "max_position_error_vs_fp64_m": max(r["max_position_error_vs_fp64_m"] for r in c["runs"]),
                   "instances_above_1e-4_m": max(len(r["instances_above_1e-4_m"]) for r in c["runs"]),
                   "within_tolerance_rule": all(r["within_tolerance_rule"] for r in c["runs"])}
    return s


def main():
    a = args_()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import torch.distributed as dist

    from paper_2510_09204_b300 import SFSolver
    from paper_2510_09204_b300.shard import max_over_ranks

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, insts, pairs, obs = workload(a.config, rank, world, a.shard_batch, a.batch)
    # work of the whole job: every rank's batch, or the one batch split over the ranks
    pairs_job = sfgen.batch_stats(sfgen.make_batch(a.config, B=cfg.B))[0] if a.shard_batch else pairs * world
    peaks = alu_peaks(dev)   # before the timed region
    iters = cfg.iters
    nd = cfg.n_d
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    solver = SFSolver(insts, nd, 11, rho=RHO, precision=a.precision, proj=a.proj, max_iters=iters,
                      ckpt_every=0 if a.forward_only else a.ckpt_every, n_refine=a.n_refine)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t_setup)
    data = solver.pack(insts, device=dev)
    tune = None
    if a.cluster:
        solver.set_launch(a.cluster, a.threads)
    elif not a.no_autotune:
        t0 = time.perf_counter()
        c, t, ms = solver.autotune(data, data["xi"], iters, reps=2, stream=stream)
        tune = {"cluster": c, "threads": t, "best_step_ms": ms, "tuning_s": time.perf_counter() - t0}
    solver.profile(True)
    step = Step(solver, data, iters, a.forward_only, stream)

    try:
        gsel = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        gsel = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(gsel)
    clocks.wait_first()
    for _ in range(max(a.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert (solver.status() == 0).all(), "non-finite iterates or a timed-out wait"

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    t_start = time.time()
    times, kts = _time_steps(step, a.steps, stream, flush, solver.kernel_times)
    barrier()
    clocks.window(t_start, time.time())
    clk = clocks.stop()
    tot_ms = max_over_ranks(sum(times), dev)
    ms_step = tot_ms / a.steps
    value = pairs_job * iters / (ms_step * 1e-3)
    r = step.res.cpu().numpy()
    chosen_pos = _positions(solver, step.xo, insts)

    # the same step replayed from a CUDA graph
    graph = None
    try:
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            gstep = Step(solver, data, iters, a.forward_only, side)
            gstep()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            gstep.stream = torch.cuda.current_stream()
            gstep()
        gt, _ = _time_steps(g.replay, a.steps, stream, flush)
        graph = {"ms_per_step": statistics.median(gt),
                 "bitwise_equal_to_eager": bool(torch.equal(gstep.xo, step.xo) and
                                                (a.forward_only or torch.equal(gstep.g[0], step.g[0])))}
    except Exception as e:  # reported, never hidden
        graph = {"error": str(e)[:200]}

    # end to end through the public API from pinned host memory: inputs (and the
    # cotangent) in, xi_out, the residuals and d/dxi_cand out
    e2e = None
    if not a.no_e2e:
        host = {k: v.cpu().pin_memory() for k, v in data.items()}
        hg = step.gxo.cpu().pin_memory()
        outs = [torch.empty(step.xo.shape, dtype=step.xo.dtype, pin_memory=True),
                torch.empty(step.res.shape, dtype=step.res.dtype, pin_memory=True)]
        if not a.forward_only:
            outs.append(torch.empty(step.xo.shape, dtype=step.xo.dtype, pin_memory=True))

        def e2e_step():
            d = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
            xo, _, res = solver.solve(d, d["xi"], iters, stream=stream)
            outs[0].copy_(xo, non_blocking=True)
            outs[1].copy_(res, non_blocking=True)
            if not a.forward_only:
                gx, _, _ = solver.backward(hg.to(dev, non_blocking=True), None, step.grp2, stream=stream)
                outs[2].copy_(gx, non_blocking=True)
            stream.synchronize()

        for _ in range(2):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            e2e_step()
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / a.steps, dev)
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        h2d += 0 if a.forward_only else hg.numel() * hg.element_size()
        d2h = sum(o.numel() * o.element_size() for o in outs)
        e2e = {"value": pairs_job * iters / e2e_s, "unit": "pair-timestep updates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s}

    # plain FP64 GPU solve of the same step, and the tensor-core / structured variants
    fp64, variants, optimizer, pipeline, convergence = None, [], None, None, None
    if not a.no_compare and rank == 0:
        v64 = _variant(insts, nd, iters, a, "fp64", "dense", 0, dev, stream, flush, None, None, reps=5)
        p64, r64 = v64.pop("_pos"), v64.pop("_res")
        fp64 = dict(v64, value=pairs * iters / (v64["ms_per_step"] * 1e-3),
                    chosen_max_position_error_m=_max_pos_err(chosen_pos, p64),
                    chosen_max_final_residual_diff_m=float(np.abs(r[:, 1] - r64[:, 1]).max()),
                    frac_instances_resid_le_1e3=float(np.mean(r64[:, 1] <= 1e-3)),
                    chosen_speedup=v64["ms_per_step"] / ms_step)
        optimizer = _optimizer(insts, nd, iters, a, dev, stream, flush, pairs)
        pipeline = _pipeline(a, dev, stream)
        convergence = _convergence(insts, nd, a, dev, stream)
        for prec, proj, nr in [("fp32", "structured" if a.proj == "dense" else "dense", 0), ("tf32", "dense", 2),
                               ("bf16x3", "dense", 1), ("bf16", "dense", 5)]:
            if (prec, proj, nr) == (a.precision, a.proj, a.n_refine):
                continue
            v = _variant(insts, nd, iters, a, prec, proj, nr, dev, stream, flush, p64, r64)
            v.pop("_pos"), v.pop("_res")
            variants.append(v)

    configs = sweep = None
    if not a.no_compare and not a.no_configs and rank == 0:
        configs = other_configs(dev, stream, flush, peaks)
        if a.config == 2 and world == 1:
            sweep = batch_sweep(dev, stream, flush, peaks)

    if rank == 0:
        peak_alu = peaks["fp32_tflops"]
        names = ["k_forward", "k_residual", "k_backward"]
        kernels = {}
        for k, nm in enumerate(names):
            if a.forward_only and nm == "k_backward":
                continue
            ms = statistics.mean(x[k] for x in kts)
            fl, mufu = algorithmic_flops(insts, iters, a.proj, nm, a.ckpt_every)
            ach = fl / (ms * 1e-3) / 1e12
            kernels[nm] = {"ms": ms, "share": ms / ms_step, "algorithmic_gflop": fl / 1e9, "achieved_tflops": ach,
                           "frac": ach / peak_alu, "rsqrt_g": mufu / 1e9,
                           "mufu_frac": (mufu / (ms * 1e-3) / 1e12 / peaks["mufu_tops"]) if peaks["mufu_tops"] else None}
        dom = max(kernels, key=lambda k: kernels[k]["ms"])
        traffic, traffic_src = profiled_traffic(dom, cfg.name, a.precision, a.proj)
        line = {
            "metric": METRIC,
            "value": value, "unit": "pair-timestep updates/s", "n_gpus": world, "steps": a.steps,
            "warmup": max(a.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong" if a.shard_batch else "weak",
            "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32", "data": "synthetic",
            "config": _config(cfg, insts, iters, a, {
                "precision": a.precision, "projection": a.proj, "n_refine": a.n_refine,
                "l2": "flushed between steps (256 MB write)",
                "cluster_ctas_per_instance": solver.launch()[0], "threads_per_cta": solver.launch()[1],
                "autotune": tune,
                "parallelism": ("one batch split over the ranks (shard.balance)" if a.shard_batch else
                                "one batch per rank") if world > 1 else "single GPU"}),
            "roofline": {"bound": "alu", "achieved": kernels[dom]["achieved_tflops"], "peak": peak_alu,
                         "unit": "TFLOP/s", "frac": kernels[dom]["frac"], "traffic": traffic,
                         "traffic_source": traffic_src, "kernel": dom,
                         "kernel_ms": kernels[dom]["ms"],
                         "algorithmic": "per pair or obstacle row %d flops (2-D) / %d (3-D) + 1 rsqrt; positions once "
                                        "and the W' aggregation twice at 2 n_d n H n_xi; 2 n_d per box entry; "
                                        "6 n_d N; projection 4 n_d n n_xi^2 (Kronecker) or 2 n_d N^2 (dense)"
                                        % (ROW_FLOPS[2], ROW_FLOPS[3]),
                         "peak_source": peaks["source"], "sms": peaks["sms"],
                         "measured_peaks": {"fp32_tflops": peaks["fp32_tflops"], "fp64_tflops": peaks["fp64_tflops"],
                                            "mufu_trsqrt_per_s": peaks["mufu_tops"]}},
            "kernels": kernels,
            "clocks": clk,
            "gpu_launches": step.launches() * a.steps,
            "graph": graph,
            "result": {"final_max_residual_m_median": float(np.median(r[:, 1])),
                       "frac_instances_resid_le_1e-3": float(np.mean(r[:, 1] <= 1e-3)),
                       "iterations_to_1e-3": [int(x) for x in r[:, 3]]},
            "setup": {"sf_create_ms": setup_ms,
                      "what": "one-time per batch: FP64 factorisation of every distinct shape on the GPU, "
                              "launch plan, FP32 copies (outside the timed step)"},
        }
        if e2e:
            line["e2e"] = e2e
        if fp64:
            line["fp64_gpu"] = fp64
        if variants:
            line["variants"] = variants
        if optimizer:
            line["trajectory_optimizer"] = optimizer
        if pipeline:
            line["pipeline"] = pipeline
        if convergence:
            line["convergence"] = convergence
        if configs:
            line["configs"] = configs
        if sweep:
            line["batch_sweep"] = sweep
        if not a.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(insts, iters, a.forward_only)
        line["summary"] = summary_of(line, configs)   # last, so a truncated tail still shows it
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    solver.close()


if __name__ == "__main__":
    main()
