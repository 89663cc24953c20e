#!/usr/bin/env python
"""Benchmark of the batched Safety-Filter solve.

One step = one full SF solve of a batch (every iteration of T on every instance,
plus the FP64 residual check of the result).  Default workload: 32 instances of
16 disc robots in a 15 x 15 m 2D map with 20 obstacles, horizon 100, 200
iterations (seeded synthetic instances from ``sfgen``).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own batch (seeds offset by rank): weak scaling,
no collective on the data path; the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sfgen  # noqa: E402

RHO = 0.3
SM_COUNT_B300 = 148
FP32_LANES_PER_SM = 128


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", type=int, default=2)
    p.add_argument("--precision", default="fp32")
    p.add_argument("--proj", default="dense")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--compare-fp64", action="store_true", help="also time the plain FP64 GPU solve")
    p.add_argument("--no-autotune", action="store_true")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(cid, rank=0):
    cfg = sfgen.CONFIGS[cid]
    insts = sfgen.make_batch(cid, start=rank * cfg.B)
    pairs, obs = sfgen.batch_stats(insts)
    return cfg, insts, pairs, obs


def algorithmic_flops(insts, iters, proj):
    """FP32 operations of one forward launch counted at the algorithmic minimum:
    per pair or obstacle row 2 n_d + 1 (line of sight, scaled squared norm), per
    (robot, timestep) 2 n_d box tests, positions and W' aggregation 2 n_d n H n_xi each,
    lambda / correction 6 n_d N, projection 2 n_d N^2 (dense) or 4 n_d n n_xi^2."""
    tot = 0.0
    for i in insts:
        nd, n, H, nxi, no = i["n_d"], i["n"], i["H"], i["n_xi"], i["n_obs"]
        N = n * nxi
        rows = (n * (n - 1) // 2 + n * no) * H
        per = rows * (2 * nd + 1) + 2 * nd * n * H + 4 * nd * n * H * nxi + 6 * nd * N
        per += 2 * nd * N * N if proj == "dense" else 4 * nd * n * nxi * nxi
        tot += per * iters
    return tot


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


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(insts, iters, budget_s=15.0):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample of the batch."""
    import oracle
    oracle.load()
    cores = os.cpu_count() or 1
    # grow the sample until it costs about budget_s (never more than the whole batch)
    t0 = time.perf_counter()
    oracle.solve_batch(insts[:1], iters, rho=RHO)
    one = max(time.perf_counter() - t0, 1e-3)
    k = int(max(1, min(len(insts), budget_s / one * cores * 0.7)))
    sample = insts[:k]
    t0 = time.perf_counter()
    oracle.solve_batch(sample, iters, rho=RHO)
    dt = time.perf_counter() - t0
    pairs, _ = sfgen.batch_stats(sample)
    return {"value": pairs * iters / dt, "unit": "pair-timestep updates/s", "cores": cores, "kind": "oracle",
            "sample": "%d of %d instances x %d iterations, FP64, OpenMP over instances (%.1f s)" % (k, len(insts), iters, dt)}


def run_reference(a):
    """The oracle as the reference arm: rank 0 only, host cores, bounded sample per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    cfg, insts, pairs_all, _ = workload(a.config)
    iters = cfg.iters
    oracle.load()
    t0 = time.perf_counter()
    oracle.solve_batch(insts[:1], iters, rho=RHO)
    one = max(time.perf_counter() - t0, 1e-3)
    cores = os.cpu_count() or 1
    k = int(max(1, min(len(insts), 4.0 / one * cores * 0.7)))  # about 4 s of CPU work per step
    sample = insts[:k]
    pairs, _ = sfgen.batch_stats(sample)
    for _ in range(a.warmup):
        oracle.solve_batch(sample, iters, rho=RHO)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.solve_batch(sample, iters, rho=RHO)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = pairs * iters * a.steps / tot
    desc = "%d of %d instances x %d iterations per step, FP64 oracle, OpenMP over instances" % (k, len(insts), iters)
    line = {"impl": "reference", "metric": "SF pair-timestep updates/s", "value": value,
            "unit": "pair-timestep updates/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * tot / a.steps * len(insts) / k, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name, "instances": len(insts), "robots": cfg.n[0], "obstacles": cfg.n_obs[0],
                       "horizon": cfg.H[0], "iterations": iters, "n_d": cfg.n_d},
            "cpu_baseline": {"value": value, "unit": "pair-timestep updates/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "pair-timestep updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = args_()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import torch.distributed as dist

    from paper_2510_09204_b300 import SFSolver

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, insts, pairs, obs = workload(a.config, rank)
    iters = cfg.iters
    nd = cfg.n_d
    solver = SFSolver(insts, nd, 11, rho=RHO, precision=a.precision, proj=a.proj, max_iters=iters)
    data = solver.pack(insts, device=dev)
    xo = torch.empty_like(data["xi"])
    lo = torch.empty_like(data["xi"])
    res = torch.empty((len(insts), 4), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2
    tune = None
    if not a.no_autotune:
        t0 = time.perf_counter()
        c, t, ms = solver.autotune(data, data["xi"], iters, reps=2)
        tune = {"cluster": c, "threads": t, "best_ms": ms, "tuning_s": time.perf_counter() - t0}
    solver.profile(True)

    def step():
        solver.solve(data, data["xi"], iters, xi_out=xo, lam_out=lo, resid=res, stream=stream)

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
    assert (solver.status() == 0).all(), "non-finite iterates"

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    t_start = time.time()
    times, fwd_ms = [], []
    for _ in range(a.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        fwd_ms.append(solver.kernel_times()[0])
    barrier()
    clocks.window(t_start, time.time())
    clk = clocks.stop()
    tot_ms = sum(times)
    if world > 1:
        t = torch.tensor([tot_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    ms_step = tot_ms / a.steps
    value = pairs * iters * world / (ms_step * 1e-3)

    # end to end through the public API from pinned host memory
    e2e = None
    if not a.no_e2e:
        host = {k: v.cpu().pin_memory() for k, v in data.items()}
        outp = (torch.empty(xo.shape, dtype=xo.dtype, pin_memory=True),
                torch.empty(res.shape, dtype=res.dtype, pin_memory=True))
        for _ in range(2):
            solver.solve_host(host, iters, outp)
        barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            solver.solve_host(host, iters, outp)
        barrier()
        e2e_s = (time.perf_counter() - t0) / a.steps
        if world > 1:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = outp[0].numel() * outp[0].element_size() + outp[1].numel() * outp[1].element_size()
        e2e = {"value": pairs * iters * world / e2e_s, "unit": "pair-timestep updates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s}

    # plain FP64 GPU solve of the same batch (the comparison the metric names)
    fp64 = None
    if a.compare_fp64 and rank == 0:
        s64 = SFSolver(insts, nd, 11, rho=RHO, precision="fp64", proj="dense", max_iters=iters)
        d64 = s64.pack(insts, device=dev)
        if not a.no_autotune:
            s64.autotune(d64, d64["xi"], iters, reps=1)
        s64.solve(d64, d64["xi"], iters)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, r64 = s64.solve(d64, d64["xi"], iters, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1)
        r32 = res.cpu().numpy()
        r64 = r64.cpu().numpy()
        fp64 = {"ms_per_batch": ms64, "value": pairs * iters / (ms64 * 1e-3), "launch": s64.launch(),
                "max_abs_final_residual_diff_m": float(np.abs(r32[:, 1] - r64[:, 1]).max()),
                "frac_instances_resid_le_1e-3": float(np.mean(r64[:, 1] <= 1e-3))}

    if rank == 0:
        peaks = measured_peaks()
        sm_max = float(peaks.get("sm_max_mhz", 2032.0))
        peak_alu = SM_COUNT_B300 * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        fwd_avg = statistics.mean(fwd_ms)
        ach = algorithmic_flops(insts, iters, a.proj) / (fwd_avg * 1e-3) / 1e12
        r = res.cpu().numpy()
        line = {
            "metric": "SF pair-timestep updates/s (ms/batch in ms_per_step)",
            "value": value, "unit": "pair-timestep updates/s", "n_gpus": world, "steps": a.steps,
            "warmup": max(a.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": cfg.name, "instances": len(insts), "robots": cfg.n[0], "obstacles": cfg.n_obs[0],
                       "horizon": cfg.H[0], "iterations": iters, "n_d": nd, "n_xi": 11, "rho": RHO,
                       "precision": a.precision, "projection": a.proj, "l2": "flushed between steps (256 MB write)",
                       "cluster_ctas_per_instance": solver.launch()[0], "threads_per_cta": solver.launch()[1],
                       "autotune": tune,
                       "parallelism": "instances sharded by rank" if world > 1 else "single GPU"},
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak_alu, "unit": "TFLOP/s", "frac": ach / peak_alu,
                         "traffic": None, "kernel": "k_forward", "kernel_ms": fwd_avg,
                         "peak_source": "148 SMs x 128 FP32 lanes x 2 x sm_max_mhz %.0f (derived)" % sm_max},
            "clocks": clk,
            "gpu_launches": 2 * a.steps,
            "result": {"final_max_residual_m_median": float(np.median(r[:, 1])),
                       "frac_instances_resid_le_1e-3": float(np.mean(r[:, 1] <= 1e-3))},
        }
        if e2e:
            line["e2e"] = e2e
        if fp64:
            line["fp64_gpu"] = fp64
        if not a.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(insts, iters)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    solver.close()


if __name__ == "__main__":
    main()
