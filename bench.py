#!/usr/bin/env python3
"""Benchmark of the MDS hot path on GB300: pairs/s and HMC leapfrog steps/s
(log-likelihood + gradient, Eq. (2) and (9) of arXiv:1905.04582) at the
paper-scale size N = 5392, D = 2.

One step = one HMC iteration on the device: momentum draw, 20 leapfrog steps
(each one fused pair pass over all M = N(N-1)/2 pairs plus its reduction and
update), energies and the Metropolis decision -- one CUDA-graph launch.
Inputs are resident in HBM before timing; the L2 (126 MB) is flushed between
timed steps (Y is 58 MB, so within a step later passes read it from L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores on the same
workload (each step: one likelihood + gradient evaluation).
Under torchrun (N > 1) every rank advances its own independent chain
("replicas only": the HMC path has no data exchange); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_LEAPFROG = 20
METRIC = "pairs/sec and HMC leapfrog steps/sec (loglik+grad) at N=5392, % HBM roofline vs FP64 path"
WORKLOAD = "paper-scale N=5392 D=2, 6-component Gaussian mixture, sigma=0.3, FP32 Y (synthetic)"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def reduce_max(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_rate(wl, evals, nthreads=1):
    """Oracle (as it stands) likelihood + gradient on the host: pairs/s."""
    import oracle
    x64 = wl.x_eval.astype(np.float64)
    t0 = time.perf_counter()
    for _ in range(evals):
        oracle.loglik(wl.y_packed, x64, wl.sigma, nthreads=nthreads)
        oracle.gradient(wl.y_packed, x64, wl.sigma, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return evals * wl.m / dt, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1905_04582_gb300 import workloads as W
    wl = W.paper_scale()
    import oracle
    oracle.build()
    x64 = wl.x_eval.astype(np.float64)
    for _ in range(args.warmup):
        oracle.loglik(wl.y_packed, x64, wl.sigma)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.loglik(wl.y_packed, x64, wl.sigma)
        oracle.gradient(wl.y_packed, x64, wl.sigma)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * wl.m / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": wl.n, "d": wl.d, "pairs": wl.m,
                   "step": "one log-likelihood + gradient evaluation of the serial FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full evaluations at N=5392 (L and dL/dX)"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1905_04582_gb300 import build as B
    from paper_1905_04582_gb300 import workloads as W
    from paper_1905_04582_gb300.mds import MDS
    B.build()

    wl = W.paper_scale()
    stream = torch.cuda.Stream(device=dev)
    model = MDS(wl.n, wl.d, "fp32c", stream=stream)
    model.set_data(wl.y_packed)
    model.set_locations(wl.x_eval)
    model.set_sigma(wl.sigma)
    eps = args.eps
    seed = 1234 + rank

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(float(np.random.rand()))

    # warm-up (autotune, graph capture, clocks)
    model.log_likelihood()
    model.hmc(max(args.warmup, 1), N_LEAPFROG, eps, seed=seed)

    # timed region: K HMC iterations, L2 flushed before each (untimed)
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    acc_total = 0
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush_l2()
            ev_s[k].record(stream)
            acc, dh, stats = model.hmc(1, N_LEAPFROG, eps, seed=seed)
            ev_e[k].record(stream)
            acc_total += int(acc.sum())
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in zip(ev_s, ev_e)]
    dev_ms = sum(step_ms)
    dev_ms_max = reduce_max(dev_ms, world)

    # the same K iterations again with CUDA events bracketing every pair-pass
    # launch inside the graph: the dominant kernel's average duration
    model.set_profiling(True)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush_l2()
        model.hmc(1, N_LEAPFROG, eps, seed=seed)
    torch.cuda.synchronize()
    n_pass, pass_ms = model.pass_time()
    model.set_profiling(False)

    pairs_per_step = N_LEAPFROG * wl.m
    value = world * args.steps * pairs_per_step / (dev_ms_max / 1e3)
    lf_steps = world * args.steps * N_LEAPFROG / (dev_ms_max / 1e3)

    # roofline of the dominant kernel (the fused pair pass), timed live
    peak, peak_kind = load_peaks()
    m_pairs, y_bytes = model.problem_size()
    pass_avg_ms = pass_ms / max(n_pass, 1)
    alg_bytes = 4.0 * m_pairs  # one FP32 y_ij per pair per pass
    achieved = alg_bytes / (pass_avg_ms / 1e3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "pair_pass_traffic.json")
    if os.path.exists(tr_path):
        try:
            with open(tr_path) as f:
                tr = json.load(f)
            if tr.get("kernel_rev") == "v1" and tr.get("n") == wl.n:
                traffic = tr.get("bytes_per_launch")
        except Exception:
            traffic = None

    # the plain FP64 GPU path on the same data (one pass, timed alone)
    with MDS(wl.n, wl.d, "fp64", stream=stream) as m64:
        m64.set_data(wl.y_packed)
        m64.set_locations(wl.x_eval)
        m64.set_sigma(wl.sigma)
        ms64 = m64.time_pass(5)
    ms32 = model.time_pass(20)

    # end to end through the C ABI with host buffers: X in, one HMC
    # iteration, X and the statistics out
    x_host = torch.from_numpy(wl.x_eval.copy()).pin_memory()
    x_out = torch.empty_like(x_host).pin_memory()
    e2e_steps = max(3, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        model.set_locations(x_host)
        model.hmc(1, N_LEAPFROG, eps, seed=seed)
        model.get_locations(out=x_out)
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    e2e_value = world * e2e_steps * pairs_per_step / e2e_s

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rate, secs = cpu_oracle_rate(wl, args.cpu_evals)
        cpu = {"value": rate, "unit": "pairs/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_evals} serial evaluations of L and dL/dX at N=5392 ({secs:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": wl.n, "d": wl.d, "pairs": m_pairs, "sigma": wl.sigma,
                       "precision": "FP32 per pair, compensated FP32 partials reduced in FP64",
                       "step": f"one HMC iteration: {N_LEAPFROG} leapfrog steps (fused L+grad pass each) + Metropolis",
                       "eps": eps, "strip": model.get_strip(),
                       "l2": "flushed (512 MB write) between timed steps; Y (58 MB) stays L2-resident within a step",
                       "parallelism": f"replicas x{world}"},
            "leapfrog_steps_per_s": lf_steps,
            "accept_rate": acc_total / args.steps,
            "hbm_fraction_of_pairs_rate": value * 4.0 / 1e9 / peak,
            "pass_alone": {"fp32c_ms": ms32, "fp64_ms": ms64, "fp32c_pairs_per_s": m_pairs / (ms32 / 1e3),
                           "fp64_pairs_per_s": m_pairs / (ms64 / 1e3), "speedup_vs_fp64": ms64 / ms32},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": f"{peak_kind} hbm_gbs",
                         "kernel": "pair_f32_kernel<2>", "launches_timed": n_pass,
                         "avg_launch_ms": pass_avg_ms, "algorithmic_bytes_per_launch": alg_bytes},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": wl.n * wl.d * 4,
                    "d2h_bytes_per_step": wl.n * wl.d * 4 + 8 + 8 + 4,
                    "note": "mds_set_locations(host X) + mds_hmc(1 iteration) + mds_get_locations(host)"},
            "gpu_launches": args.steps * (2 + 2 * N_LEAPFROG),
            "wall_s": wall,
        }
        clk = clocks.summary()
        if clk is not None:
            line["clocks"] = clk
        print(json.dumps(line), flush=True)
    model.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_pass_only(args):
    """Time the fused pass alone (likelihood + gradient, no HMC) at a chosen
    size: the command the kernel profiles under profiles/ were taken with."""
    import torch
    from paper_1905_04582_gb300 import build as B
    from paper_1905_04582_gb300 import workloads as W
    from paper_1905_04582_gb300.mds import MDS
    B.build()
    torch.cuda.set_device(0)
    if args.n == 5392:
        wl = W.paper_scale(d=args.d)
    else:
        wl = W.make(f"mixture N={args.n} D={args.d}", args.n, args.d, 0.3, 5, 0.3, mixture=(6, 0.3))
    with MDS(wl.n, wl.d, args.precision, strip=args.strip) as m:
        m.set_data(wl.y_packed)
        m.set_locations(wl.x_eval)
        m.set_sigma(wl.sigma)
        ms = m.time_pass(args.reps)
        print(json.dumps({"pass_only": True, "n": wl.n, "d": wl.d, "precision": args.precision,
                          "strip": m.get_strip(), "ms_per_pass": ms, "pairs_per_s": wl.m / (ms / 1e3),
                          "alg_gb_per_s": 4.0 * wl.m / (ms / 1e3) / 1e9}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--eps", type=float, default=2e-4)
    ap.add_argument("--cpu-evals", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pass-only", action="store_true", help="time the fused pass alone (profiling runs)")
    ap.add_argument("--n", type=int, default=5392)
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--strip", type=int, default=None)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    if args.pass_only:
        return run_pass_only(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
