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


SM_MAX_MHZ = 2070.0


def fp32_ops_per_pair(d):
    """FP32 lane operations per pair in pair2_f32 (pair_math.cuh), an FMA
    counting once: per coordinate the exact-split differences (3), squares
    (1), cross term (2) and the two gradient accumulations (2); fixed: d^2,
    residual (2), half inverse, corrected e (2), exp argument, Mills ratio
    P and D (3 + 3), D Phi, 1/Phi, phi/Phi, log-product, e^2, m delta, w (2),
    w/delta."""
    return 8 * d + 22


PAIR_KERNEL_SOURCES = ("pair_kernel.cu", "pair_math.cuh", "mds_internal.h", "mills_ratio_coeffs.h")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "pair_f32_kernel_N5392_D2_traffic.txt")


def pair_kernel_sha256():
    """Hash of the sources the FP32C pair kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for name in PAIR_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1905_04582_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_traffic(n, d):
    """DRAM bytes per launch of the pair pass from the committed ncu capture
    (`key: value` lines), if it was taken on the current kernel source at
    this N and D; else None."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as f:
            for ln in f:
                if ":" in ln and not ln.startswith("#"):
                    k, v = ln.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sha256") == pair_kernel_sha256() and int(kv.get("n", -1)) == n \
                and int(kv.get("d", -1)) == d:
            return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


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
    """Max of a per-rank number over the ranks (NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, seconds, world):
    """Whole-job throughput of `world` independent replicas: all ranks' units
    over the slowest rank's time (max over ranks)."""
    return world * units_per_rank / reduce_max(seconds, world)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def pass_distribution(model, wl, flush_l2, stream, n_warm=100, n_cold=20):
    """Pair-kernel launch times (CUDA events around the launch): p10 / p50 /
    p90 over n_warm back-to-back evaluations (Y L2-resident) and over n_cold
    evaluations each after an L2 flush (Y from HBM)."""
    import torch
    x_dev = torch.from_numpy(wl.x_eval.copy()).to(device=torch.device("cuda", torch.cuda.current_device()))

    def run(n, cold):
        out = []
        for _ in range(n):
            if cold:
                flush_l2()
            model.set_profiling(True)  # restarts the launch timer
            model.set_locations(x_dev)  # invalidates the cached pass (Y untouched)
            model.log_likelihood()
            out.append(model.pass_time()[1])
        model.set_profiling(False)
        q = np.quantile(np.array(out) * 1e3, [0.1, 0.5, 0.9])
        return {"p10": float(q[0]), "p50": float(q[1]), "p90": float(q[2]), "n": n}

    torch.cuda.synchronize()
    return {"warm": run(n_warm, False), "cold": run(n_cold, True)}


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

    # timed region: K HMC iterations queued back to back on the stream (no
    # host round trip between them), each bracketed by its own CUDA events,
    # L2 flushed before each one outside the brackets
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush_l2()
            ev_s[k].record(stream)
            model.hmc_enqueue(1, N_LEAPFROG, eps, seed=seed)
            ev_e[k].record(stream)
        acc, dh, stats = model.hmc_collect()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    acc_total = int(acc.sum())
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
    value = replica_rate(args.steps * pairs_per_step, dev_ms / 1e3, world)
    lf_steps = world * args.steps * N_LEAPFROG / (dev_ms_max / 1e3)

    # roofline of the dominant kernel (the fused pair pass), timed live.  It
    # is bound by the FP32 pipe: FP32_OPS_PER_PAIR lane operations per pair
    # (counted from the kernel source; an FMA counts once) against
    # SMs x 128 FP32 lanes x the SM clock.  The HBM view (4 B of Y per pair
    # against the measured copy bandwidth) is reported beside it.
    hbm_peak, peak_kind = load_peaks()
    m_pairs, y_bytes = model.problem_size()
    pass_avg_ms = pass_ms / max(n_pass, 1)
    alg_bytes = 4.0 * m_pairs  # one FP32 y_ij per pair per pass
    achieved_gbs = alg_bytes / (pass_avg_ms / 1e3) / 1e9
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = clocks.summary()
    sm_mhz = (clk or {}).get("sm_max_mhz") or SM_MAX_MHZ
    alu_peak = sm_count * 128 * sm_mhz * 1e6 / 1e12  # TFP32-op/s
    ops = fp32_ops_per_pair(wl.d)
    alu_achieved = m_pairs * ops / (pass_avg_ms / 1e3) / 1e12
    traffic = kernel_traffic(wl.n, wl.d)

    # the plain FP64 GPU path on the same data (one pass, timed alone)
    with MDS(wl.n, wl.d, "fp64", stream=stream) as m64:
        m64.set_data(wl.y_packed)
        m64.set_locations(wl.x_eval)
        m64.set_sigma(wl.sigma)
        ms64 = m64.time_pass(5)
    ms32 = model.time_pass(20)
    pass_dist = pass_distribution(model, wl, flush_l2, stream)

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
    e2e_value = replica_rate(e2e_steps * pairs_per_step, time.perf_counter() - t0, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rate, secs = cpu_oracle_rate(wl, args.cpu_evals)
        cpu = {"value": rate, "unit": "pairs/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_evals} serial evaluations of L and dL/dX at N=5392 ({secs:.1f} s)"}
        ncores = os.cpu_count() or 1
        rate_mt, secs_mt = cpu_oracle_rate(wl, args.cpu_evals, nthreads=ncores)
        cpu["all_cores"] = {"value": rate_mt, "unit": "pairs/s", "cores": ncores, "kind": "oracle (OpenMP rows)",
                            "sample": f"{args.cpu_evals} evaluations of L and dL/dX at N=5392 ({secs_mt:.1f} s)"}

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
            "hbm_fraction_of_pairs_rate": value * 4.0 / 1e9 / hbm_peak,
            "pass_alone": {"fp32c_ms": ms32, "fp64_ms": ms64, "fp32c_pairs_per_s": m_pairs / (ms32 / 1e3),
                           "fp64_pairs_per_s": m_pairs / (ms64 / 1e3), "speedup_vs_fp64": ms64 / ms32,
                           "pair_kernel_warm_us": pass_dist["warm"], "pair_kernel_cold_us": pass_dist["cold"]},
            "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFP32-op/s",
                         "frac": alu_achieved / alu_peak, "traffic": traffic,
                         "peak_kind": f"derived: {sm_count} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz",
                         "ops_per_pair": ops, "kernel": f"pair_f32_kernel<{wl.d}>", "launches_timed": n_pass,
                         "avg_launch_ms": pass_avg_ms, "pairs_per_launch": m_pairs,
                         "hbm_view": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                                      "frac": achieved_gbs / hbm_peak, "peak_kind": f"{peak_kind} hbm_gbs",
                                      "algorithmic_bytes_per_launch": alg_bytes}},
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


def _alu_peak_tflops():
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * SM_MAX_MHZ * 1e6 / 1e12


def run_sweep(args):
    """The scale sweep (N = 20000, 50000; D = 2, 6; FP32C, autotuned strip):
    one JSON line per size with the pass time and its HBM and ALU fractions,
    Y (0.8 / 5.0 GB) far larger than L2, so every pass streams it from HBM."""
    import torch
    from paper_1905_04582_gb300 import build as B
    from paper_1905_04582_gb300 import workloads as W
    from paper_1905_04582_gb300.mds import MDS
    B.build()
    torch.cuda.set_device(0)
    hbm_peak, peak_kind = load_peaks()
    alu_peak = _alu_peak_tflops()
    for n, d in ((20000, 2), (20000, 6), (50000, 2), (50000, 6)):
        wl = W.scale_sweep(n, d)
        with MDS(wl.n, wl.d, "fp32c") as m:
            m.set_data(wl.y_packed)
            m.set_locations(wl.x_eval)
            m.set_sigma(wl.sigma)
            ms = m.time_pass(args.reps)
            strip = m.get_strip()
        line = {"sweep": True, "workload": wl.name, "n": n, "d": d, "pairs": wl.m, "strip": strip,
                "ms_per_pass": ms, "pairs_per_s": wl.m / (ms / 1e3),
                "hbm": {"achieved_gbs": 4.0 * wl.m / (ms / 1e3) / 1e9, "peak_gbs": hbm_peak,
                        "frac": 4.0 * wl.m / (ms / 1e3) / 1e9 / hbm_peak, "peak_kind": peak_kind},
                "alu": {"achieved_tflops": wl.m * fp32_ops_per_pair(d) / (ms / 1e3) / 1e12, "peak_tflops": alu_peak,
                        "frac": wl.m * fp32_ops_per_pair(d) / (ms / 1e3) / 1e12 / alu_peak}}
        if n == 20000 and d == 2:
            with MDS(wl.n, wl.d, "fp64") as m64:
                m64.set_data(wl.y_packed)
                m64.set_locations(wl.x_eval)
                m64.set_sigma(wl.sigma)
                ms64 = m64.time_pass(2)
            line["fp64_ms_per_pass"] = ms64
            line["speedup_vs_fp64"] = ms64 / ms
        print(json.dumps(line), flush=True)
        del wl
    return 0


def run_batch(args):
    """Batched datasets x chains (N = 1600, 1500, 1300, 992; 8 chains each):
    pair evaluations per second of one batched pass for all 32 chains, and
    HMC leapfrog steps per second over all chains."""
    import torch
    from paper_1905_04582_gb300 import build as B
    from paper_1905_04582_gb300 import workloads as W
    from paper_1905_04582_gb300.mds import Batch
    B.build()
    torch.cuda.set_device(0)
    ds = W.batch_datasets()
    chains = 8
    b = Batch([w.n for w in ds], 2, [chains] * len(ds))
    for k, w in enumerate(ds):
        b.set_data(k, w.y_packed)
        b.set_sigma(k, w.sigma)
        for j in range(chains):
            b.set_locations(k, j, w.x_eval)
    ms = b.time_pass(args.reps)
    evals = sum(w.m for w in ds) * chains
    b.hmc(2, N_LEAPFROG, [5e-4] * len(ds), seed=1)  # warm-up (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    acc, dh = b.hmc(args.steps, N_LEAPFROG, [5e-4] * len(ds), seed=2)
    wall = time.perf_counter() - t0
    alu_peak = _alu_peak_tflops()
    print(json.dumps({"batch": True, "datasets": [w.n for w in ds], "chains_per_dataset": chains,
                      "strip": b.get_strip(), "ms_per_pass": ms, "pair_evals_per_pass": evals,
                      "pair_evals_per_s": evals / (ms / 1e3),
                      "alu": {"achieved_tflops": evals * fp32_ops_per_pair(2) / (ms / 1e3) / 1e12,
                              "peak_tflops": alu_peak,
                              "frac": evals * fp32_ops_per_pair(2) / (ms / 1e3) / 1e12 / alu_peak},
                      "hmc_iterations": args.steps, "leapfrog_steps_per_s_all_chains":
                          args.steps * N_LEAPFROG * len(ds) * chains / wall,
                      "accept_rate": float(np.mean(acc)), "wall_s": wall}), flush=True)
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
    ap.add_argument("--kernel-hash", action="store_true", help="print the pair kernel's source hash and exit")
    ap.add_argument("--sweep", action="store_true", help="the N = 20000 / 50000 scale sweep (pass only)")
    ap.add_argument("--batch", action="store_true", help="batched datasets x chains")
    args = ap.parse_args()
    if args.kernel_hash:
        print(pair_kernel_sha256())
        return 0
    if args.sweep:
        return run_sweep(args)
    if args.batch:
        return run_batch(args)
    if args.pass_only:
        return run_pass_only(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
