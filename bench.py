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
import math
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


def fp32_ops_per_pair(d, far_frac=0.0, chunked=True):
    """FP32 lane operations per pair that the pass executes, an FMA counting
    once.  Chunked pass (chunk_kernel.cu): per coordinate the exact-split
    differences (3), the square (1), the cross term (2) and the two gradient
    accumulations (2); then d^2, the residual (2), the corrected e (2), e^2
    and the gradient weight (1): 8 D + 7 where every pair of the warp's block
    lies at z >= 8 (Phi terms skipped); with Phi: the exp argument, the Mills
    ratio P and D (3 + 3), D Phi, 1/Phi, phi/Phi, the log-product, m delta and
    one more for the weight: 8 D + 20.  The strip pass (pair_math.cuh) takes
    8 D + 9 and 8 D + 22.  far_frac is the fraction of warp blocks that took
    the far body."""
    far, near = (8 * d + 7, 8 * d + 20) if chunked else (8 * d + 9, 8 * d + 22)
    return (1.0 - far_frac) * near + far_frac * far


PAIR_KERNEL_SOURCES = ("pair_kernel.cu", "chunk_kernel.cu", "pair_math.cuh", "mills_ratio_coeffs.h")
# the part of mds_internal.h the pair kernel is compiled from: the tile
# geometry through the end of its argument struct, and the error bits
PAIR_KERNEL_INTERNAL = (("// Tile geometry of the pair pass.", "cudaError_t launch_pair_batch"),)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "pair_chunk_kernel_N5392_D2_traffic.txt")


def pair_kernel_sha256():
    """Hash of the sources the FP32C pair kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1905_04582_gb300", "csrc")
    for name in PAIR_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    text = open(os.path.join(csrc, "mds_internal.h")).read()
    for begin, end in PAIR_KERNEL_INTERNAL:
        i, j = text.index(begin), text.index(end)
        h.update(text[i:j].encode())
    return h.hexdigest()


# mds_get_pass_shape kinds: strips, chunks per slot, a chunk count, and the
# chunks of one CTA per SM run as groups of four warps
PASS_KINDS = ["strips", "chunks", "chunks", "sm-chunks"]


def kernel_traffic(n, d, kind="chunks"):
    """DRAM bytes per launch of the pair pass from the committed ncu capture
    (`key: value` lines), if it was taken on the current kernel source at
    this N, D and pass kind (strips / chunks); else None."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as f:
            for ln in f:
                if ":" in ln and not ln.startswith("#"):
                    k, v = ln.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sha256") == pair_kernel_sha256() and int(kv.get("n", -1)) == n \
                and int(kv.get("d", -1)) == d and kv.get("shape", "").split(" ")[0] == kind:
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


def eps_pilot(model, eps0, seed, target=0.65, rounds=8, iters=10):
    """A short pilot that picks the leapfrog step for acceptance ~ target
    (section 2.3 leaves it to the user): blocks of `iters` HMC iterations, the
    step moved on a log scale by the acceptance of each block (the gain
    shrinking), starting from the evaluation point (the pilot also burns
    the chain in).  Returns the step and the (eps, acceptance) history."""
    eps = eps0
    hist = []
    for r in range(rounds):
        acc, _, _ = model.hmc(iters, N_LEAPFROG, eps, seed=seed + 7919 * (r + 1))
        a = float(np.mean(acc))
        hist.append({"eps": eps, "accept": a})
        eps *= math.exp(2.0 * (a - target) / math.sqrt(r + 1))
    return eps, hist


def parity_entry(model, wl, nthreads):
    """Errors of the benchmarked path against the FP64 oracle at the model's
    current locations (the bench configuration: locality order, tuned pass
    shape, Phi cut-off): relative errors of L, sum r and dL/dsigma, max and
    p99.9 of the per-coordinate gradient error, and the coordinates that pass
    only through the cancellation / rounding branches (stated tolerances)."""
    import oracle
    oracle.build()
    x = model.get_locations(dtype=np.float64)  # the FP32 state, widened exactly
    ll, g, ds = model.gradient()
    _, sr = model.log_likelihood()
    ll_r, sr_r = oracle.loglik(wl.y_packed, x, wl.sigma, nthreads=nthreads)
    g_r, s_abs, s_sq = oracle.gradient(wl.y_packed, x, wl.sigma, nthreads=nthreads, with_abs=True, with_sq=True)
    ds_r = oracle.dsigma(wl.y_packed, x, wl.sigma, nthreads=nthreads)
    u, tol = 2.0 ** -24, 1e-5
    err = np.abs(g - g_r)
    rel = err / np.maximum(np.abs(g_r), 1e-300)
    rel_ok = err <= tol * np.abs(g_r)
    kappa = s_abs / np.maximum(np.abs(g_r), 1e-300)
    cond_ok = (kappa > 1e3) & (err <= max(tol * 1e-3, u) * s_abs)
    round_ok = err <= 8.0 * u * s_sq
    esc = ~rel_ok & (cond_ok | round_ok)
    # coordinates above the rounding line |g| > 2 * 8 u / tol * S2 must meet
    # the relative tolerance (the escape branches serve the ones below it)
    line = 2.0 * 8.0 * u / tol
    above = np.abs(g_r) > line * s_sq
    ratio = np.abs(g_r) / np.maximum(s_sq, 1e-300)
    return {"n_coords": int(g.size), "L_rel": abs(ll - ll_r) / abs(ll_r), "sum_r_rel": abs(sr - sr_r) / abs(sr_r),
            "dsigma_rel": abs(ds - ds_r) / abs(ds_r), "dsigma_abs": abs(ds - ds_r),
            "grad_max_rel": float(rel.max()), "grad_p999_rel": float(np.quantile(rel, 0.999)),
            "grad_median_rel": float(np.median(rel)),
            "grad_max_rel_above_line": float(rel[above].max()) if np.any(above) else 0.0,
            "n_above_line": int(np.sum(above)),
            "escape_max_g_over_s2": float(ratio[esc].max()) if np.any(esc) else 0.0, "escape_line": line,
            "n_kappa_branch": int(np.sum(~rel_ok & cond_ok)),
            "n_rounding_branch": int(np.sum(~rel_ok & ~cond_ok & round_ok)),
            "n_out_of_tolerance": int(np.sum(~(rel_ok | cond_ok | round_ok))),
            "tolerances": {"L": 1e-6, "grad_coord": tol, "dsigma": tol},
            "oracle_threads": nthreads}


def sweep_entries(reps, order="locality", with_fp64=True):
    """The scale sweep (N = 20000, 50000; D = 2, 6; 12-component mixtures;
    FP32C, autotuned pass shape): per size the pass span (stamps, so only the
    pass), pairs/s and the fraction of the measured HBM copy bandwidth for
    4 B of Y per pair (Y is 0.8 / 5.0 GB, far larger than L2, so every pass
    streams it from HBM); the FP64 pass at N = 20000, D = 2."""
    import torch
    from paper_1905_04582_gb300 import workloads as W
    from paper_1905_04582_gb300.mds import MDS
    hbm_peak, peak_kind = load_peaks()
    out = []
    for n, d in ((20000, 2), (20000, 6), (50000, 2), (50000, 6)):
        t0 = time.perf_counter()
        wl = W.scale_sweep(n, d)
        gen_s = time.perf_counter() - t0
        with MDS(wl.n, wl.d, "fp32c") as m:
            m.set_data(wl.y_packed)
            m.set_locations(wl.x_eval)
            m.set_sigma(wl.sigma)
            if order == "locality":
                m.reorder()
            far, total = m.far_blocks()
            m.set_pass_stamps(True)
            ms = m.time_pass(reps)
            n_pass, span_ms = m.get_pass_span()
            m.set_pass_stamps(False)
            span = span_ms / max(n_pass, 1)
            kind, param, ctas = m.get_pass_shape()
        gbs = 4.0 * wl.m / (span / 1e3) / 1e9
        e = {"workload": wl.name, "n": n, "d": d, "pairs": wl.m, "y_bytes": 4 * wl.m, "order": order,
             "pass_shape": {"kind": PASS_KINDS[kind], "param": param, "ctas": ctas},
             "far_fraction": far / total, "pass_span_ms": span, "pass_and_reduction_ms": ms,
             "pairs_per_s": wl.m / (span / 1e3),
             "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                     "peak_kind": f"{peak_kind} hbm_gbs"},
             "ops_per_pair": fp32_ops_per_pair(d, far / total, kind != 0), "gen_s": gen_s}
        if with_fp64 and n == 20000 and d == 2:
            with MDS(wl.n, wl.d, "fp64") as m64:
                m64.set_data(wl.y_packed)
                m64.set_locations(wl.x_eval)
                m64.set_sigma(wl.sigma)
                m64.set_pass_stamps(True)
                ms64 = m64.time_pass(2)
                n64, sp64 = m64.get_pass_span()
            e["fp64_pass_span_ms"] = sp64 / max(n64, 1)
            e["speedup_vs_fp64"] = e["fp64_pass_span_ms"] / span
        out.append(e)
        del wl
        torch.cuda.synchronize()
    return out


def batch_entry(reps, steps):
    """Batched datasets x chains (N = 1600, 1500, 1300, 992; 8 chains each):
    pair evaluations per second of one batched pass for all 32 chains, and
    HMC leapfrog steps per second over all chains."""
    import torch
    from paper_1905_04582_gb300 import workloads as W
    from paper_1905_04582_gb300.mds import Batch, MDS
    ds = W.batch_datasets()
    chains = 8
    b = Batch([w.n for w in ds], 2, [chains] * len(ds))
    try:
        for k, w in enumerate(ds):
            b.set_data(k, w.y_packed)
            b.set_sigma(k, w.sigma)
            for j in range(chains):
                b.set_locations(k, j, w.x_eval)
        b.reorder()  # each dataset's locality order, shared by its chains
        ms = b.time_pass(reps)
        evals = sum(w.m for w in ds) * chains
        b.hmc(2, N_LEAPFROG, [5e-4] * len(ds), seed=1)  # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        acc, dh = b.hmc(steps, N_LEAPFROG, [5e-4] * len(ds), seed=2)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        strip = b.get_strip()
    finally:
        b.close()
    with MDS(128, 2, "fp32c") as mc:
        mc.set_sigma(ds[0].sigma)
        ceil_near = mc.pair_body_ceiling(far=False)
    shape = (f"batched strip kernel, {strip} tiles per strip" if strip > 0 else
             f"every chain's chunked pass (about {-strip} tiles per chunk) as concurrent graph branches")
    return {"datasets": [w.n for w in ds], "chains_per_dataset": chains, "order": "locality (mds_batch_reorder)",
            "strip": strip,
            "shape": shape,
            "ms_per_pass": ms, "pair_evals_per_pass": evals, "pair_evals_per_s": evals / (ms / 1e3),
            "measured_ceiling": {"near_pairs_per_s": ceil_near, "frac": evals / (ms / 1e3) / ceil_near,
                                 "note": "the full per-pair body (Phi evaluated) on register operands"},
            "hmc_iterations": steps, "leapfrog_steps_per_s_all_chains": steps * N_LEAPFROG * len(ds) * chains / wall,
            "accept_rate": float(np.mean(acc))}


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
    if args.order == "locality":
        model.reorder()  # tile layouts in the locality order of the start point
    far_blocks, total_blocks = model.far_blocks()
    far_frac = far_blocks / total_blocks
    seed = 1234 + rank

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(float(np.random.rand()))

    # warm-up (autotune, graph capture, clocks), then the step size: fixed by
    # --eps, else a short pilot for acceptance ~0.65
    model.log_likelihood()
    model.hmc(max(args.warmup, 1), N_LEAPFROG, 2e-4, seed=seed)
    if args.eps > 0:
        eps, pilot = args.eps, None
    else:
        eps, pilot = eps_pilot(model, 1e-3, seed)
    model.hmc(1, N_LEAPFROG, eps, seed=seed)  # graph for this step size

    # timed region: K HMC iterations queued back to back on the stream (no
    # host round trip between them), each bracketed by its own CUDA events,
    # L2 flushed before each one outside the brackets.  The pair pass's span
    # inside each leapfrog step is taken by %globaltimer stamps (no events
    # between the launches, so programmatic dependent launch stays intact).
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    model.set_pass_stamps(True)
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
    n_pass, span_total_ms = model.get_pass_span()
    model.set_pass_stamps(False)
    acc_total = int(acc.sum())
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in zip(ev_s, ev_e)]
    dev_ms = sum(step_ms)
    dev_ms_max = reduce_max(dev_ms, world)

    pairs_per_step = N_LEAPFROG * wl.m
    value = replica_rate(args.steps * pairs_per_step, dev_ms / 1e3, world)
    lf_steps = world * args.steps * N_LEAPFROG / (dev_ms_max / 1e3)

    # roofline of the dominant kernel (the fused pair pass): HBM-bound by
    # design, 4 B of Y per pair per pass, against the measured copy bandwidth;
    # its time is the pass's span inside the timed steps
    hbm_peak, peak_kind = load_peaks()
    m_pairs, y_bytes = model.problem_size()
    span_ms = span_total_ms / max(n_pass, 1)
    alg_bytes = 4.0 * m_pairs  # one FP32 y_ij per pair per pass
    achieved_gbs = alg_bytes / (span_ms / 1e3) / 1e9
    kind, param, ctas = model.get_pass_shape()
    kname = PASS_KINDS[kind]
    chunked = kind != 0
    kernel_name = f"pair_chunk_kernel<{wl.d}>" if chunked else f"pair_f32_kernel<{wl.d}>"
    traffic = kernel_traffic(wl.n, wl.d, kname)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = clocks.summary()
    sm_mhz = (clk or {}).get("sm_max_mhz") or SM_MAX_MHZ
    alu_peak = sm_count * 128 * sm_mhz * 1e6 / 1e12  # T FP32 lane-op/s
    ops = fp32_ops_per_pair(wl.d, far_frac, chunked)
    kernel_rate = m_pairs / (span_ms / 1e3)

    # the plain FP64 GPU path on the same data (pass spans, timed alone)
    with MDS(wl.n, wl.d, "fp64", stream=stream) as m64:
        m64.set_data(wl.y_packed)
        m64.set_locations(wl.x_eval)
        m64.set_sigma(wl.sigma)
        m64.set_pass_stamps(True)
        ms64 = m64.time_pass(5)
        n64, sp64 = m64.get_pass_span()
    model.set_pass_stamps(True)
    ms32 = model.time_pass(20)
    n32, sp32 = model.get_pass_span()
    model.set_pass_stamps(False)
    # the same FP32C pass with the items in the caller's (random) order: no
    # warp block is all far, every pair evaluates Phi
    with MDS(wl.n, wl.d, "fp32c", stream=stream) as m_u:
        m_u.set_data(wl.y_packed)
        m_u.set_locations(wl.x_eval)
        m_u.set_sigma(wl.sigma)
        m_u.set_pass_stamps(True)
        ms32_unordered = m_u.time_pass(20)
        nu, spu = m_u.get_pass_span()
    # the measured ceiling of the per-pair arithmetic: the bodies with their
    # operands in registers, no memory traffic or epilogue; far blocks take
    # the body without the Phi terms
    ceil_near = model.pair_body_ceiling(far=False)
    ceil_far = model.pair_body_ceiling(far=True)
    ceil_w = 1.0 / (far_frac / ceil_far + (1.0 - far_frac) / ceil_near)

    # end to end through the C ABI with host buffers: X in, one HMC
    # iteration, X and the statistics out
    x_host = torch.from_numpy(model.get_locations(dtype=np.float32).copy()).pin_memory()
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
    parity = None
    if rank == 0 and world == 1:
        ncores = os.cpu_count() or 1
        parity = parity_entry(model, wl, ncores)
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            rate, secs = cpu_oracle_rate(wl, args.cpu_evals)
            cpu = {"value": rate, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                   "sample": f"{args.cpu_evals} serial evaluations of L and dL/dX at N=5392 ({secs:.1f} s)"}
            rate_mt, secs_mt = cpu_oracle_rate(wl, args.cpu_evals, nthreads=ncores)
            cpu["all_cores"] = {"value": rate_mt, "unit": "pairs/s", "cores": ncores,
                                "kind": "oracle (OpenMP rows)",
                                "sample": f"{args.cpu_evals} evaluations of L and dL/dX at N=5392 ({secs_mt:.1f} s)"}
    model.close()

    sweep = None
    if rank == 0 and world == 1 and not args.no_sweep:
        with ClockSampler(local) as sclk:
            sweep = {"scale": sweep_entries(3), "batched": batch_entry(5, 5)}
        sweep["clocks"] = sclk.summary()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": wl.n, "d": wl.d, "pairs": m_pairs, "sigma": wl.sigma,
                       "precision": "FP32 per pair, compensated FP32 partials reduced in FP64",
                       "step": f"one HMC iteration: {N_LEAPFROG} leapfrog steps (fused L+grad pass each) + Metropolis",
                       "eps": eps, "eps_pilot": pilot,
                       "pass_shape": {"kind": kname, "param": param, "ctas": ctas},
                       "order": ("locality order of the start point (mds_reorder)" if args.order == "locality"
                                 else "caller's item order"),
                       "l2": "flushed (512 MB write) between timed steps; Y (58 MB) stays L2-resident within a step",
                       "parallelism": f"replicas x{world}"},
            "leapfrog_steps_per_s": lf_steps,
            "accept_rate": acc_total / args.steps,
            "far_blocks": {"far": far_blocks, "total": total_blocks, "fraction": far_frac,
                           "note": "warp blocks of 64 x 8 pairs all at z >= 8: Phi terms skipped (start point)"},
            "pass_alone": {"fp32c_span_ms": sp32 / max(n32, 1), "fp32c_with_reduction_ms": ms32,
                           "fp64_span_ms": sp64 / max(n64, 1), "fp64_with_reduction_ms": ms64,
                           "fp32c_caller_order_span_ms": spu / max(nu, 1),
                           "fp32c_pairs_per_s": m_pairs / (sp32 / max(n32, 1) / 1e3),
                           "fp64_pairs_per_s": m_pairs / (sp64 / max(n64, 1) / 1e3),
                           "speedup_vs_fp64": (sp64 / max(n64, 1)) / (sp32 / max(n32, 1))},
            "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                         "peak_kind": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                         "kernel": kernel_name, "algorithmic_bytes_per_launch": alg_bytes,
                         "pass_span_ms": span_ms, "passes_timed": n_pass,
                         "span_note": "per pass: the first warp past the dependency wait to the last warp's "
                                      "end (%globaltimer), inside the timed HMC steps",
                         "passes_x_span_ms_per_step": N_LEAPFROG * span_ms,
                         "measured_ceiling": {"near_pairs_per_s": ceil_near, "far_pairs_per_s": ceil_far,
                                              "weighted_pairs_per_s": ceil_w, "kernel_pairs_per_s": kernel_rate,
                                              "frac": kernel_rate / ceil_w,
                                              "note": "mds_pair_body_ceiling: the strip pass's per-pair bodies "
                                                      "on register operands at its occupancy, weighted by the "
                                                      "far-block fraction"},
                         "alu_view": {"ops_per_pair": ops, "achieved_tflops": kernel_rate * ops / 1e12,
                                      "peak_tflops": alu_peak, "frac": kernel_rate * ops / 1e12 / alu_peak,
                                      "peak_kind": f"derived: {sm_count} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz",
                                      "note": "FP32 lane operations the pass executes per pair (exact-split "
                                              "arithmetic included), weighted by the far-block fraction"}},
            "parity": parity,
            "sweep": sweep,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": wl.n * wl.d * 4,
                    "d2h_bytes_per_step": wl.n * wl.d * 4 + 8 + 8 + 4,
                    "note": "mds_set_locations(host X) + mds_hmc(1 iteration) + mds_get_locations(host)"},
            "gpu_launches": args.steps * (2 + 2 * N_LEAPFROG),
            "wall_s": wall,
        }
        if clk is not None:
            line["clocks"] = clk
        print(json.dumps(line), flush=True)
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
    chunks = ("sm", args.sm_chunks) if args.sm_chunks else args.chunks
    with MDS(wl.n, wl.d, args.precision, strip=args.strip, chunks=chunks) as m:
        m.set_data(wl.y_packed)
        m.set_locations(wl.x_eval)
        m.set_sigma(wl.sigma)
        if args.order == "locality":
            m.reorder()
        far, total = m.far_blocks()
        m.set_pass_stamps(True)
        ms = m.time_pass(args.reps)
        n_pass, span = m.get_pass_span()
        span /= max(n_pass, 1)
        print(json.dumps({"pass_only": True, "n": wl.n, "d": wl.d, "precision": args.precision,
                          "order": args.order, "far_fraction": far / total, "pass_shape": m.get_pass_shape(),
                          "pass_and_reduction_ms": ms, "pass_span_ms": span, "pairs_per_s": wl.m / (span / 1e3),
                          "alg_gb_per_s": 4.0 * wl.m / (span / 1e3) / 1e9}), flush=True)
    return 0


def run_sweep(args):
    """The scale sweep alone: one JSON line per size (see sweep_entries)."""
    import torch
    from paper_1905_04582_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    with ClockSampler(0) as clk:
        entries = sweep_entries(args.reps, args.order)
    for e in entries:
        print(json.dumps(dict(e, sweep=True)), flush=True)
    print(json.dumps({"sweep_clocks": clk.summary()}), flush=True)
    return 0


def run_batch(args):
    """Batched datasets x chains alone (see batch_entry)."""
    import torch
    from paper_1905_04582_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    print(json.dumps(dict(batch_entry(args.reps, args.steps), batch=True)), flush=True)
    return 0


def run_tree(args):
    """HMC at N = 5392 with the phylogenetic prior of section 2.2 in the
    target (four coalescent trees of the paper's subtype sizes, locations
    drawn from the Brownian process, Y from those locations): ms per
    iteration with and without the prior, and the prior's evaluation alone."""
    import torch
    from scipy.spatial.distance import pdist
    from paper_1905_04582_gb300 import build as B
    from paper_1905_04582_gb300 import workloads as W
    from paper_1905_04582_gb300.mds import MDS
    B.build()
    torch.cuda.set_device(0)
    f = W.random_forest(W.SUBTYPE_SIZES, n_lone=0, d=2, seed=1, rate=0.05)
    x_true = W.brownian_tips(f, seed=2)
    rng = np.random.default_rng(3)
    sigma = 0.3
    y = np.abs(pdist(x_true) + sigma * rng.standard_normal(f.n * (f.n - 1) // 2)).astype(np.float32)
    x_eval = (x_true + 0.02 * rng.standard_normal(x_true.shape)).astype(np.float32)
    stream = torch.cuda.Stream()
    eps = args.eps if args.eps > 0 else 2e-4
    out = {"tree": True, "n": f.n, "trees": list(W.SUBTYPE_SIZES), "steps": N_LEAPFROG, "eps": eps}
    for with_tree in (False, True):
        with MDS(f.n, 2, "fp32c", stream=stream) as m:
            m.set_data(y)
            m.set_locations(x_eval)
            m.set_sigma(sigma)
            if with_tree:
                m.set_tree_prior(f.parent, f.length, f.sigma_mat, f.mu, f.tau0, f.tau_u)
            m.reorder()
            m.hmc(3, N_LEAPFROG, eps, seed=5)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            m.hmc_enqueue(args.steps, N_LEAPFROG, eps, seed=6)
            ev1.record(stream)
            acc, _, _ = m.hmc_collect()
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / args.steps
            key = "with_tree_prior" if with_tree else "likelihood_only"
            out[key] = {"ms_per_iteration": ms, "leapfrog_steps_per_s": N_LEAPFROG / (ms / 1e3),
                        "accept_rate": float(np.mean(acc))}
            if with_tree:
                g = torch.empty((f.n, 2), dtype=torch.float64, device="cuda")
                m.tree_prior(out=g)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                reps = 50
                for _ in range(reps):
                    m.tree_prior(out=g)
                torch.cuda.synchronize()
                out["tree_prior_call_us"] = 1e6 * (time.perf_counter() - t0) / reps
                # the traversal kernel alone: evaluations queued back to back
                # (no outputs copied, no synchronisation), CUDA events
                ev0.record(stream)
                for _ in range(reps):
                    m._check(m._lib.mds_tree_prior(m._h, None, None, 0, 0))
                ev1.record(stream)
                torch.cuda.synchronize()
                out["tree_prior_kernel_us"] = 1e3 * ev0.elapsed_time(ev1) / reps
    out["tree_prior_cost_per_step_us"] = 1e3 * (out["with_tree_prior"]["ms_per_iteration"] -
                                               out["likelihood_only"]["ms_per_iteration"]) / N_LEAPFROG
    print(json.dumps(out), flush=True)
    return 0


def ess(chain):
    """Effective sample size of a scalar chain: n / tau, tau = 1 + 2 sum of
    autocorrelations over Geyer's initial positive sequence (pairs of lags
    summed while positive)."""
    x = np.asarray(chain, dtype=np.float64)
    n = len(x)
    x = x - x.mean()
    v = np.dot(x, x) / n
    if n < 4 or v == 0.0:
        return float(n)
    f = np.fft.rfft(x, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n] / (n * v)
    tau = -1.0
    for k in range(0, n - 1, 2):
        pair = acf[k] + acf[k + 1]
        if pair <= 0:
            break
        tau += 2 * pair
    return float(n / max(tau, 1.0))


def run_mixing(args):
    """Mixing of HMC against the single-item random-walk Metropolis sampler
    (section 2.3's prior art) at N = 5392: effective sample size per second of
    sampler device time for rotation-invariant statistics (the
    log-likelihood and distances of fixed item pairs), both from the same
    HMC-burned-in state, step sizes from short pilots."""
    import torch
    from paper_1905_04582_gb300 import build as B
    from paper_1905_04582_gb300 import workloads as W
    from paper_1905_04582_gb300.mds import MDS
    B.build()
    torch.cuda.set_device(0)
    wl = W.paper_scale()
    stream = torch.cuda.Stream()
    pairs = np.array([[0, 1], [2, 3], [10, 500], [100, 4000], [7, 2500]])

    def stats_of(m):
        ll, _ = m.log_likelihood()
        x = m.get_locations()
        return [ll] + list(np.linalg.norm(x[pairs[:, 0]] - x[pairs[:, 1]], axis=1))

    def timed(stream, fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    with MDS(wl.n, wl.d, "fp32c", stream=stream) as m:
        m.set_data(wl.y_packed)
        m.set_locations(wl.x_eval)
        m.set_sigma(wl.sigma)
        m.reorder()
        # burn-in from the jittered start, then the HMC step: the largest of a
        # few whose pilot acceptance is >= 0.6
        m.hmc(200, N_LEAPFROG, 2e-4, seed=11)
        x0 = m.get_locations()
        eps = 2e-4
        for cand in (4e-4, 8e-4, 1.6e-3):
            acc, _, _ = m.hmc(30, N_LEAPFROG, cand, seed=12)
            m.set_locations(x0)
            if np.mean(acc) >= 0.6:
                eps = cand
        m.reorder()  # the burned-in configuration
        x0 = m.get_locations()
        # random-walk step: pilot acceptance closest to 0.35
        best, step = None, 1e-3
        for cand in (1e-3, 2e-3, 4e-3, 8e-3, 1.6e-2):
            acc, _ = m.rwmh(2000, cand, seed=13)
            m.set_locations(x0)
            if best is None or abs(np.mean(acc) - 0.35) < best:
                best, step = abs(np.mean(acc) - 0.35), cand
        # HMC chain
        n_hmc = args.steps if args.steps > 20 else 300
        hmc_stats, hmc_s, hmc_acc = [], 0.0, []
        for _ in range(n_hmc):
            (acc, _, _), dt = timed(stream, lambda: m.hmc(1, N_LEAPFROG, eps, seed=14))
            hmc_s += dt
            hmc_acc.append(acc[0])
            hmc_stats.append(stats_of(m))
        # random-walk chain from the same state: one record per sweep of N proposals
        m.set_locations(x0)
        n_sweeps = 60
        rw_stats, rw_s, rw_acc = [], 0.0, []
        for _ in range(n_sweeps):
            (acc, _), dt = timed(stream, lambda: m.rwmh(wl.n, step, seed=15))
            rw_s += dt
            rw_acc.append(float(np.mean(acc)))
            rw_stats.append(stats_of(m))
    hs, rs = np.array(hmc_stats), np.array(rw_stats)
    names = ["loglik"] + [f"dist({a},{b})" for a, b in pairs]
    out = {"mixing": True, "n": wl.n, "workload": WORKLOAD,
           "hmc": {"eps": eps, "leapfrog_steps": N_LEAPFROG, "iterations": n_hmc, "device_s": hmc_s,
                   "accept_rate": float(np.mean(hmc_acc)),
                   "ess": {k: ess(hs[:, c]) for c, k in enumerate(names)}},
           "rwmh": {"step": step, "proposals_per_sweep": wl.n, "sweeps": n_sweeps, "device_s": rw_s,
                    "proposals_per_s": n_sweeps * wl.n / rw_s, "accept_rate": float(np.mean(rw_acc)),
                    "ess": {k: ess(rs[:, c]) for c, k in enumerate(names)}}}
    out["ess_per_s_ratio_hmc_over_rwmh"] = {
        k: (out["hmc"]["ess"][k] / hmc_s) / max(out["rwmh"]["ess"][k] / rw_s, 1e-300) for k in names}
    print(json.dumps(out), flush=True)
    return 0


def run_rwmh_only(args):
    """Proposals per second of the single-item random-walk sampler at
    N = 5392 (locality order), the command its kernel profile is taken with."""
    import torch
    from paper_1905_04582_gb300 import build as B
    from paper_1905_04582_gb300 import workloads as W
    from paper_1905_04582_gb300.mds import MDS
    B.build()
    torch.cuda.set_device(0)
    wl = W.paper_scale()
    with MDS(wl.n, wl.d, "fp32c") as m:
        m.set_data(wl.y_packed)
        m.set_locations(wl.x_eval)
        m.set_sigma(wl.sigma)
        m.reorder()
        m.rwmh(args.props, 0.008, seed=1)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        acc, _ = m.rwmh(args.props, 0.008, seed=2)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    print(json.dumps({"rwmh_only": True, "n": wl.n, "proposals": args.props, "s": dt,
                      "proposals_per_s": args.props / dt, "accept_rate": float(np.mean(acc))}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--eps", type=float, default=0.0, help="leapfrog step (0: a short pilot for acceptance ~0.65)")
    ap.add_argument("--cpu-evals", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="leave the scale sweep and the batched case out")
    ap.add_argument("--pass-only", action="store_true", help="time the fused pass alone (profiling runs)")
    ap.add_argument("--n", type=int, default=5392)
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--strip", type=int, default=None)
    ap.add_argument("--chunks", type=int, default=None, help="chunked pass, chunks per resident CTA slot")
    ap.add_argument("--sm-chunks", type=int, default=None,
                    help="chunked pass in its grouped form (one CTA per SM), chunks per slot")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--kernel-hash", action="store_true", help="print the pair kernel's source hash and exit")
    ap.add_argument("--sweep", action="store_true", help="the N = 20000 / 50000 scale sweep (pass only)")
    ap.add_argument("--batch", action="store_true", help="batched datasets x chains")
    ap.add_argument("--tree", action="store_true", help="HMC with the phylogenetic prior (section 2.2)")
    ap.add_argument("--mixing", action="store_true", help="ESS/s of HMC against single-item random-walk MH")
    ap.add_argument("--rwmh-only", action="store_true", help="proposals/s of the random-walk sampler")
    ap.add_argument("--props", type=int, default=5392)
    ap.add_argument("--order", default="locality", choices=["locality", "caller"],
                    help="tile layouts in the locality order (mds_reorder) or the caller's item order")
    args = ap.parse_args()
    if args.kernel_hash:
        print(pair_kernel_sha256())
        return 0
    if args.sweep:
        return run_sweep(args)
    if args.batch:
        return run_batch(args)
    if args.tree:
        return run_tree(args)
    if args.mixing:
        return run_mixing(args)
    if args.rwmh_only:
        return run_rwmh_only(args)
    if args.pass_only:
        return run_pass_only(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
