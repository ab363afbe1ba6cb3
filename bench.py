#!/usr/bin/env python3
"""Throughput benchmark: psi coefficients/s of FFT-Newton inversion on GB300.

One step = one call of the public inverse (mrc_inverse) on the whole workload:
Gauss-Jordan of A(0), all Newton doubling levels and, for the mixed path, the
double-float residual and FP32 correction sweep.  Inputs are resident in HBM
when the timed region starts; the e2e figure repeats the measurement through
mrc_inverse_host, from pinned host buffers, with the host->device upload of A
(in the row ranges the Newton levels consume, overlapping them) and the
device->host copy of psi inside the timed region.

Default workload (the precision configuration of the metric): d = 64 states,
horizon N = 2^18, Lognormal sojourns sigma ~ U[1,2], mu ~ U[0,3] reduced by the
endpoint mean-value rule with h = 0.05 (A(0) = I - Q(h)/2), Dirichlet(1)
zero-diagonal embedded chain, seed 0.  A and psi are 8.6 GB each, far larger
than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mrc|reference]
                    [--workload NAME] [--prec mixed|fp64]

Multi-GPU (torchrun): the workload is one model, which does not shard
(replicas only): each rank inverts its own replica; value = all ranks'
coefficients / max-over-ranks time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (d, N, kind, extra)
    "lognormal_d64_N262144": (64, 1 << 18, "lognormal", {}),
    "weibull_d16_N65536": (16, 1 << 16, "weibull", {}),
    "weibull_d4_N1024": (4, 1024, "weibull", {}),
    "lognormal_d64_N65536": (64, 1 << 16, "lognormal", {}),
    # the default workload's d with a device footprint of a few GB (profiler captures)
    "lognormal_d64_N16384": (64, 1 << 14, "lognormal", {}),
    # the default workload's transform lengths with E = 256 (small profiler captures)
    "lognormal_d16_N262144": (16, 1 << 18, "lognormal", {}),
    # dense precision stress: iterative refinement with two sweeps
    "weibull_d256_N32768": (256, 1 << 15, "weibull", {"alpha": 0.5, "shape": (0.5, 3.0), "sweeps": 2}),
    # 256 independent models, d ~ U{3..48}, N = round(2^U[10,16]), half discrete Weibull,
    # half Lognormal mean-value (h = 0.05), one captured batch
    "batch256": (0, 0, "batch", {"n": 256}),
    # continuous-time Markov renewal equation (mrc_mre_solve, mean-value rule):
    # the paper's four-state exponential benchmark, N = 2^15, h = 0.005, transition function
    "mre_exponential_N32768": (4, 1 << 15, "mre", {"h": 0.005}),
    # FFT-Gauss-Jordan (mrc_inverse_gj) against FFT-Newton (mrc_inverse, FP64) on the kernels of the
    # paper's scaling experiments (Section 5): s = 2, 4, 6, 8 shifted Poisson, N = 2^7 .. 2^16
    "gj_scaling": (0, 0, "gj", {"s": (2, 4, 6, 8), "logN": tuple(range(7, 17))}),
}
DEFAULT_WORKLOAD = "lognormal_d64_N262144"
# the metric both arms report (mrc and the oracle reference arm)
METRIC = "\u03c8 coefficients/s (N\u00b7d\u00b2) mixed-precision vs FP64 GPU at \u22641e-10 residual"

# kernel classes of the library's profiler (include/mrc.h MRC_K_*)
KCLASS = {1: "fft_f64", 2: "fft_f32", 3: "fft_dd", 4: "pairmul_f64", 5: "pairmul_f32", 6: "pairmul_dd", 7: "misc"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 DFMA rate measured on this machine's GB300 by a dependent-chain-free FMA
# loop (1.19 TFLOP/s); FP32 FFMA: 152 SMs x 128 lanes x 2 flops per clock.
FP32_LANES = 152 * 128
FP64_TFLOPS_MEASURED = 1.19


def roofline_for(kclass, ms_total, launches, bytes_, flops, peaks, sm_mhz, d=None):
    """Roofline of one kernel class from its timed launches: achieved =
    algorithmic bytes (or flops) per launch / average launch time.  FFT
    passes, the tensor-core digit products (whose FP32 and tensor pipes are
    not the binding resource at d <= 64) and the small kernels are reported
    against the measured HBM copy bandwidth; FP64 products against the
    measured DFMA rate, FP32-pipe products against the FFMA peak."""
    if not launches:
        return None
    per_ms = ms_total / launches
    name = KCLASS[kclass]
    clk = (sm_mhz or 2070.0) * 1e6
    on_tc = name in ("pairmul_dd", "pairmul_f32") and d is not None and 32 <= d <= (512 if name == "pairmul_dd" else 64)
    if name.startswith("fft_") or name == "misc" or on_tc:
        ach = bytes_ / launches / (per_ms * 1e-3) / 1e9
        peak = peaks["hbm_gbs"]
        src = "MEASURED_PEAKS.json hbm_gbs (of measured)" + ("; tensor-core digit products" if on_tc else "")
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": None, "launches": launches, "avg_ms": per_ms, "peak_source": src}
    if name.endswith("_f64"):
        ach = flops / launches / (per_ms * 1e-3) / 1e12
        peak = FP64_TFLOPS_MEASURED
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "launches": launches, "avg_ms": per_ms,
                "peak_source": "FP64 DFMA loop measured on GB300 (1.19 TFLOP/s)"}
    # FP32-pipe or double-float SIMT products: FP32 FFMA bound at d >= 16
    ach = flops / launches / (per_ms * 1e-3) / 1e12
    peak = FP32_LANES * 2 * clk / 1e12
    return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None, "launches": launches, "avg_ms": per_ms,
            "peak_source": f"FP32 FFMA: 152x128 lanes x 2 x {clk/1e6:.0f} MHz"}


# Sources each kernel class is built from: a committed DRAM-traffic capture
# of a class stays valid while these files are unchanged.
_CLASS_SOURCES = {
    "fft": ["kernels.cuh", "launchers.cuh", "arith.cuh", "mrc_internal.h"],
    "tc": ["pair_tc.cu", "ozaki_tc.cu", "tcgen05.cuh", "digits.cuh", "kernels.cuh", "arith.cuh", "mrc_internal.h"],
    "simt": ["kernels.cuh", "launchers.cuh", "arith.cuh", "mrc_internal.h"],
}


def class_sources(kernel):
    if kernel.startswith("fft_"):
        prec = kernel[4:]
        return _CLASS_SOURCES["fft"] + [f"k_{prec}_fft_lo.cu", f"k_{prec}_fft_hi.cu", f"k_{prec}.cu"]
    if kernel in ("pairmul_dd", "pairmul_f32"):
        return _CLASS_SOURCES["tc"]
    return _CLASS_SOURCES["simt"] + ["k_f64.cu", "k_f32.cu", "k_dd.cu", "misc.cu"]


def sources_digest(kernel):
    """sha256 over the sources of one kernel class, as recorded beside an ncu
    traffic capture of that class."""
    import hashlib
    h = hashlib.sha256()
    for f in class_sources(kernel):
        rel = os.path.join("paper_2605_30379_gb300", "csrc", f)
        h.update(rel.encode())
        with open(os.path.join(HERE, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, bytes_per_launch):
    """DRAM traffic per launch of one kernel class: the ratio of DRAM bytes
    (dram__bytes_read.sum + dram__bytes_write.sum) to the algorithmic bytes
    that profiles/traffic_<kernel>.json records from an ncu capture of that
    class on a smaller case of the same d (the traffic of these kernels grows
    with the units they process), times this run's algorithmic bytes per
    launch -- only while the class's sources are the ones the capture was
    taken on; else (None, None)."""
    path = os.path.join(HERE, "profiles", f"traffic_{kernel}.json")
    try:
        with open(path) as fh:
            doc = json.load(fh)
    except (OSError, ValueError):
        return None, None
    if doc.get("sources_sha256") != sources_digest(kernel):
        return None, None
    return doc["dram_over_algorithmic"] * bytes_per_launch, os.path.relpath(path, HERE)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_input(name):
    from paper_2605_30379_gb300 import synth
    d, N, kind, extra = WORKLOADS[name]
    if kind == "batch":
        return [m["A"] for m in synth.batch_models(n=extra["n"], seed=0)]
    if kind == "lognormal":
        A, _ = synth.lognormal_model(d, N, seed=0, h=0.05)
    else:
        q, _ = synth.weibull_model(d, N, seed=0, **{k: v for k, v in extra.items() if k != "sweeps"})
        A = synth.identity_minus(q)
    return A


def max_over_ranks_on(x, world, device):
    """The slowest rank's time (all ranks receive it); identity at world size 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def model_cost(d, N):
    """Cost model of one inverse, ~ N d^2 (log2 N + d): the FFT and
    per-frequency product terms of Proposition 2.4."""
    return float(N) * d * d * (max(1, int(N - 1).bit_length()) + d)


def lpt_partition(costs, world):
    """Greedy longest-processing-time assignment of independent models to
    ranks: models in decreasing cost (ties by index) go to the least-loaded
    rank (ties to the lowest rank).  Deterministic, so every rank computes the
    same partition without a collective.  Returns per-rank sorted index lists."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def job_throughput(units_per_rank, ms_step, world):
    """Whole-job rate: the units every rank processed per second of the
    slowest rank's step time (replicas: each rank processes units_per_rank)."""
    return world * units_per_rank / (ms_step * 1e-3)


def cpu_oracle_sample(A_host, d, budget_s=15.0):
    """Time the FP64 oracle (direct recursion) on a prefix of the same input,
    doubling the prefix until one call takes >= budget_s / 4 (then one timed
    call).  Returns (n, seconds, threads, the oracle's inverse of the prefix)."""
    import oracle
    n = 64
    while True:
        t0 = time.perf_counter()
        oracle.inverse_left(A_host[:n])
        dt = time.perf_counter() - t0
        if dt >= budget_s / 4 or 2 * n > A_host.shape[0]:
            break
        n *= 2
    t0 = time.perf_counter()
    psi = oracle.inverse_left(A_host[:n])
    dt = time.perf_counter() - t0
    return n, dt, oracle.num_threads(), psi


def per_output_errors(mrc, A_host, psi_dev, psi_ref, prec):
    """Errors of the library's outputs against the oracle's on the prefix
    k < n that the oracle inverted (Proposition 2.3: a prefix of the inverse
    depends only on the same prefix of A): psi; P = psi * Hbar (mrc_transition)
    and the first-entrance distribution F_D and reliability S_D = 1 - F_D
    (mrc_first_entrance, D = the last ceil(d/4) states, alpha_C = e_1), all
    for the kernel q = e0 - A of the workload."""
    import oracle
    import torch
    n, d = psi_ref.shape[0], psi_ref.shape[1]
    got = psi_dev[:n].cpu().numpy()
    num = np.sqrt(((got - psi_ref) ** 2).sum(axis=(1, 2))).sum()
    den = np.sqrt((psi_ref ** 2).sum(axis=(1, 2))).sum()
    out = {"prefix": n, "psi": {"max_abs": float(np.abs(got - psi_ref).max()), "e_rel": float(num / den)}}
    q = -np.ascontiguousarray(A_host[:n])
    q[0] += np.eye(d)
    qd = torch.from_numpy(q).cuda()
    P = mrc.transition(psi_dev[:n].contiguous(), qd, prec=prec).cpu().numpy()
    out["P"] = {"max_abs": float(np.abs(P - oracle.transition(psi_ref, q)).max())}
    nD = (d + 3) // 4
    D = list(range(d - nD, d))
    alpha = np.zeros(d - nD)
    alpha[0] = 1.0
    g, F, S = mrc.first_entrance(qd, D, torch.from_numpy(alpha), prec=prec)
    _, F_ref, S_ref = oracle.first_entrance(q, D, alpha)
    out["first_entrance_F"] = {"max_abs": float(np.abs(F.cpu().numpy() - F_ref).max())}
    out["reliability_S"] = {"max_abs": float(np.abs(S.cpu().numpy() - S_ref).max())}
    return out


def run_mre(args, rank, world, local):
    """One step = mrc_mre_solve (Eq. (mre-solution)) of the transition
    function on the exponential benchmark; metric: K_h coefficients (N d^2)
    per second, inputs resident; roofline of the dominant kernel class;
    the oracle's mre_solve timed on a prefix as the CPU baseline."""
    import ctypes
    import torch
    from paper_2605_30379_gb300 import mrc, synth
    torch.cuda.set_device(local)
    d, N, _, extra = WORKLOADS[args.workload]
    b = synth.exponential_benchmark(extra["h"], N)
    Q = torch.from_numpy(b["Q"]).cuda()
    L = torch.from_numpy(b["Hbar"]).cuda()
    lib = mrc.load()
    lib.mrc_launch_count.restype = ctypes.c_ulonglong
    lib.mrc_profile_begin.argtypes = [ctypes.c_int]
    lib.mrc_profile_end.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    stream = torch.cuda.current_stream()

    def step():
        return mrc.mre_solve(Q, L, scheme="mean_value", prec=args.prec)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    breakdown = {}
    for kc in KCLASS:
        lib.mrc_profile_begin(kc)
        step()
        ms, n, bb, ff = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        lib.mrc_profile_end(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(bb), ctypes.byref(ff))
        if n.value:
            breakdown[KCLASS[kc]] = {"ms": ms.value, "launches": n.value}
    dominant = max((kc for kc in KCLASS if KCLASS[kc] in breakdown), key=lambda kc: breakdown[KCLASS[kc]]["ms"])
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    lib.mrc_profile_begin(dominant)
    l0 = lib.mrc_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        K = step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = lib.mrc_launch_count() - l0
    pms, pn, pb, pf = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    lib.mrc_profile_end(ctypes.byref(pms), ctypes.byref(pn), ctypes.byref(pb), ctypes.byref(pf))
    clocks = sampler.stop()
    ms_step = e0.elapsed_time(e1) / args.steps
    coeffs = N * d * d
    peaks, peak_kind = load_peaks()
    roof = roofline_for(dominant, pms.value, pn.value, pb.value, pf.value, peaks, clocks["sm_mhz"] if clocks else None,
                        d=d)
    if roof:
        roof["peak_kind"] = peak_kind
        roof["traffic"], roof["traffic_source"] = measured_traffic(roof["kernel"], pb.value / max(pn.value, 1))
    # accuracy: availability against the exact solution (exp(G h) powers)
    import scipy.linalg as sl
    step_m = sl.expm(b["G"] * extra["h"])
    Kh = K.cpu().numpy()
    P = np.eye(4)
    one_u = np.array([1.0, 1.0, 1.0, 0.0])
    err = 0.0
    for m in range(N):
        err = max(err, abs(b["alpha"] @ (P - Kh[m]) @ one_u))
        P = P @ step_m
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        n = 512
        while True:
            t0 = time.perf_counter()
            oracle.mre_solve(b["Q"][:n + 1], b["Hbar"][:n])
            dt = time.perf_counter() - t0
            if dt >= 4.0 or 2 * n > N:
                break
            n *= 2
        cpu = {"value": n * d * d / dt, "unit": "coefficients/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"oracle mre_solve on the prefix m < {n} of the same benchmark ({dt:.1f} s)"}
    line = {"metric": "K_h coefficients/s (N*d^2), continuous-time transition function, mean-value rule",
            "value": coeffs / (ms_step * 1e-3), "unit": "coefficients/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+dd" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "d": d, "N": N, "h": extra["h"], "prec": args.prec,
                       "l2": "inputs below L2 size (latency-bound case)", "parallelism": "single"},
            "accuracy": {"max_abs_availability_error_vs_exact": err, "paper": 2.53e-8},
            "gpu_launches": int(launches), "stage_ms": breakdown, "roofline": roof, "clocks": clocks,
            "e2e": None, "cpu_baseline": cpu}
    if rank == 0:
        print(json.dumps(line))


def run_reference(args, rank, world):
    """The oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    name = args.workload
    d, N, kind, _ = WORKLOADS[name]
    from paper_2605_30379_gb300 import synth
    # prefix of the same seeded workload (the generator is prefix-consistent)
    if kind == "mre":
        import oracle
        b = synth.exponential_benchmark(WORKLOADS[name][3]["h"], 2048)
        times = []
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oracle.mre_solve(b["Q"], b["Hbar"])
            if it >= args.warmup:
                times.append(time.perf_counter() - t0)
        ms = 1e3 * float(np.mean(times))
        value = 2048 * d * d / (ms * 1e-3)
        cpu = {"value": value, "unit": "coefficients/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"oracle mre_solve on the prefix m < 2048 of the {name} workload"}
        print(json.dumps({"impl": "reference", "metric": "K_h coefficients/s (N*d^2), continuous-time transition "
                          "function, mean-value rule", "value": value, "unit": "coefficients/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": name, "d": d, "N": N}, "cpu_baseline": cpu,
                          "e2e": {"value": value, "unit": "coefficients/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    if kind == "batch":
        A = synth.batch_models(n=1, seed=0)[0]["A"]
        d, N = A.shape[1], A.shape[0]
    elif kind == "lognormal":
        A, _ = synth.lognormal_model(d, min(N, 8192), seed=0, h=0.05)
    else:
        q, _ = synth.weibull_model(d, min(N, 8192), seed=0,
                                   **{k: v for k, v in WORKLOADS[name][3].items() if k != "sweeps"})
        A = synth.identity_minus(q)
    import oracle
    n, dt, cores, _ = cpu_oracle_sample(A, d, budget_s=8.0)
    for _ in range(args.warmup):
        oracle.inverse_left(A[:n])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.inverse_left(A[:n])
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = n * d * d / (ms * 1e-3)
    sample = f"prefix k < {n} of the {name} workload (the oracle costs d^3 n^2 / 2, so its rate falls as 1/n)"
    out = {"impl": "reference", "metric": METRIC, "value": value,
           "unit": "coefficients/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "config": {"workload": name, "d": d, "N": N},
           "cpu_baseline": {"value": value, "unit": "coefficients/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "coefficients/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_gj_compare(args, rank, world):
    """Per (s, N): device time of one FP64 inverse by series Gauss-Jordan and
    by Newton doubling, each launched as a captured CUDA graph (the launch
    cost of the host calls removed) and eagerly; the Gauss-Jordan result
    against the Newton one.  One JSON line; rank 0 only."""
    import torch
    from paper_2605_30379_gb300 import mrc, synth
    if rank != 0:
        return
    extra = WORKLOADS[args.workload][3]
    rows = []
    reps = max(args.steps, 3)
    # size the context workspace for the largest case first: a captured graph
    # holds workspace addresses, so the workspace must not move afterwards
    Abig = torch.from_numpy(synth.identity_minus(
        synth.poisson_paper_e2(max(extra["s"]), 1 << max(extra["logN"])))).cuda()
    mrc.inverse_gj(Abig)
    mrc.inverse(Abig, prec="fp64")
    torch.cuda.synchronize()
    del Abig
    for s_ in extra["s"]:
        for lg in extra["logN"]:
            N = 1 << lg
            A = torch.from_numpy(synth.identity_minus(synth.poisson_paper_e2(s_, N))).cuda()
            out = {"gj": torch.empty_like(A), "newton": torch.empty_like(A)}
            calls = {"gj": lambda: mrc.inverse_gj(A, out=out["gj"]),
                     "newton": lambda: mrc.inverse(A, prec="fp64", out=out["newton"])}
            row = {"s": s_, "N": N}
            for name, fn in calls.items():
                for _ in range(max(args.warmup, 3)):
                    fn()
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                g.replay()
                torch.cuda.synchronize()
                e0.record()
                for _ in range(reps):
                    g.replay()
                e1.record()
                torch.cuda.synchronize()
                row[name + "_graph_ms"] = e0.elapsed_time(e1) / reps
                e0.record()
                for _ in range(reps):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                row[name + "_eager_ms"] = e0.elapsed_time(e1) / reps
            row["gj_over_newton_graph"] = row["gj_graph_ms"] / row["newton_graph_ms"]
            row["max_abs_gj_minus_newton"] = float((out["gj"] - out["newton"]).abs().max())
            rows.append(row)
    print(json.dumps({"workload": args.workload, "metric": "ms per FP64 inverse (CUDA events)",
                      "data": "synthetic (shifted Poisson kernel of the paper's state-dimension experiment)",
                      "reps": reps, "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mrc", choices=["mrc", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-breakdown", action="store_true", help="skip the per-kernel-class timing steps")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-autotune", action="store_true",
                    help="built-in product-kernel choices instead of tuning them during warm-up")
    ap.add_argument("--traffic-step", action="store_true",
                    help="after warm-up, one step per kernel class inside a cudaProfilerStart/Stop window, "
                         "printing each class's algorithmic bytes and launches (for an ncu DRAM capture with "
                         "--profile-from-start off); no timed region")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if WORKLOADS[args.workload][2] == "mre":
        run_mre(args, rank, world, local)
        return
    if WORKLOADS[args.workload][2] == "gj":
        run_gj_compare(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2605_30379_gb300 import mrc

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return max_over_ranks_on(x, world, "cuda")

    d, N, kind, _ = WORKLOADS[args.workload]
    hosts = make_input(args.workload)
    batch = kind == "batch"
    total_coeffs = None
    n_models = len(hosts) if batch else 1
    if batch and world > 1:
        # independent models: each rank inverts its greedy-LPT share of the batch
        total_coeffs = sum(a.shape[0] * a.shape[1] * a.shape[2] for a in hosts)
        share = lpt_partition([model_cost(a.shape[1], a.shape[0]) for a in hosts], world)[rank]
        hosts = [hosts[i] for i in share]
    if not batch:
        hosts = [hosts]
    coeffs = sum(a.shape[0] * a.shape[1] * a.shape[2] for a in hosts)
    A_pins = [torch.from_numpy(a).pin_memory() for a in hosts]
    As = [p.to("cuda", non_blocking=False) for p in A_pins]
    psis = [torch.empty_like(a) for a in As]
    psi_pins = [torch.empty(a.shape, dtype=torch.float64).pin_memory() for a in As]
    A_host_np = hosts[0]
    lib = mrc.load()
    import ctypes
    lib.mrc_launch_count.restype = ctypes.c_ulonglong
    lib.mrc_profile_begin.argtypes = [ctypes.c_int]
    lib.mrc_profile_end.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    stream = torch.cuda.current_stream()

    tune = not args.no_autotune
    sweeps = WORKLOADS[args.workload][3].get("sweeps", 1)

    def step(prec=args.prec):
        if batch:
            mrc.inverse_batched(As, prec=prec, sweeps=sweeps, outs=psis, autotune=tune)
        else:
            mrc.inverse(As[0], prec=prec, sweeps=sweeps, out=psis[0], autotune=tune)

    def prof(kclass, fn):
        lib.mrc_profile_begin(kclass)
        fn()
        ms, n, b, f = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        lib.mrc_profile_end(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b), ctypes.byref(f))
        return ms.value, n.value, b.value, f.value

    lw = lib.mrc_launch_count()
    step()  # first warm-up step (captures the batch graph)
    torch.cuda.synchronize()
    launches_per_step = lib.mrc_launch_count() - lw
    for _ in range(max(args.warmup, 3) - 1):
        step()
    torch.cuda.synchronize()

    if args.traffic_step:
        # one profiler window per kernel class, in KCLASS order
        out = {}
        for kc in KCLASS:
            lib.mrc_profile_begin(kc)
            torch.cuda.profiler.start()
            step()
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
            ms, n, b, f = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
            lib.mrc_profile_end(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b), ctypes.byref(f))
            out[KCLASS[kc]] = {"window": len(out), "algorithmic_bytes": b.value, "launches": n.value}
        if rank == 0:
            print(json.dumps({"workload": args.workload, "traffic_windows": out}), flush=True)
        return

    # per-class device time of one step (untimed), to pick the dominant kernel
    breakdown = {}
    class_work = {}
    for kc in ([] if args.no_breakdown else KCLASS):
        ms, n, b, f = prof(kc, step)
        if n:
            breakdown[KCLASS[kc]] = {"ms": ms, "launches": n}
            class_work[kc] = (ms, n, b, f)
    dominant = max((kc for kc in KCLASS if KCLASS[kc] in breakdown), key=lambda kc: breakdown[KCLASS[kc]]["ms"],
                   default=2 if args.prec == "mixed" else 4)

    # ---- timed region (device-resident inputs)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    # a batch is timed as its graph replays; its per-launch class timing comes
    # from the eager breakdown step above (a timed class makes the batch run eagerly)
    if not batch:
        lib.mrc_profile_begin(dominant)
    l0 = lib.mrc_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = lib.mrc_launch_count() - l0
    if batch:  # graph replays bypass the launch counter: the eager breakdown step's launches per step
        per_step = sum(v[1] for v in class_work.values()) if class_work else launches_per_step
        launches = per_step * args.steps
    pms, pn, pb, pf = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    if not batch:
        lib.mrc_profile_end(ctypes.byref(pms), ctypes.byref(pn), ctypes.byref(pb), ctypes.byref(pf))
    elif dominant in class_work:
        pms.value, pn.value, pb.value, pf.value = class_work[dominant]
    barrier()
    clocks = sampler.stop()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    # replicas: every rank's units; a partitioned batch: the whole batch once
    def rate(ms):
        return job_throughput(coeffs, ms, world) if total_coeffs is None else total_coeffs / (ms * 1e-3)

    value = rate(ms_step)

    # ---- the plain FP64 path on the same inputs
    fp64 = None
    if args.prec == "mixed" and args.fp64_steps > 0:
        step("fp64")
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(args.fp64_steps):
            step("fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1) / args.fp64_steps)
        fp64 = {"value": rate(ms64), "ms_per_step": ms64, "steps": args.fp64_steps}
        # the FP64 path's own residuals (double-float evaluation), beside the mixed path's below
        r64 = {"res_max_abs": 0.0, "res_left_l1": 0.0, "res_right_l1": 0.0}
        for a, p_ in zip(As, psis):
            _, _, r = mrc.residual(a, p_, sides=3, prec="mixed", want_rho=False)
            r64 = {k: max(r64[k], r[k]) for k in r64}
        fp64["accuracy"] = {"max_abs_rho_L": r64["res_max_abs"], "rho_L_l1": r64["res_left_l1"],
                            "rho_R_l1": r64["res_right_l1"]}
        step()  # leave the mixed result in psi for the accuracy check
        torch.cuda.synchronize()

    # ---- accuracy of the timed path: double-float residual of psi (worst model)
    rep = {"res_max_abs": 0.0, "res_left_l1": 0.0, "res_right_l1": 0.0}
    for a, p_ in zip(As, psis):
        _, _, r = mrc.residual(a, p_, sides=3, prec="mixed", want_rho=False)
        rep = {k: max(rep[k], r[k]) for k in rep}

    # ---- e2e through the public API with host buffers
    ms_e2e = None
    if not args.no_e2e:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            if batch:
                for a, p_ in zip(As, A_pins):
                    a.copy_(p_, non_blocking=True)
                step()
                for p_, q_ in zip(psi_pins, psis):
                    p_.copy_(q_, non_blocking=True)
            else:  # mrc_inverse_host: uploads in row ranges overlap the Newton levels
                mrc.inverse_host(A_pins[0], prec=args.prec, sweeps=sweeps, out=psi_pins[0], autotune=tune)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps)

    peaks, peak_kind = load_peaks()
    roof = roofline_for(dominant, pms.value, pn.value, pb.value, pf.value, peaks,
                        clocks["sm_mhz"] if clocks else None, d=None if batch else d)
    if roof:
        roof["peak_kind"] = peak_kind
        roof["traffic"], roof["traffic_source"] = measured_traffic(roof["kernel"], pb.value / max(pn.value, 1))
    # the same roofline for every kernel class of the untimed breakdown step
    by_class = {}
    for kc, (cms, cn, cb, cf) in class_work.items():
        r_ = roofline_for(kc, cms, cn, cb, cf, peaks, clocks["sm_mhz"] if clocks else None, d=None if batch else d)
        if r_ and KCLASS[kc] != "misc":
            by_class[r_["kernel"]] = {k_: r_[k_] for k_ in ("bound", "achieved", "peak", "unit", "frac", "avg_ms")}

    cpu = None
    outputs = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dc = A_host_np.shape[1]
        n, dt, cores, psi_ref = cpu_oracle_sample(A_host_np, dc)
        cpu = {"value": n * dc * dc / dt, "unit": "coefficients/s", "cores": cores, "kind": "oracle",
               "sample": f"one call on the prefix k < {n} of the same workload, {dt:.1f} s "
                         f"(direct recursion, cost d^3 n^2 / 2: its rate falls as 1/n)"}
        if not batch:
            outputs = per_output_errors(mrc, A_host_np, psis[0], psi_ref, args.prec)

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value, "unit": "coefficients/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+dd" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "autotune": tune, "d": d if not batch else "3..48",
                       "N": N if not batch else "round(2^U[10,16])", "models": n_models, "prec": args.prec, "sweeps": sweeps,
                       "l2": (f"inputs ({coeffs * 8 / 1e9:.1f} GB) larger than L2; no flush" if coeffs * 8 > 2e8
                              else "inputs smaller than L2: latency-bound, no flush"),
                       "parallelism": ("single" if world == 1 else "replicas" if total_coeffs is None
                                       else f"greedy LPT partition of the models over {world} ranks")},
            "accuracy": {"max_abs_rho_L": rep["res_max_abs"], "rho_L_l1": rep["res_left_l1"],
                         "rho_R_l1": rep["res_right_l1"], "vs_oracle": outputs},
            "fp64_path": fp64,
            "mixed_over_fp64": (value / fp64["value"]) if fp64 else None,
            "gpu_launches": int(launches),
            "stage_ms": breakdown,
            "roofline": roof,
            "roofline_by_class": by_class or None,
            "clocks": clocks,
            "e2e": None if ms_e2e is None else {
                "value": rate(ms_e2e), "unit": "coefficients/s",
                "h2d_bytes_per_step": coeffs * 8, "d2h_bytes_per_step": coeffs * 8, "ms_per_step": ms_e2e},
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
