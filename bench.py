#!/usr/bin/env python3
"""Benchmark of the dimension-incremental sparse FFT over multiple rank-1
lattices (Algorithm 3) on GB300.

Headline workload (one "step" = one complete sparse FFT, every hot-path
stage: 1-D detections, Algorithm 1 lattice searches, sampling, Algorithm 2
transforms, selections):
  d = 25, N = 32 (search box [-32, 32]^25), s = 10^4 planted frequencies,
  |c| log-uniform in [1e-2, 10] with uniform phase, complex Gaussian noise at
  SNR 20 dB, r = 10 detection iterations fused per increment, theta = 1e-12
  relative, b = 10 (about 9.7e9 samples per solve).

Prints one JSON line (rank 0).  `value` is detected coefficients per second
over all ranks with the planted signal resident in HBM; `e2e` is the same
metric through the host-buffer API.  `roofline` describes the dominant
kernel (live CUDA-event timing of every library launch during the timed
region), `memory_bound_kernels` the HBM rate of every other kernel;
`cpu_baseline` is the CPU oracle on a bounded sample.  `secondary` holds the
d = 10 workload, the 256-signal batch and the differentiable transform, each
batched and plain.  A solve of the headline workload takes seconds, so the
timed steps are capped by a time budget (`steps` is the count timed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload large_d25|plain_d10|batch256|diff]
"""

from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import math
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

import workloads as W

METRIC = "detected coeffs/sec & lattice-transform HBM GB/s (% peak), batched vs plain, same GB300"
UNIT = "coeffs/s"
WORKLOAD = "large_d25"
HEADLINE_BUDGET_S = 50.0    # timed region of the headline form
SECONDARY_BUDGET_S = 12.0   # each other form and workload
DESCRIPTIONS = {
    "plain_d10": "plain_d10: d=10, N=32 (box [-32,32]^10), s=1000 planted, |c|~U[1,10] uniform phase, "
                 "SNR 40 dB, r=5, theta=1e-12 relative, b=10",
    "large_d25": "large_d25: d=25, N=32, s=10000 planted, |c| log-uniform in [1e-2,10], SNR 20 dB, r=10, "
                 "theta=1e-12 relative, b=10",
    "batch256": "batch256: 256 independent noiseless signals, d~U{5..12}, N in {16,32,64}, s log-uniform "
                "in [100,2000], r=3, theta=1e-12 relative, b=10",
}
FORMS = {
    "plain_d10": ("batched: the r repetitions of an increment fused in each launch",
                  "plain: one repetition per launch sequence"),
    "large_d25": ("batched: the r repetitions of an increment fused in each launch",
                  "plain: one repetition per launch sequence"),
    "batch256": ("batched: 16 signals in flight on their own streams, repetitions fused",
                 "plain: one signal after another on one stream, one repetition per launch sequence"),
}
L2_NOTE = "256 MiB buffer written before every timed GPU step (the workloads' arrays also exceed L2)"


def config_of(name: str, seed: int) -> dict:
    """The config object both arms print for a workload."""
    return {"workload": DESCRIPTIONS[name], "seed": seed, "l2": L2_NOTE}


class Workload:
    """Planted inputs of a named workload and its two GPU forms."""

    def __init__(self, name: str, seed: int, dev):
        import torch
        self.name = name
        if name == "batch256":
            self.items = W.batch_signals(256, seed)
        else:
            self.items = [W.workload(name, seed)]
        self.seeds = [seed * 1000 + i if name == "batch256" else seed for i in range(len(self.items))]
        self.dev_arrays = [(torch.from_numpy(np.ascontiguousarray(sig.freqs, dtype=np.int32)).to(dev),
                            torch.from_numpy(np.ascontiguousarray(sig.coeffs)).to(dev)) for sig, _ in self.items]

    def problems(self, host: bool, batched: bool, fft: str = "f64"):
        out = []
        for (sig, p), sd, (fd, cd) in zip(self.items, self.seeds, self.dev_arrays):
            out.append(dict(d=sig.d, N=sig.N, s=p["s"], s_local=p["s_local"], r=p["r"], b=p["b"],
                            theta=p["theta"], theta_mode=p["theta_mode"], seed=sd,
                            freqs=sig.freqs if host else fd, coeffs=sig.coeffs if host else cd,
                            sigma=sig.sigma, batch_reps=batched, fft=fft))
        return out

    def solve(self, batched: bool, host: bool = False, fft: str = "f64"):
        import paper_1711_05152_gb300 as P
        probs = self.problems(host, batched, fft)
        if self.name == "batch256" and batched:
            return P.sfft_dimincr_batch(probs, concurrency=16)
        outs = []
        for q in probs:
            outs.append(P.sfft_dimincr(q["d"], q["N"], q["s"], q["r"], q["theta"], q["theta_mode"], seed=q["seed"],
                                       s_local=q["s_local"], b=q["b"], freqs=q["freqs"], coeffs=q["coeffs"],
                                       sigma=q["sigma"], batch_reps=batched, fft=fft))
        return outs

    def exact(self, outs) -> bool:
        return all(set(map(tuple, o.freqs.tolist())) == set(map(tuple, sig.freqs.astype(int).tolist()))
                   for o, (sig, _) in zip(outs, self.items))
# FP64 pipe of GB300: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz max SM clock
SM_COUNT, FP64_FMA_PER_CLK, SM_MAX_GHZ = 152, 2, 2.070
FP64_PEAK_TFLOPS = SM_COUNT * FP64_FMA_PER_CLK * 2 * SM_MAX_GHZ / 1e3
L2_FLUSH_BYTES = 256 << 20
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


# the sources of the Bluestein kernels whose DRAM traffic profiles/traffic.json records
KERNEL_SOURCES = ("fft.cu", "fft.cuh", "arith.cuh", "common.cuh")


def _src_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1711_05152_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.file.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_scalar(x: float, op: str, world: int, device=None) -> float:
    """Across ranks: "max" (the slowest rank's time), "min" (a step count all
    ranks can run) or "sum" (all ranks' units).  A no-op for one rank; uses
    the default process group otherwise."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    ops = {"max": dist.ReduceOp.MAX, "min": dist.ReduceOp.MIN, "sum": dist.ReduceOp.SUM}
    dist.all_reduce(t, op=ops[op])
    return float(t.item())


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------
# CPU oracle legs
# ----------------------------------------------------------------------------

def oracle_sample(name: str, wl, outs) -> dict:
    """The oracle as it stands on a bounded sample of the same workload, its
    time scaled to the full job by the sample counts (the lattice FFT work per
    sample dominates every increment):
      plain_d10 / large_d25: increments t <= 6 / t <= 3 of the timed signal
      (about 10-20 s of one host core);
      batch256: the three signals with the smallest d s (2N+1), complete."""
    from oracle import sfft as osfft
    full_samples = sum(o.samples for o in outs)
    full_detected = sum(o.freqs.shape[0] for o in outs)
    t0 = time.perf_counter()
    if name == "batch256":
        cost = [sig.d * p["s"] * (2 * sig.N + 1) for sig, p in wl.items]
        pick = list(np.argsort(cost)[:3])
        sample_samples = 0
        for i in pick:
            sig, p = wl.items[i]
            res = osfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"],
                             seed=wl.seeds[i])
            sample_samples += res.samples
        what = f"oracle on signals {pick} of batch256 (complete solves)"
    else:
        t_stop = 6 if name == "plain_d10" else 3
        sig, p = wl.items[0]
        res = osfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=wl.seeds[0],
                         t_stop=t_stop)
        sample_samples = res.samples
        what = f"oracle increments t<={t_stop} of {name} seed {wl.seeds[0]}"
    dt = time.perf_counter() - t0
    scaled = dt * full_samples / max(sample_samples, 1)
    return {"value": full_detected / scaled, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host": f"{host_cpu()}, {host_cores()} cores",
            "sample": f"{what}: {sample_samples} of {full_samples} samples in {dt:.1f} s (numpy, one "
                      f"thread), time scaled by samples"}


def _oracle_job(job):
    """One worker of the all-cores leg: the bounded oracle sample on one
    signal of the workload (its own seed).  Returns (samples, start, end) on
    the host's wall clock."""
    name, seed, t_stop = job
    from oracle import sfft as osfft
    sig, p = W.workload(name, seed)
    t0 = time.time()
    res = osfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=seed,
                     t_stop=t_stop)
    return res.samples, t0, time.time()


def host_cpu() -> str:
    """The host's CPU model (lscpu's "Model name", else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_all_cores(name: str, wl, outs, cores: int | None = None, t_stop: int | None = None) -> dict:
    """The same bounded oracle sample on every host core at once: one
    single-threaded process per core (spawned, so no process inherits a CUDA
    context), each on its own signal of the workload, seeds seed, seed + 1, ...
    Throughput = all samples / the wall time from the first start to the last
    end, scaled to detected coefficients by the timed job's coefficients per
    sample."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    cores = cores or host_cores()
    if t_stop is None:
        t_stop = 6 if name == "plain_d10" else 3
    full_samples = sum(o.samples for o in outs)
    full_detected = sum(o.freqs.shape[0] for o in outs)
    jobs = [(name, wl.seeds[0] + i, t_stop) for i in range(cores)]
    # a worker that dies raises BrokenProcessPool here instead of hanging
    with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
        res = list(pool.map(_oracle_job, jobs))
    samples = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    value = samples / wall * full_detected / max(full_samples, 1)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "host": f"{host_cpu()}, {host_cores()} cores",
            "sample": f"oracle increments t<={t_stop} of {name} seeds {jobs[0][1]}..{jobs[-1][1]}, one "
                      f"single-threaded process per core: {samples} samples in {wall:.1f} s wall, "
                      f"scaled by the timed job's coefficients per sample"}


ORACLE_LARGE = os.path.join(ROOT, "tests", "golden", "oracle_large_d25_seed1.npz")


def _oracle_full_totals(name: str, seed: int):
    """(samples, detected) of the oracle's complete run of a workload, when
    the oracle's stored run exists (written by tests/golden/make_oracle_golden.py)."""
    if name == "large_d25" and seed == 1 and os.path.exists(ORACLE_LARGE):
        z = np.load(ORACLE_LARGE)
        return int(z["samples"]), int(z["freqs"].shape[0])
    return None


def run_reference(args):
    """The CPU oracle as it stands (numpy, one thread) on the same workload,
    metric and config.  plain_d10: complete solves.  large_d25: a complete
    oracle solve takes hours, so each step is the bounded sample of
    increments t <= 3, and the rate is scaled to the complete job by samples
    (the oracle's own complete run gives its total samples and detected
    coefficients).  Steps stop once about 150 s have been spent."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import sfft as osfft
    name = args.workload if args.workload in ("plain_d10", "large_d25") else WORKLOAD
    tiny, tp = W.workload("tiny_d3", 1)
    for _ in range(args.warmup):
        osfft.sfft(tiny, tp["s"], tp["s_local"], tp["r"], tp["b"], tp["theta"], tp["theta_mode"], seed=1)
    sig, p = W.workload(name, args.seed)
    t_stop = 3 if name == "large_d25" else None
    totals = _oracle_full_totals(name, args.seed) if t_stop else None
    if t_stop and totals is None:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle's complete run of this workload and "
                                                              "seed (its sample total) is not stored"}), flush=True)
        return 0
    times, detected, samples = [], 0, 0
    budget = 150.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = osfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=args.seed,
                         t_stop=t_stop)
        times.append(time.perf_counter() - t0)
        detected += res.freqs.shape[0]
        samples += res.samples
        if sum(times) + times[-1] > budget:
            break
    total = sum(times)
    if t_stop:
        full_samples, full_detected = totals
        value = samples / total * full_detected / full_samples
        ms_step = 1e3 * total / len(times) * full_samples / (samples / len(times))
        sample = (f"{len(times)} oracle runs of increments t<={t_stop} of {name} seed {args.seed} (of --steps "
                  f"{args.steps}; capped at about {budget:.0f} s), {samples // len(times)} of the complete run's "
                  f"{full_samples} samples each, time scaled by samples; warm-up: {args.warmup} solves of the d=3 "
                  f"workload")
    else:
        value = detected / total
        ms_step = 1e3 * total / len(times)
        sample = (f"{len(times)} full {name} oracle solves (of --steps {args.steps}; capped at about "
                  f"{budget:.0f} s); warm-up: {args.warmup} solves of the d=3 workload")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(name, args.seed), "form": "CPU oracle (numpy, pocketfft)",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": f"{host_cpu()}, {host_cores()} cores"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def fast_profile(prof) -> dict:
    """Kernel shares of the double-float form and the FP64-equivalent rate of
    its dominant kernel (FFT flops by the 5 n log2 n convention per second)."""
    if not prof:
        return {}
    tot = sum(v["ms"] for v in prof.values()) or 1.0
    name, dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    out = {"kernel_share": {k: round(v["ms"] / tot, 4) for k, v in
                            sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]}}
    if dom["flops"]:
        rate = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        out["dominant"] = {"kernel": name, "fp64_equivalent_tflops": rate,
                           "over_fp64_pipe_peak": rate / FP64_PEAK_TFLOPS}
    return out


def timed_solves(wl, batched, *, fft="f64", warmup, steps, min_warmup, budget_s, flush, profile=False,
                 host=False, world=1, dev=None):
    """W warm-up solves (at least min_warmup; more up to `warmup` while they
    take under 20 s), then K timed solves with K = min(steps, budget_s / the
    median warm-up time) (at least 2; the smallest K of all ranks), the L2
    flushed before each.  Device time from CUDA events around each solve
    (host=False, inputs resident in HBM) or host wall time around each solve
    through the host-buffer API (host=True: copies of inputs and results
    inside the timed region)."""
    import torch

    import paper_1711_05152_gb300 as P
    wtimes = []
    while len(wtimes) < max(min_warmup, 1):
        t0 = time.perf_counter()
        wl.solve(batched, host=host, fft=fft)
        torch.cuda.synchronize()
        wtimes.append(time.perf_counter() - t0)
        if len(wtimes) >= min_warmup and (len(wtimes) >= warmup or sum(wtimes) > 20.0):
            break
    est = statistics.median(wtimes)
    k = int(min(steps, max(2, math.floor(budget_s / max(est, 1e-6)))))
    k = int(reduce_scalar(float(k), "min", world, dev))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if profile:
        P.prof_reset()
        P.prof_enable(True)
    launches0 = P.prof_launches()
    total_ms, samp_ms, detected, last = 0.0, 0.0, 0, None
    for _ in range(k):
        flush.fill_(1)                       # evict L2 between steps (not timed)
        torch.cuda.synchronize()
        if host:
            t0 = time.perf_counter()
            last = wl.solve(batched, host=True, fft=fft)
            total_ms += 1e3 * (time.perf_counter() - t0)
        else:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            last = wl.solve(batched, fft=fft)
            e1.record()
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
        samp_ms += sum(o.ms_sampling for o in last)
        detected += sum(o.freqs.shape[0] for o in last)
    launches = P.prof_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    prof = None
    if profile:
        P.prof_enable(False)
        prof = P.prof_read()
    return dict(ms=reduce_scalar(total_ms, "max", world, dev), detected=reduce_scalar(float(detected), "sum", world, dev),
                launches=launches, prof=prof, last=last, samp_ms=reduce_scalar(samp_ms, "max", world, dev), steps=k,
                warmup=len(wtimes))


def _rate(m) -> float:
    return m["detected"] / (m["ms"] / 1e3)


def memory_bound_kernels(prof, hbm) -> dict:
    """Achieved algorithmic GB/s of every kernel that is not a Bluestein FFT
    pass (live CUDA-event times of the timed region), against the HBM peak."""
    out = {}
    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]):
        if k.startswith("blue_") or not v["bytes"] or not v["ms"]:
            continue
        gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9
        out[k] = {"launches": v["launches"], "ms": round(v["ms"], 4), "GBps": round(gbs, 1),
                  "frac_of_hbm": round(gbs / hbm, 4), "bytes_per_launch": v["bytes"] / v["launches"]}
    return out


def measure_diff(dev, steps, warmup, budget_s, flush, seed=1) -> dict:
    """The differentiable transform on 10^5 frequencies in [-64, 64]^20 with
    64 complex right-hand sides: one step = forward Algorithm 2 plus the
    backward pass (the ADJOINT kernel path) of ||reconstruct(y) - c||^2
    through the torch.autograd.Function, device-timed.  The plain form makes
    one forward and one adjoint call per right-hand side."""
    import torch

    import paper_1711_05152_gb300 as P
    from paper_1711_05152_gb300 import autograd as AG
    I, rng = W.diff_problem(100000, 20, 64, 64, seed=seed)
    pl = P.plan_search(I, seed=seed + 1)
    y0 = torch.from_numpy(W.complex_normal(rng, (64, pl.sum_M))).to(dev)
    c = torch.from_numpy(W.complex_normal(rng, (64, pl.nI))).to(dev)

    def batched():
        y = y0.detach().requires_grad_(True)
        loss = (AG.reconstruct(y, pl) - c).abs().pow(2).sum()
        loss.backward()
        return y.grad

    def plain():
        return torch.stack([pl.evaluate(2.0 * (pl.reconstruct(y0[h]) - c[h]), P.MR1L_ADJOINT) for h in range(64)])

    def timed(fn, w, k_max):
        t_w = []
        for _ in range(max(w, 1)):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            t_w.append(time.perf_counter() - t0)
        k = int(min(k_max, max(2, math.floor(budget_s / max(statistics.median(t_w), 1e-6)))))
        total = 0.0
        g = None
        for _ in range(k):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g = fn()
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        return total / k, k, g

    b_ms, b_k, gb = timed(batched, warmup, steps)
    p_ms, p_k, gp = timed(plain, 1, steps)
    diff = float((gb - gp).abs().max() / gp.abs().max())
    return {"workload": "diff: 10^5 frequencies in [-64,64]^20 (Algorithm 1 lattice, L=%d, sum M=%d), 64 complex "
                        "right-hand sides; one step = forward + backward of ||reconstruct(y)-c||^2" % (pl.L, pl.sum_M),
            "value": 64 / (b_ms / 1e3), "unit": "right-hand sides/s (forward + adjoint)", "ms_per_step": b_ms,
            "steps": b_k, "plain": {"value": 64 / (p_ms / 1e3), "ms_per_step": p_ms, "steps": p_k,
                                    "form": "one forward and one adjoint call per right-hand side"},
            "batched_over_plain": p_ms / b_ms, "form": "torch.autograd.Function over all 64 right-hand sides",
            "max_rel_grad_diff_vs_plain": diff}


def run_ours(args):
    import torch

    import paper_1711_05152_gb300 as P

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.lib()
    seed = args.seed + rank                      # independent signals per GPU (weak scaling)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    common = dict(flush=flush, world=world, dev=dev)

    if args.workload == "diff":
        d = measure_diff(dev, args.steps, max(args.warmup, 3), HEADLINE_BUDGET_S, flush, seed)
        if rank == 0:
            print(json.dumps({"metric": METRIC, **d, "n_gpus": world, "warmup": max(args.warmup, 3),
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                              "data": "synthetic", "config": {"workload": d["workload"], "seed": args.seed}}),
                  flush=True)
        return 0

    wl = Workload(args.workload, seed, dev)
    clocks = ClockSampler(local)
    clocks.start()
    bat = timed_solves(wl, True, warmup=args.warmup, steps=args.steps, min_warmup=3, budget_s=HEADLINE_BUDGET_S,
                       profile=True, **common)
    clock_info = clocks.stop()
    sec = SECONDARY_BUDGET_S
    plain = timed_solves(wl, False, warmup=1, steps=args.steps, min_warmup=1, budget_s=sec, **common)
    fast = None if args.no_fast_fft else timed_solves(wl, True, fft="df", warmup=1, steps=args.steps, min_warmup=1,
                                                       budget_s=sec, profile=True, **common)
    e2e = timed_solves(wl, True, host=True, warmup=1, steps=args.steps, min_warmup=1, budget_s=sec, **common)
    h2d = sum(sig.freqs.size * 4 + sig.coeffs.size * 16 for sig, _ in wl.items)
    d2h = int(sum(o.freqs.size * 4 + o.coeffs.size * 16 for o in e2e["last"]))

    # The batched form of the 256-signal workload runs 16 streams at once, so a
    # kernel's events also cover time its CTAs wait behind other streams; its
    # per-kernel times come from one extra, untimed solve of the single-stream
    # form instead.
    prof_src = "the batched timed region"
    prof = bat["prof"] or {}
    if args.workload == "batch256":
        torch.cuda.synchronize()
        P.prof_reset()
        P.prof_enable(True)
        wl.solve(False)
        torch.cuda.synchronize()
        P.prof_enable(False)
        prof = P.prof_read()
        prof_src = "one extra solve of the single-stream form (the batched form overlaps 16 streams)"

    # the other workloads, batched and plain (and the differentiable transform)
    secondary = {}
    if not args.no_secondary:
        for name in ("plain_d10", "batch256"):
            if name == args.workload:
                continue
            w2 = Workload(name, seed, dev)
            b2 = timed_solves(w2, True, warmup=3, steps=args.steps, min_warmup=3, budget_s=sec, **common)
            p2 = timed_solves(w2, False, warmup=1, steps=args.steps, min_warmup=1, budget_s=sec, **common)
            secondary[name] = {"workload": DESCRIPTIONS[name], "value": _rate(b2), "unit": UNIT,
                               "ms_per_step": b2["ms"] / b2["steps"], "steps": b2["steps"],
                               "form": FORMS[name][0], "plain": {"value": _rate(p2), "ms_per_step": p2["ms"] / p2["steps"],
                                                                 "steps": p2["steps"], "form": FORMS[name][1]},
                               "batched_over_plain": (p2["ms"] / p2["steps"]) / (b2["ms"] / b2["steps"]),
                               "support_exact": w2.exact(b2["last"]),
                               "excluding_sampling": ({"value": b2["detected"] / ((b2["ms"] - b2["samp_ms"]) / 1e3)}
                                                      if name != "batch256" else None)}
            del w2
        secondary["diff"] = measure_diff(dev, args.steps, 3, sec, flush, seed)

    if rank != 0:
        return 0

    last = bat["last"]
    value = _rate(bat)
    total_prof_ms = sum(v["ms"] for v in prof.values()) or 1.0
    dom_name, dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else (None, None)
    peaks, peak_src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    roofline = None
    if dom is not None:
        per_launch_ms = dom["ms"] / dom["launches"]
        traffic = None
        try:
            tr = json.load(open(TRAFFIC_FILE))
            ent = tr.get("kernels", {}).get(dom_name)
            if ent and tr.get("src_hash") == _src_hash():
                traffic = ent["dram_over_algorithmic"] * dom["bytes"] / dom["launches"]
        except (OSError, ValueError, KeyError):
            traffic = None
        if dom_name.startswith("blue_"):
            achieved = dom["flops"] / dom["launches"] / (per_launch_ms * 1e-3) / 1e12
            roofline = {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                        "peak_source": "FP64 pipe: 152 SM x 2 FMA/clk x 2 flop x 2.07 GHz (derived)",
                        "share_of_kernel_time": dom["ms"] / total_prof_ms, "launches": dom["launches"],
                        "timed_in": prof_src}
        else:
            achieved = dom["bytes"] / dom["launches"] / (per_launch_ms * 1e-3) / 1e9
            roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src,
                        "share_of_kernel_time": dom["ms"] / total_prof_ms, "launches": dom["launches"],
                        "timed_in": prof_src}

    # lattice transform (Algorithm 2): Bluestein reconstruct passes + gather
    recon = [k for k in prof if k.endswith("_recon") or k == "gather_kernel"]
    recon_ms = sum(prof[k]["ms"] for k in recon)
    alg_bytes = 0
    for o, (sig, p) in zip(last, wl.items):
        for st in o.steps:
            reps = p["r"] if st["t"] < sig.d else 1
            alg_bytes += reps * (16 * st["sum_M"] + 24 * st["n_cand"])
    alg_bytes *= bat["steps"] if args.workload != "batch256" else 1
    lat_gbs = alg_bytes / (recon_ms * 1e-3) / 1e9 if recon_ms else None
    kernel_share = {k: round(v["ms"] / total_prof_ms, 4) for k, v in
                    sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]}

    cpu = cpu_all = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.workload, wl, last)
        if args.workload != "batch256":
            cpu_all = oracle_sample_all_cores(args.workload, wl, last)

    form_b, form_p = FORMS[args.workload]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": bat["steps"],
        "steps_requested": args.steps, "warmup": bat["warmup"], "warmup_requested": args.warmup,
        "ms_per_step": bat["ms"] / bat["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args.workload, args.seed),
        "form": form_b, "parallelism": f"{world} GPU(s), independent signals per GPU",
        "budget": f"timed steps = min(--steps, {HEADLINE_BUDGET_S:.0f} s / the median warm-up solve), at least 2",
        "plain": {"value": _rate(plain), "ms_per_step": plain["ms"] / plain["steps"], "steps": plain["steps"],
                  "form": form_p},
        "batched_over_plain": (plain["ms"] / plain["steps"]) / (bat["ms"] / bat["steps"]),
        # the paper's runtimes leave out sampling: the same rate with the time of
        # the sampler's kernels (GPU events around them) taken off the step
        "excluding_sampling": ({"value": bat["detected"] / ((bat["ms"] - bat["samp_ms"]) / 1e3),
                                "ms_per_step": (bat["ms"] - bat["samp_ms"]) / bat["steps"],
                                "sampling_ms_per_step": bat["samp_ms"] / bat["steps"]}
                               if args.workload != "batch256" and bat["ms"] > bat["samp_ms"] else None),
        "fast_fft": None if fast is None else {
            "value": _rate(fast), "ms_per_step": fast["ms"] / fast["steps"], "steps": fast["steps"],
            "form": "batched, Bluestein butterflies in double-float (FP32 pairs) instead of FP64",
            "same_support_as_f64": all(np.array_equal(a.freqs, b.freqs) for a, b in zip(fast["last"], last)),
            "max_rel_coeff_diff_vs_f64": max((float(np.max(np.abs(a.coeffs - b.coeffs) / np.abs(b.coeffs)))
                                             for a, b in zip(fast["last"], last) if b.coeffs.size and
                                             np.array_equal(a.freqs, b.freqs)), default=None),
            "gpu_launches": int(fast["launches"]), **fast_profile(fast["prof"])},
        "e2e": {"value": _rate(e2e), "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h,
                "steps": e2e["steps"], "l2": "flushed before every step, as in the device-timed loop"},
        "gpu_launches": int(bat["launches"]),
        "roofline": roofline,
        "memory_bound_kernels": memory_bound_kernels(prof, hbm),
        "lattice_transform": {"GBps": lat_gbs, "frac_of_hbm": (lat_gbs / hbm) if lat_gbs else None,
                              "hbm_peak": hbm, "ms_per_step": recon_ms / bat["steps"],
                              "note": "Algorithm 2 passes (Bluestein + gather), algorithmic bytes "
                                      "16*sum_M + 24*|J| per pass; FP64-bound, see roofline"},
        "kernel_share": kernel_share,
        # summed kernel time of the timed region per step (against ms_per_step:
        # the share of the step the device spends in kernels)
        "kernel_ms_per_step": (total_prof_ms / bat["steps"]) if prof and args.workload != "batch256" else None,
        "tile_tuner": tile_summary(P.tune_read()),
        "clocks": clock_info,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "detected": int(sum(o.freqs.shape[0] for o in last)), "support_exact": wl.exact(last),
        "samples": int(sum(o.samples for o in last)),
        "secondary": secondary or None,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def tile_summary(table):
    """Column/row tile chosen per Bluestein length, mode and arithmetic
    ("P/mode[/df]": [col_tile, row_tile]) by the library's tile tuner."""
    return {f"{e['P']}/{e['mode']}{'/df' if e['df'] else ''}": [e["col_tile"], e["row_tile"]]
            for e in sorted(table, key=lambda e: (e["df"], e["P"], e["mode"]))}


# ---------------------------------------------------------------------------
# The paper's statistical experiments (Tables 5.1, 5.2, 5.4) on the GPU path
# ---------------------------------------------------------------------------
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _paper_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


def _run_stats(problems, sigs, fft, concurrency=16):
    """Detected-set and coefficient statistics of a list of planted problems."""
    import paper_1711_05152_gb300 as P
    for q in problems:
        q["fft"] = fft
    outs = P.sfft_dimincr_batch(problems, concurrency=concurrency)
    samples, correct, success, err = [], [], [], []
    for sig, o in zip(sigs, outs):
        truth = {tuple(f): c for f, c in zip(sig.freqs.astype(int).tolist(), sig.coeffs)}
        got = {tuple(f): c for f, c in zip(o.freqs.tolist(), o.coeffs)}
        keys = set(truth) | set(got)
        num = sum(abs(got.get(k, 0.0) - truth.get(k, 0.0)) ** 2 for k in keys)
        samples.append(o.samples)
        correct.append(len(set(truth) & set(got)))
        success.append(set(truth) == set(got))
        err.append(float(np.sqrt(num / sum(abs(c) ** 2 for c in truth.values()))))
    return {"max_samples": int(max(samples)), "mean_samples": float(np.mean(samples)), "min_correct": int(min(correct)),
            "success_rate": float(np.mean(success)), "max_rel_l2": float(max(err))}


def _bspline_l2_error(desc, out) -> float:
    """Relative L2(T^d) error of a Section 5.3 run (the formula of that
    section): sqrt(||f||^2 - sum_I |f^_k|^2 + sum_I |p~_k - f^_k|^2) / ||f||
    with the exact coefficients f^_k = sum_g [k = 0 off S_g] prod_{t in S_g}
    C_m sinc(pi k_t / m)^m (-1)^k_t, C_m = (m B_2m(m))^-1/2 and
    ||f||^2 = G + sum_{g != h} C_g^|S_g| C_h^|S_h| (disjoint groups)."""
    def c_m(m):
        b2m = sum((-1) ** j * math.comb(2 * m, j) * (m - j) ** (2 * m - 1) for j in range(m + 1))
        return 1.0 / math.sqrt(m * b2m / math.factorial(2 * m - 1))

    K = np.asarray(out.freqs, dtype=np.int64)
    fk = np.zeros(K.shape[0])
    means = []
    for dims, m in zip(desc.groups, desc.orders):
        C = c_m(m)
        means.append(C ** len(dims))
        off = [t for t in range(desc.d) if t not in dims]
        val = np.all(K[:, off] == 0, axis=1).astype(np.float64)
        for t in dims:
            x = np.pi * K[:, t] / m
            sinc = np.where(K[:, t] == 0, 1.0, np.sin(x) / np.where(K[:, t] == 0, 1.0, x))
            val = val * C * sinc ** m * np.where(K[:, t] % 2 == 0, 1.0, -1.0)
        fk += val
    n2 = len(means) + sum(a * b for i, a in enumerate(means) for j, b in enumerate(means) if i != j)
    e2 = n2 - float(np.sum(fk ** 2)) + float(np.sum(np.abs(out.coeffs - fk) ** 2))
    return math.sqrt(max(e2, 0.0) / n2)


def run_paper_table(args):
    """One JSON line per row of the paper's Table 5.1 (samples and errors,
    Section 5.1), 5.2 (success rates over r and the absolute threshold), 5.4
    (noise, Section 5.2) or 5.7 (the B-spline function of Section 5.3,
    s-sparse), measured on the GPU path with the paper's protocol and seeded
    synthetic signals, beside the paper's printed values
    (tests/golden/paper_table_*.txt)."""
    import paper_1711_05152_gb300 as P
    reps, base = args.reps, 1000 * args.seed
    if args.paper_table == "5.1":
        sizes = {int(x) for x in args.sizes.split(",")}
        for d, supp, pmax, perr in _paper_rows("paper_table_5_1.txt"):
            d, supp = int(d), int(supp)
            if supp not in sizes:
                continue
            t0 = time.time()
            sigs = [W.planted_signal(d, 32, supp, seed=base + i, model="box") for i in range(reps)]
            probs = [dict(d=d, N=32, s=supp, s_local=supp, r=1, b=10, theta=1e-12, theta_mode="abs",
                          seed=base + i, freqs=g.freqs, coeffs=g.coeffs, redraw=args.redraw)
                     for i, g in enumerate(sigs)]
            # |supp| = 1e5 solves hold about 25 GB of device buffers each: two at a time
            st = _run_stats(probs, sigs, args.fft, concurrency=16 if supp < 100000 else 2)
            print(json.dumps({"paper_table": "5.1", "d": d, "supp": supp, "reps": reps, "fft": args.fft,
                              "redraw": args.redraw, **st,
                              "paper": {"max_samples": int(pmax), "max_rel_l2": perr},
                              "samples_over_paper": st["max_samples"] / pmax,
                              "seconds": round(time.time() - t0, 2)}), flush=True)
    elif args.paper_table == "5.2":
        for r, delta, pmin, prate in _paper_rows("paper_table_5_2.txt"):
            t0 = time.time()
            sigs = [W.planted_signal(5, 32, 1000, seed=base + i, model="unimodular") for i in range(reps)]
            probs = [dict(d=5, N=32, s=1000, s_local=1000, r=int(r), b=10, theta=delta, theta_mode="abs",
                          seed=base + i, freqs=g.freqs, coeffs=g.coeffs) for i, g in enumerate(sigs)]
            st = _run_stats(probs, sigs, args.fft)
            print(json.dumps({"paper_table": "5.2", "r": int(r), "delta": delta, "reps": reps, "fft": args.fft,
                              **st, "paper": {"min_correct": int(pmin), "success_rate": prate, "reps": 1000},
                              "seconds": round(time.time() - t0, 2)}), flush=True)
    elif args.paper_table == "5.7":
        # Section 5.3, s-sparse strategy; s_local = 2 s for the intermediate increments
        for N, s_, pmax, perr in _paper_rows("paper_table_5_7.txt"):
            N, s_ = int(N), int(s_)
            t0 = time.time()
            desc = W.paper_bspline(N)
            samples, errs = [], []
            for i in range(reps):
                o = P.sfft_dimincr(10, N, s_, 5, 1e-12, "abs", seed=base + i, s_local=2 * s_, function=desc,
                                   batch_reps=True, fft=args.fft)
                samples.append(o.samples)
                errs.append(_bspline_l2_error(desc, o))
            print(json.dumps({"paper_table": "5.7", "N": N, "s": s_, "s_local": 2 * s_, "reps": reps,
                              "fft": args.fft, "max_samples": int(max(samples)), "max_rel_l2": max(errs),
                              "paper": {"max_samples": int(pmax), "max_rel_l2": perr},
                              "samples_over_paper": max(samples) / pmax,
                              "seconds": round(time.time() - t0, 2)}), flush=True)
    else:
        for snr, r, pmax, pmin, prate, perr in _paper_rows("paper_table_5_4.txt"):
            t0 = time.time()
            sigs = [W.planted_signal(10, 32, 1000, seed=base + i, model="unimodular", snr_db=snr)
                    for i in range(reps)]
            probs = [dict(d=10, N=32, s=1000, s_local=1000, r=int(r), b=10, theta=1e-12, theta_mode="abs",
                          seed=base + i, freqs=g.freqs, coeffs=g.coeffs, sigma=g.sigma) for i, g in enumerate(sigs)]
            st = _run_stats(probs, sigs, args.fft)
            print(json.dumps({"paper_table": "5.4", "snr_db": int(snr), "r": int(r), "reps": reps, "fft": args.fft,
                              **st, "paper": {"max_samples": int(pmax), "min_correct": int(pmin),
                                              "success_rate": prate, "max_rel_l2": perr, "reps": 1000},
                              "seconds": round(time.time() - t0, 2)}), flush=True)
    return 0


def run_kernel_case(args):
    """The lattice transform alone at a workload-like size: |J| = 65 x
    `--kc-prefix` candidates in Z^10 (a prefix set times the 65 values of the
    last component, as in the d = 10 workload), its Algorithm 1 lattice and
    `--kc-rhs` right-hand sides (5): one warm-up and one measured reconstruct + adjoint, two
    evaluations of sparse coefficient vectors (every 35th and every 400th
    coefficient kept, as in the planted sampler), then the memory-bound steps
    around them on data of the same size (the selection of the 5 coefficient
    vectors, a small-segment selection, the lattice noise of the 5 passes).
    For ncu captures."""
    import torch

    import paper_1711_05152_gb300 as P
    rng = np.random.default_rng(args.seed)
    npre = args.kc_prefix
    pre = np.unique(rng.integers(-32, 33, size=(npre + npre // 10 + 10, 9)), axis=0)[:npre]
    J = np.concatenate([np.repeat(pre, 65, axis=0), np.tile(np.arange(-32, 33), npre)[:, None]], axis=1)
    pl = P.plan_search(J, seed=args.seed, fft=args.fft)
    y = torch.from_numpy(W.complex_normal(rng, (args.kc_rhs, pl.sum_M))).cuda()
    for _ in range(2):
        c = pl.reconstruct(y)
        pl.evaluate(c, P.MR1L_ADJOINT)
    # sparse evaluations (as in the planted sampler): about 8 and 1 non-zero
    # bins per column of the evaluation column pass
    for keep in (35, 400):
        cs = torch.zeros_like(c)
        cs[:, ::keep] = c[:, ::keep]
        for _ in range(2):
            pl.evaluate(cs, P.MR1L_EVAL)
    for _ in range(2):
        P.select(c, 1000, 1e-12, "rel")
        P.select(c[:, :50000].contiguous(), 1000, 1e-12, "rel")
        for h in range(args.kc_rhs):
            P.lattice_noise(args.seed, 5, h, pl.M, 1.0)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": "reconstruct+adjoint, selections, noise", "fft": args.fft, "n": int(J.shape[0]),
                      "L": pl.L, "sum_M": int(pl.sum_M), "M0": int(pl.M[0])}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(DESCRIPTIONS) + ["diff"],
                    help="large_d25 (default line), plain_d10, batch256, or diff (the differentiable transform)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the other workloads of the default line")
    ap.add_argument("--no-fast-fft", action="store_true", help="skip the double-float FFT form")
    ap.add_argument("--fft", default="f64", choices=["f64", "df"], help="arithmetic of --kernel-case and --paper-table")
    ap.add_argument("--kc-prefix", type=int, default=1000,
                    help="prefix rows of the --kernel-case candidate set (|J| = 65 x this)")
    ap.add_argument("--kc-rhs", type=int, default=5, help="right-hand sides of the --kernel-case transforms")
    ap.add_argument("--kernel-case", action="store_true",
                    help="run only the lattice transform at the workload size (for ncu captures)")
    ap.add_argument("--paper-table", choices=["5.1", "5.2", "5.4", "5.7"],
                    help="rerun one of the paper's statistical experiments on the GPU path")
    ap.add_argument("--reps", type=int, default=10, help="repetitions per row of --paper-table")
    ap.add_argument("--sizes", default="1000,10000", help="sparsities of the --paper-table 5.1 rows")
    ap.add_argument("--redraw", action="store_true",
                    help="--paper-table 5.1 with the redraw rule of Algorithm 1 (the remark after it)")
    args = ap.parse_args()
    if args.kernel_case:
        return run_kernel_case(args)
    if args.paper_table:
        return run_paper_table(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
