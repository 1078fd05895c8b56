#!/usr/bin/env python3
"""Writes the oracle's complete results on the two largest workloads, so that
the GPU tests can compare whole runs with them without re-running the oracle
(hours of CPU time at these sizes).  Every stored value comes from `oracle/`
alone (Algorithm 3 with Algorithms 1 and 2, numpy FFTs); the inputs come from
the seeded generators in `workloads`.

  large_d25, seed 1 (d = 25, N = 32, s = 10^4, log-uniform amplitudes in
  [1e-2, 10], 20 dB noise, r = 10): the detected frequencies (int8), their
  coefficients (complex128) and the statistics of every increment;

  batch256, seed 1 (256 noiseless signals, d in 5..12, N in {16, 32, 64}, s
  log-uniform in [100, 2000], r = 3, problem i seeded 1000 + i): per signal
  the SHA-256 of the detected set (int32 rows, lexicographic), its size, the
  sample count, the smallest selection gaps, whether the set is the planted
  support, and for those that are the oracle's coefficients as complex64
  offsets from the planted ones (planted + offset restores the oracle's value
  to about 1e-22 relative, far inside the 1e-10 parity tolerance).

  python tests/golden/make_oracle_golden.py [large|batch|all] [--workers W]

Runs the independent detection iterations of an increment (large) or the
independent signals (batch) in spawned worker processes.
"""

from __future__ import annotations

import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import sfft as osfft  # noqa: E402

LARGE_FILE = os.path.join(HERE, "oracle_large_d25_seed1.npz")
BATCH_FILE = os.path.join(HERE, "oracle_batch256_seed1.npz")
STEP_FIELDS = ("t", "I_t", "n_candidates", "L", "sum_M", "attempts", "covered", "samples")


def set_sha(freqs: np.ndarray) -> str:
    """SHA-256 of a frequency set as contiguous int32 rows (the order given)."""
    return hashlib.sha256(np.ascontiguousarray(freqs, dtype=np.int32).tobytes()).hexdigest()


def _steps(res) -> dict:
    out = {f"step_{f}": np.array([getattr(st, f) for st in res.steps], dtype=np.int64) for f in STEP_FIELDS}
    out["step_min_gap_rank"] = np.array([st.min_gap_rank for st in res.steps], dtype=np.float64)
    out["step_min_gap_thr"] = np.array([st.min_gap_thr for st in res.steps], dtype=np.float64)
    return out


def make_large(workers: int) -> None:
    sig, p = W.workload("large_d25", 1)
    t0 = time.time()
    with mp.get_context("spawn").Pool(workers) as pool:
        res = osfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=1,
                         rep_map=pool.map)
    dt = time.time() - t0
    assert np.all(np.abs(res.freqs) <= 127)
    np.savez_compressed(LARGE_FILE, freqs=res.freqs.astype(np.int8), coeffs=res.coeffs.astype(np.complex128),
                        samples=np.int64(res.samples), seconds=np.float64(dt), **_steps(res))
    print(f"large_d25: {res.freqs.shape[0]} frequencies, {res.samples} samples, {dt:.0f} s", flush=True)


def _batch_job(i: int):
    sig, prm = W.batch_signals(256, seed=1)[i]
    res = osfft.sfft(sig, prm["s"], prm["s_local"], prm["r"], prm["b"], prm["theta"], prm["theta_mode"],
                     seed=1000 + i)
    planted = sig.freqs.astype(np.int64)
    exact = res.freqs.shape == planted.shape and bool(np.array_equal(res.freqs, planted))
    delta = (res.coeffs - sig.coeffs).astype(np.complex64) if exact else None
    gr = min((st.min_gap_rank for st in res.steps), default=np.inf)
    gt = min((st.min_gap_thr for st in res.steps), default=np.inf)
    return i, set_sha(res.freqs), int(res.freqs.shape[0]), int(res.samples), gr, gt, exact, delta


def make_batch(workers: int) -> None:
    t0 = time.time()
    with mp.get_context("spawn").Pool(workers) as pool:
        rows = sorted(pool.map(_batch_job, range(256), chunksize=1))
    dt = time.time() - t0
    bad = [r[0] for r in rows if not r[6]]
    if bad:
        raise SystemExit(f"signals {bad}: the oracle's set is not the planted support; store them in full")
    np.savez_compressed(
        BATCH_FILE,
        sha=np.array([r[1] for r in rows]), n=np.array([r[2] for r in rows], dtype=np.int64),
        samples=np.array([r[3] for r in rows], dtype=np.int64),
        min_gap_rank=np.array([r[4] for r in rows], dtype=np.float64),
        min_gap_thr=np.array([r[5] for r in rows], dtype=np.float64),
        exact=np.array([r[6] for r in rows]),
        delta=np.concatenate([r[7] for r in rows]).astype(np.complex64),
        offsets=np.cumsum([0] + [r[2] for r in rows]).astype(np.int64), seconds=np.float64(dt))
    print(f"batch256: {sum(r[2] for r in rows)} frequencies over 256 signals, {dt:.0f} s", flush=True)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="?", default="all", choices=["large", "batch", "all"])
    ap.add_argument("--workers", type=int, default=min(10, os.cpu_count() or 1))
    a = ap.parse_args()
    if a.which in ("batch", "all"):
        make_batch(a.workers)
    if a.which in ("large", "all"):
        make_large(a.workers)
    return 0


if __name__ == "__main__":
    sys.exit(main())
