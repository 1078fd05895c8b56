"""Complete GPU runs of the two largest workloads against the oracle's
complete runs of the same inputs, stored by tests/golden/make_oracle_golden.py
(the oracle takes about an hour of CPU time for them, so its results are
stored rather than recomputed here):

  * large_d25 seed 1 (d = 25, N = 32, s = 10^4, 20 dB noise, r = 10): every
    increment's statistics and the detected set bit for bit, every
    coefficient within 1e-10 relative;
  * all 256 signals of the batch workload (d in 5..12, N in {16, 32, 64}, s
    log-uniform in [100, 2000], noiseless, r = 3) through one
    sfft_dimincr_batch call: each detected set bit for bit (SHA-256 of its
    rows), sample counts, and every coefficient within 1e-10 relative.

A selection whose cut the oracle recorded within 1e-9 (relative) of a tie or
of the threshold would make the comparison depend on rounding; the stored
gaps are checked first."""

import hashlib
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
LARGE = os.path.join(HERE, "golden", "oracle_large_d25_seed1.npz")
BATCH = os.path.join(HERE, "golden", "oracle_batch256_seed1.npz")
RTOL = 1e-10
GAP = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()


def _sha(freqs) -> str:
    return hashlib.sha256(np.ascontiguousarray(freqs, dtype=np.int32).tobytes()).hexdigest()


@pytest.mark.slow
def test_large_d25_complete_run_matches_oracle():
    z = np.load(LARGE)
    assert z["step_min_gap_rank"].min() > GAP and z["step_min_gap_thr"].min() > GAP, "degenerate seed (near tie)"
    sig, p = W.workload("large_d25", 1)
    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=1, s_local=p["s_local"],
                         b=p["b"], freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma, batch_reps=True)
    got = [(st["t"], st["n_line"], st["n_cand"], st["L"], st["sum_M"], st["attempts"], int(st["covered"]),
            st["samples"]) for st in out.steps]
    want = list(zip(*(z[f"step_{f}"].tolist() for f in ("t", "I_t", "n_candidates", "L", "sum_M", "attempts",
                                                          "covered", "samples"))))
    assert got == [tuple(w) for w in want]
    np.testing.assert_array_equal(out.freqs, z["freqs"].astype(np.int64))
    assert out.samples == int(z["samples"])
    ref = z["coeffs"]
    assert np.max(np.abs(out.coeffs - ref) / np.abs(ref)) < RTOL


@pytest.mark.slow
def test_batch256_all_signals_match_oracle():
    z = np.load(BATCH)
    assert z["min_gap_rank"].min() > GAP and z["min_gap_thr"].min() > GAP, "degenerate seed (near tie)"
    assert z["exact"].all()
    batch = W.batch_signals(256, seed=1)
    probs = [dict(d=sig.d, N=sig.N, s=prm["s"], s_local=prm["s_local"], r=prm["r"], b=prm["b"], theta=prm["theta"],
                  theta_mode=prm["theta_mode"], seed=1000 + i, freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma)
             for i, (sig, prm) in enumerate(batch)]
    outs = P.sfft_dimincr_batch(probs, concurrency=16)
    off = z["offsets"]
    for i, ((sig, _), out) in enumerate(zip(batch, outs)):
        assert out.freqs.shape[0] == int(z["n"][i]), f"signal {i}"
        assert _sha(out.freqs) == str(z["sha"][i]), f"signal {i}: detected set differs from the oracle's"
        assert out.samples == int(z["samples"][i]), f"signal {i}"
        # the oracle's coefficients: the planted ones plus the stored offsets
        ref = sig.coeffs + z["delta"][off[i]:off[i + 1]].astype(np.complex128)
        assert np.max(np.abs(out.coeffs - ref) / np.abs(ref)) < RTOL, f"signal {i}"


@pytest.mark.slow
def test_large_d25_complete_run_double_float_matches_oracle():
    """The same complete run with the Bluestein butterflies in double-float
    arithmetic (MR1L_FFT_DF): the same increments and set, and coefficients
    within the same 1e-10 of the oracle's FP64 values."""
    z = np.load(LARGE)
    assert z["step_min_gap_rank"].min() > GAP and z["step_min_gap_thr"].min() > GAP, "degenerate seed (near tie)"
    sig, p = W.workload("large_d25", 1)
    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=1, s_local=p["s_local"],
                         b=p["b"], freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma, batch_reps=True, fft="df")
    assert [st["L"] for st in out.steps] == z["step_L"].tolist()
    np.testing.assert_array_equal(out.freqs, z["freqs"].astype(np.int64))
    assert out.samples == int(z["samples"])
    ref = z["coeffs"]
    assert np.max(np.abs(out.coeffs - ref) / np.abs(ref)) < RTOL
