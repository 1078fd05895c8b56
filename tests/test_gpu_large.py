"""The large workload (d = 25, N = 32, s = 10^4, log-uniform amplitudes in
[1e-2, 10], 20 dB noise, r = 10 repetitions fused per increment).

The oracle needs about an hour for the whole run (tests/test_gpu_oracle_runs.py
compares the GPU with its stored complete run); here
the first increments (t <= 3, where |J_3| = 274,625 candidates and each
lattice has about 5.5e5 nodes) are compared with the oracle bit for bit, and
the full run is checked against what the planted signal fixes at any size."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
import workloads as W
from oracle import sfft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()


@pytest.mark.slow
def test_large_first_increments_match_oracle():
    sig, p = W.workload("large_d25", 1)
    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=1, b=p["b"],
                         freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma, batch_reps=True, t_stop=3)
    ref = sfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=1, t_stop=3)
    assert min(st.min_gap_rank for st in ref.steps) > 1e-9, "degenerate seed (near tie)"
    for st, rs in zip(out.steps, ref.steps):
        assert (st["n_line"], st["n_cand"], st["L"], st["attempts"], st["samples"]) == \
            (rs.I_t, rs.n_candidates, rs.L, rs.attempts, rs.samples)
    np.testing.assert_array_equal(out.freqs, ref.freqs)
    assert out.samples == ref.samples


@pytest.mark.slow
def test_large_full_run_properties():
    """Every increment covers its candidates; no false frequency carries more
    than the noise level; every planted coefficient well above the noise is
    detected, with its value within the noise-limited error."""
    sig, p = W.workload("large_d25", 1)
    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=1, b=p["b"],
                         freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma, batch_reps=True)
    assert out.freqs.shape[0] <= p["s"]
    assert all(st["covered"] for st in out.steps)
    truth = {tuple(f): c for f, c in zip(sig.freqs.astype(int).tolist(), sig.coeffs)}
    got = {tuple(f): c for f, c in zip(out.freqs.tolist(), out.coeffs)}
    # each reconstructed coefficient averages >= 1 lattice of >= 5e5 noisy
    # samples: its noise std is at most sigma / sqrt(5e5)
    noise = sig.sigma / np.sqrt(5e5)
    for f, c in got.items():
        if f in truth:
            assert abs(c - truth[f]) < 8 * noise + 1e-9 * abs(truth[f])
        else:
            assert abs(c) < 8 * noise
    strong = [f for f, c in truth.items() if abs(c) > 20 * noise]
    assert all(f in got for f in strong)


@pytest.mark.slow
def test_large_first_increments_redraw_match_oracle():
    """The redraw rule of Algorithm 1 at the large workload's sizes (|J_3| =
    274,625 candidates): the first increments against the oracle."""
    sig, p = W.workload("large_d25", 1)
    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=1, b=p["b"],
                         freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma, batch_reps=True, t_stop=3, redraw=True)
    ref = sfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=1, t_stop=3,
                    redraw=True)
    assert min(st.min_gap_rank for st in ref.steps) > 1e-9, "degenerate seed (near tie)"
    for st, rs in zip(out.steps, ref.steps):
        assert (st["n_line"], st["n_cand"], st["L"], st["attempts"], st["samples"]) == \
            (rs.I_t, rs.n_candidates, rs.L, rs.attempts, rs.samples)
    np.testing.assert_array_equal(out.freqs, ref.freqs)
