"""The per-run cache of Bluestein filter spectra.

Increments with as many candidates take the same lattice sizes (the smallest
admissible primes above lambda = 2 (|J| - 1)), so a run reuses their filter
spectra.  A reused spectrum is the same computation as a fresh one, so the
run's output must not change by a single bit with the cache turned off."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()


def _run(name, fft, cache):
    sig, p = W.workload(name, 1)
    old = os.environ.get("MR1L_FILTER_CACHE")
    os.environ["MR1L_FILTER_CACHE"] = "1" if cache else "0"
    try:
        return P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=1, b=p["b"],
                              freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma, batch_reps=True, fft=fft)
    finally:
        if old is None:
            del os.environ["MR1L_FILTER_CACHE"]
        else:
            os.environ["MR1L_FILTER_CACHE"] = old


@pytest.mark.parametrize("fft", ["f64", "df"])
def test_cache_changes_no_bit(fft):
    a = _run("plain_d10", fft, True)
    b = _run("plain_d10", fft, False)
    np.testing.assert_array_equal(a.freqs, b.freqs)
    np.testing.assert_array_equal(a.coeffs.view(np.float64), b.coeffs.view(np.float64))
    assert a.samples == b.samples
    # the run does repeat lattice sizes: increments t = 5..10 all have 65,000 candidates
    n_cand = [st["n_cand"] for st in a.steps]
    assert n_cand.count(65000) >= 2
