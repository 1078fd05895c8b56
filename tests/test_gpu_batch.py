"""Many independent signals of uneven d, N and s through sfft_dimincr_batch."""

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


def _problem(sig, prm, seed):
    return dict(d=sig.d, N=sig.N, s=prm["s"], s_local=prm["s_local"], r=prm["r"], b=prm["b"],
                theta=prm["theta"], theta_mode=prm["theta_mode"], seed=seed, freqs=sig.freqs,
                coeffs=sig.coeffs, sigma=sig.sigma)


def _assert_equal(out, ref):
    np.testing.assert_array_equal(out.freqs, ref.freqs)
    assert out.samples == ref.samples
    if ref.coeffs.size:
        assert np.max(np.abs(out.coeffs - ref.coeffs) / np.abs(ref.coeffs)) < 1e-10


def test_batch_small_parity():
    """Eight ragged small problems, each against the oracle."""
    rng = np.random.default_rng(11)
    probs, refs = [], []
    for i in range(8):
        d, N, s = int(rng.integers(2, 6)), int(rng.integers(4, 17)), int(rng.integers(5, 60))
        sig = W.planted_signal(d, N, s, seed=100 + i, model="u1_10", snr_db=None if i % 2 else 30.0)
        prm = dict(s=s, s_local=s, r=2, b=10, theta=1e-12, theta_mode="rel")
        probs.append(_problem(sig, prm, 100 + i))
        refs.append(sfft.sfft(sig, s, s, 2, 10, 1e-12, "rel", seed=100 + i))
    outs = P.sfft_dimincr_batch(probs, concurrency=4)
    for out, ref in zip(outs, refs):
        _assert_equal(out, ref)
