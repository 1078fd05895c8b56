"""Every Bluestein length the transforms use, against the oracle.

For each length P = 2^k or 3 * 2^k up to 2^21 that some prime lattice size
reaches, the largest such prime M gets one lattice.  Up to M < 2^15 every
residue is a candidate (I = 0..M-1, z = 1), so the reconstruction is the
whole length-M DFT (Algorithm 2 with L = 1); above (frequencies are limited
to |k_j| < 2^15) the 32767 candidates |k| < 2^14 with z = 7919 read it at as
many residues spread over [0, M).  The adjoint evaluation is the whole
inverse DFT in both cases.  Together the cases
run every sub-FFT length of the one-CTA and 4-step paths, and so every radix
(8, 4, 2, 3) at every stage stride, with and without turned first-level
twiddles, in both arithmetics.  Bar: 1e-10 normwise relative error."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
from oracle import lattice

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()


def _bluestein_length(n: int) -> int:
    """Smallest 2^k or 3 * 2^k >= n (2^k >= 4)."""
    p2 = 4
    while p2 < n:
        p2 *= 2
    p3 = 3
    while p3 < n:
        p3 *= 2
    return min(p2, p3)


def _cases(max_p: int = 1 << 21):
    out = []
    lengths = sorted({1 << k for k in range(2, 22)} | {3 << k for k in range(0, 20)})
    for p in lengths:
        if p > max_p:
            break
        m = (p + 1) // 2
        while m >= 2 and not (lattice.is_prime(m) and _bluestein_length(2 * m - 1) == p):
            m -= 1
        if m >= 2 and _bluestein_length(2 * m - 1) == p:
            out.append((p, m))
    return out


CASES = _cases()


def test_every_length_is_reached():
    """All lengths but 4 (2 M - 1 = 3 takes length 3) have a prime."""
    ps = [p for p, _ in CASES]
    assert 4 not in ps and 3 in ps and (1 << 21) in ps and (3 << 19) in ps
    assert len(ps) == 38


def _normwise(got, want):
    return np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300)


@pytest.mark.parametrize("fft", ["f64", "df"])
@pytest.mark.parametrize("p,m", CASES, ids=[f"P{p}" for p, _ in CASES])
def test_full_dft_at_every_length(p, m, fft):
    if m < 1 << 15:
        I, z = np.arange(m, dtype=np.int64).reshape(-1, 1), 1
    else:
        I, z = np.arange(-(1 << 14) + 1, 1 << 14, dtype=np.int64).reshape(-1, 1), 7919
    pl = P.plan(I, [m], [[z]], strict=True, fft=fft)
    ml = lattice.MultiLattice([m], [np.array([z])], [np.ones(I.shape[0], dtype=bool)], True, 1)
    rng = np.random.default_rng(p)
    y = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    got = pl.reconstruct(torch.from_numpy(y).cuda()).cpu().numpy().reshape(-1)
    tier = "direct" if m <= 4099 else "fft"
    want, _ = lattice.reconstruct(I, ml, [y], tier)
    assert _normwise(got, want) < RTOL
    c = rng.standard_normal(I.shape[0]) + 1j * rng.standard_normal(I.shape[0])
    gota = pl.evaluate(torch.from_numpy(c).cuda(), P.MR1L_ADJOINT).cpu().numpy().reshape(-1)
    wanta = np.concatenate(lattice.evaluate(I, ml, c, "adjoint", tier))
    assert _normwise(gota, wanta) < RTOL
