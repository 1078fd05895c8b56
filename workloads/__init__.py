"""Seeded synthetic inputs for the sparse-FFT hot path.

This module is shared by the CPU oracle, the tests and the benchmark.  It only
draws inputs (planted sparse trigonometric polynomials, frequency sets and
right-hand sides); it contains none of the method's arithmetic (no residues,
collisions, DFTs or selections).

The planted model follows Section 5.1 (random sparse polynomial: frequencies
uniform in the full grid [-N, N]^d, coefficients drawn per coefficient model)
and Section 5.2 (additive complex Gaussian noise at a target SNR in dB, with
sigma^2 = sum |c_k|^2 / 10^(SNR_dB/10)).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "BsplineFunction",
    "bspline_function",
    "paper_bspline",
    "PlantedSignal",
    "planted_signal",
    "noise_sigma",
    "workload",
    "WORKLOADS",
    "batch_signals",
    "diff_problem",
]


@dataclasses.dataclass
class PlantedSignal:
    """A sparse trigonometric polynomial p(x) = sum_k c_k exp(2 pi i k.x).

    freqs:  int32 [s, d], distinct, sorted lexicographically.
    coeffs: complex128 [s].
    sigma:  standard deviation of the complex noise added to every sample
            (eta = sigma/sqrt(2) * (g1 + i g2)); 0 for noiseless sampling.
    """

    d: int
    N: int
    freqs: np.ndarray
    coeffs: np.ndarray
    sigma: float = 0.0

    @property
    def s(self) -> int:
        return int(self.freqs.shape[0])


def _distinct_freqs(rng: np.random.Generator, d: int, N: int, s: int) -> np.ndarray:
    """s distinct frequencies uniform on {-N..N}^d, sorted lexicographically."""
    total = (2 * N + 1) ** d
    if s > total:
        raise ValueError("more frequencies requested than the grid holds")
    got = np.zeros((0, d), dtype=np.int64)
    while got.shape[0] < s:
        need = s - got.shape[0]
        cand = rng.integers(-N, N + 1, size=(max(2 * need, 16), d), dtype=np.int64)
        got = np.unique(np.concatenate([got, cand], axis=0), axis=0)
        if got.shape[0] > s:
            # keep a uniformly random subset of the distinct rows
            keep = rng.choice(got.shape[0], size=s, replace=False)
            got = got[np.sort(keep)]
    order = np.lexsort(got.T[::-1])
    return got[order].astype(np.int32)


def _coefficients(rng: np.random.Generator, s: int, model: str) -> np.ndarray:
    """Coefficient models.

    "u1_10":     amplitude a ~ U[1, 10], phase ~ U[0, 1)
    "logu":      amplitude log-uniform on [1e-2, 10], phase ~ U[0, 1)
    "unimodular": a = 1, phase ~ U[0, 1)                  (Sections 5.1.3, 5.2)
    "box":       Re, Im ~ U[-1, 1), redrawn while |c| < 1e-6 (Section 5.1)
    "posre":     Re ~ U[1e-3, 1), Im ~ U[-1, 1): every real part positive
                 (the coefficients of the deterministic variant, Section 3)
    """
    if model == "box":
        c = rng.uniform(-1, 1, s) + 1j * rng.uniform(-1, 1, s)
        bad = np.abs(c) < 1e-6
        while bad.any():
            c[bad] = rng.uniform(-1, 1, bad.sum()) + 1j * rng.uniform(-1, 1, bad.sum())
            bad = np.abs(c) < 1e-6
        return c.astype(np.complex128)
    if model == "posre":
        return (rng.uniform(1e-3, 1, s) + 1j * rng.uniform(-1, 1, s)).astype(np.complex128)
    if model == "u1_10":
        a = rng.uniform(1.0, 10.0, s)
    elif model == "logu":
        a = np.exp(rng.uniform(math.log(1e-2), math.log(10.0), s))
    elif model == "unimodular":
        a = np.ones(s)
    else:
        raise ValueError(f"unknown coefficient model {model!r}")
    phi = rng.uniform(0.0, 1.0, s)
    return (a * np.exp(2j * np.pi * phi)).astype(np.complex128)


def noise_sigma(coeffs: np.ndarray, snr_db: float | None) -> float:
    """sigma with sigma^2 = sum |c|^2 / 10^(SNR_dB/10); 0 when snr_db is None."""
    if snr_db is None:
        return 0.0
    energy = float(np.sum(np.abs(coeffs) ** 2))
    return math.sqrt(energy / 10.0 ** (snr_db / 10.0))


def planted_signal(d: int, N: int, s: int, seed: int, model: str = "u1_10",
                   snr_db: float | None = None) -> PlantedSignal:
    rng = np.random.default_rng([seed, d, N, s])
    freqs = _distinct_freqs(rng, d, N, s)
    coeffs = _coefficients(rng, s, model)
    return PlantedSignal(d=d, N=N, freqs=freqs, coeffs=coeffs, sigma=noise_sigma(coeffs, snr_db))


# The five benchmark workloads (parameters of the sparse FFT run).  "theta" is
# relative (threshold = theta * max |p~| of the pass) unless theta_mode="abs".
WORKLOADS = {
    "tiny_d3": dict(d=3, N=16, s=20, model="u1_10", snr_db=None, r=2, theta=1e-12,
                    theta_mode="rel", b=10),
    "plain_d10": dict(d=10, N=32, s=1000, model="u1_10", snr_db=40.0, r=5, theta=1e-12,
                      theta_mode="rel", b=10),
    "large_d25": dict(d=25, N=32, s=10000, model="logu", snr_db=20.0, r=10, theta=1e-12,
                      theta_mode="rel", b=10),
}


def workload(name: str, seed: int) -> tuple[PlantedSignal, dict]:
    """Planted signal plus the sparse-FFT parameters of a named workload."""
    w = dict(WORKLOADS[name])
    sig = planted_signal(w.pop("d"), w.pop("N"), w.pop("s"), seed, w.pop("model"),
                         w.pop("snr_db"))
    w["s"] = sig.s
    w["s_local"] = sig.s
    return sig, w


def batch_signals(count: int, seed: int, d_range=(5, 12), N_choices=(16, 32, 64),
                  s_range=(100, 2000)) -> list[tuple[PlantedSignal, dict]]:
    """Many independent noiseless signals of uneven d, N and s (log-uniform s)."""
    rng = np.random.default_rng([seed, 0xBA7C4])
    out = []
    for i in range(count):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        N = int(rng.choice(N_choices))
        s = int(math.floor(math.exp(rng.uniform(math.log(s_range[0]), math.log(s_range[1])))))
        sig = planted_signal(d, N, s, seed * 100003 + i, "u1_10", None)
        out.append((sig, dict(s=s, s_local=s, r=3, theta=1e-12, theta_mode="rel", b=10)))
    return out


def diff_problem(n_freq: int, d: int, N: int, nrhs: int, seed: int):
    """A fixed frequency set I (distinct, uniform in [-N,N]^d, lexicographic)
    plus complex Gaussian right-hand sides generator state."""
    rng = np.random.default_rng([seed, 0xD1FF])
    I = _distinct_freqs(rng, d, N, n_freq)
    return I, rng


def complex_normal(rng: np.random.Generator, shape) -> np.ndarray:
    return ((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)).astype(
        np.complex128)


@dataclasses.dataclass
class BsplineFunction:
    """The description (no evaluation) of a Section 5.3 test function
    f(x) = sum_g prod_{t in groups[g]} N_{orders[g]}(x_t): disjoint 0-based
    dimension groups and one B-spline order per group; N is the search box
    [-N, N]^d of the sparse FFT run; noiseless."""

    d: int
    N: int
    groups: list
    orders: list
    sigma: float = 0.0


def bspline_function(d: int, N: int, groups, orders) -> BsplineFunction:
    groups = [sorted(int(t) for t in g) for g in groups]
    flat = [t for g in groups for t in g]
    if len(set(flat)) != len(flat) or any(t < 0 or t >= d for t in flat) or len(groups) != len(orders):
        raise ValueError("groups must be disjoint subsets of range(d), one order per group")
    return BsplineFunction(d=d, N=N, groups=groups, orders=[int(m) for m in orders])


def paper_bspline(N: int) -> BsplineFunction:
    """Section 5.3: f(x) = N_2(x1) N_2(x3) N_2(x8) + N_4(x2) N_4(x5) N_4(x6) N_4(x10)
    + N_6(x4) N_6(x7) N_6(x9) on T^10."""
    return bspline_function(10, N, [[0, 2, 7], [1, 4, 5, 9], [3, 6, 8]], [2, 4, 6])

