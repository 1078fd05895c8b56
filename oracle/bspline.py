"""The tensor-product B-spline test function of Section 5.3 (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 5.3 approximates f(x) = sum_g prod_{t in S_g} N_{m_g}(x_t) (disjoint
dimension groups S_g, B-spline orders m_g) whose univariate factor is given
by its Fourier series

    N_m(x) = C_m sum_k sinc(pi k / m)^m (-1)^k e^{2 pi i k x},

with C_m > 0 such that ||N_m||_{L2(T)} = 1.  The oracle evaluates it in the
spatial domain: with the cardinal B-spline B_m of order m (degree m - 1,
support [0, m], integer knots), the 1-periodic function m B_m(m x) has
Fourier coefficients sinc(pi k / m)^m (-1)^k (the centred B-spline has
transform sinc^m; the shift by half a period gives (-1)^k), so

    N_m(x) = C_m m B_m(m (x mod 1)),

with B_m evaluated by the Cox-de Boor recurrence (the truncated-power closed
form is kept beside it as a cross-check).  C_m is taken from its definition,
C_m^-2 = sum_k sinc(pi k / m)^{2m}, summed with a tail bound;
tests/test_oracle_bspline.py pins all of it.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


def cardinal_bspline(m: int, u: np.ndarray) -> np.ndarray:
    """B_m(u) by the Cox-de Boor recurrence B_1 = 1 on [0, 1),
    B_k(v) = (v B_{k-1}(v) + (k - v) B_{k-1}(v - 1)) / (k - 1), which only
    combines non-negative terms (0 outside [0, m))."""
    u = np.asarray(u, dtype=np.float64)
    vals = [((u - s >= 0) & (u - s < 1)).astype(np.float64) for s in range(m)]   # B_1(u - s)
    for k in range(2, m + 1):
        vals = [((u - s) * vals[s] + (k - (u - s)) * vals[s + 1]) / (k - 1) for s in range(m - k + 1)]
    return vals[0]


def cardinal_bspline_truncated_power(m: int, u: np.ndarray) -> np.ndarray:
    """B_m(u) = 1/(m-1)! sum_{j=0}^{m} (-1)^j binom(m, j) (u - j)_+^{m-1}, the
    closed form (cancellation costs it some digits away from the knots)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    for j in range(m + 1):
        out += (-1) ** j * math.comb(m, j) * np.where(u > j, u - j, 0.0) ** (m - 1)
    out /= math.factorial(m - 1)
    return np.where((u >= 0) & (u < m), out, 0.0)


def fourier_factor(m: int, k: np.ndarray) -> np.ndarray:
    """sinc(pi k / m)^m (-1)^k (sinc(x) = sin(x) / x, sinc(0) = 1)."""
    k = np.asarray(k, dtype=np.float64)
    x = np.pi * k / m
    s = np.where(k == 0, 1.0, np.sin(x) / np.where(k == 0, 1.0, x))
    return s ** m * np.where(np.mod(k, 2) == 0, 1.0, -1.0)


def norm_constant(m: int, terms: int = 200000) -> float:
    """C_m = (sum_k sinc(pi k/m)^{2m})^{-1/2}: the series summed to |k| <=
    terms, plus the bound of its tail sum_{|k| > terms} (m / (pi k))^{2m}."""
    k = np.arange(1, terms + 1, dtype=np.float64)
    s = 1.0 + 2.0 * float(np.sum(fourier_factor(m, k) ** 2))
    tail = 2.0 * (m / math.pi) ** (2 * m) / ((2 * m - 1) * terms ** (2 * m - 1))
    return 1.0 / math.sqrt(s + tail)


@dataclasses.dataclass
class BsplineSignal:
    """f(x) = sum_g prod_{t in groups[g]} N_{orders[g]}(x_t) on T^d, sampled by
    Algorithm 3 in the search box [-N, N]^d (noiseless: sigma = 0)."""

    d: int
    N: int
    groups: list            # list of lists of 0-based dimensions (disjoint)
    orders: list            # B-spline order per group
    sigma: float = 0.0

    def __post_init__(self):
        self.C = [norm_constant(m) for m in self.orders]

    def factor(self, g: int, x: np.ndarray) -> np.ndarray:
        m = self.orders[g]
        return self.C[g] * m * cardinal_bspline(m, m * np.mod(x, 1.0))

    def value(self, X: np.ndarray) -> np.ndarray:
        """f at the rows of X [n, d] (complex, imaginary part 0)."""
        X = np.asarray(X, dtype=np.float64)
        f = np.zeros(X.shape[0])
        for g, dims in enumerate(self.groups):
            prod = np.ones(X.shape[0])
            for t in dims:
                prod *= self.factor(g, X[:, t])
            f += prod
        return f.astype(np.complex128)

    def coeff(self, K: np.ndarray) -> np.ndarray:
        """The exact Fourier coefficients f^_k at the integer rows of K [n, d]:
        the g-th term contributes prod_{t in S_g} C_m sinc^m (-1)^k_t when
        k_t = 0 off S_g."""
        K = np.asarray(K, dtype=np.int64)
        out = np.zeros(K.shape[0])
        for g, dims in enumerate(self.groups):
            off = [t for t in range(self.d) if t not in dims]
            val = np.all(K[:, off] == 0, axis=1).astype(np.float64)
            for t in dims:
                val = val * self.C[g] * fourier_factor(self.orders[g], K[:, t])
            out += val
        return out.astype(np.complex128)

    def norm2(self) -> float:
        """||f||^2: each term has norm 1 (a product of unit-norm factors in
        disjoint variables); two terms g != h in disjoint variables have inner
        product (mean of term g) (mean of term h), the mean of a factor being
        its zeroth coefficient C_m."""
        means = [self.C[g] ** len(dims) for g, dims in enumerate(self.groups)]
        return float(len(self.groups) + sum(means[a] * means[b] for a in range(len(means))
                                             for b in range(len(means)) if a != b))

    def rel_l2_error(self, freqs: np.ndarray, coeffs: np.ndarray) -> float:
        """||f - S~_I f|| / ||f|| = sqrt(||f||^2 - sum_I |f^_k|^2 + sum_I |p~_k - f^_k|^2) / ||f||
        (Section 5.3), for the detected set I = freqs with coefficients coeffs."""
        fk = self.coeff(freqs) if len(freqs) else np.zeros(0)
        n2 = self.norm2()
        e2 = n2 - float(np.sum(np.abs(fk) ** 2)) + float(np.sum(np.abs(coeffs - fk) ** 2))
        return math.sqrt(max(e2, 0.0) / n2)


def signal(desc) -> BsplineSignal:
    """The oracle's evaluator for a workload description (workloads.BsplineFunction)."""
    return BsplineSignal(desc.d, desc.N, list(desc.groups), list(desc.orders), desc.sigma)

