"""Pins for the oracle's Section 5.3 test function (tensor-product B-splines)."""

import math

import numpy as np
import pytest

import workloads as W
from oracle import bspline as B
from oracle import sfft


@pytest.mark.parametrize("m", [2, 3, 4, 6])
def test_norm_constant_two_ways(m):
    """C_m from its Fourier-series definition equals 1 / sqrt(m B_2m(m)):
    the autocorrelation of the cardinal B-spline is B_2m, so
    ||m B_m(m .)||^2 = m B_2m(m); C_2 = sqrt(3)/2 (the hat function)."""
    closed = 1.0 / math.sqrt(m * float(B.cardinal_bspline_truncated_power(2 * m, np.array([float(m)]))[0]))
    assert abs(B.norm_constant(m) - closed) < 1e-14
    if m == 2:
        assert abs(B.norm_constant(2) - math.sqrt(3) / 2) < 1e-15


@pytest.mark.parametrize("m", [2, 3, 4, 6, 8])
def test_recurrence_matches_closed_form(m):
    """Cox-de Boor against the truncated-power formula (whose cancellation
    allows a few times 1e-13 at order 8), and B_m(u) = B_m(m - u)."""
    u = np.random.default_rng(m).uniform(-0.5, m + 0.5, 4000)
    a, b = B.cardinal_bspline(m, u), B.cardinal_bspline_truncated_power(m, u)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    inside = (u > 0) & (u < m)
    np.testing.assert_allclose(a[inside], B.cardinal_bspline(m, m - u[inside]), rtol=0, atol=1e-15)


@pytest.mark.parametrize("m", [2, 3, 4, 6])
def test_partition_of_unity(m):
    u = np.linspace(0, 1, 101, endpoint=False)
    tot = sum(B.cardinal_bspline(m, u + n) for n in range(m))
    np.testing.assert_allclose(tot, 1.0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("m", [2, 4, 6])
def test_fourier_coefficients_of_the_factor(m):
    """The DFT of N_m on 2^16 points reproduces C_m sinc(pi k/m)^m (-1)^k up
    to aliasing (sum over the other periods, < 1e-9 for m = 2)."""
    n = 1 << 16
    sig = B.BsplineSignal(1, 1, [[0]], [m])
    x = np.arange(n) / n
    c = np.fft.fft(sig.factor(0, x)) / n
    k = np.arange(-40, 41)
    want = sig.C[0] * B.fourier_factor(m, k)
    np.testing.assert_allclose(c[np.mod(k, n)].real, want, rtol=0, atol=2e-9)
    assert np.max(np.abs(c[np.mod(k, n)].imag)) < 1e-12


@pytest.mark.parametrize("m", [2, 4, 6])
def test_unit_norm_by_gauss_legendre(m):
    """||N_m||^2 = 1: Gauss-Legendre with m points on each knot interval of
    m x is exact for the piecewise polynomial N_m^2 of degree 2m - 2."""
    sig = B.BsplineSignal(1, 1, [[0]], [m])
    g, w = np.polynomial.legendre.leggauss(m)
    tot = 0.0
    for q in range(m):
        a, b = q / m, (q + 1) / m
        xs = (a + b) / 2 + (b - a) / 2 * g
        tot += (b - a) / 2 * float(np.sum(w * sig.factor(0, xs) ** 2))
    assert abs(tot - 1.0) < 1e-13


def test_multivariate_coefficients_norm_and_error():
    """A 3-variate instance f = N_2(x1) N_2(x3) + N_4(x2): the exact
    coefficient function against the 3-D DFT of f on a 64^3 grid, and the L2
    error formula against Parseval over that grid's frequencies."""
    sig = B.BsplineSignal(3, 8, [[0, 2], [1]], [2, 4])
    n = 64
    ax = np.arange(n) / n
    X = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    F = np.fft.fftn(sig.value(X).real.reshape(n, n, n)) / n ** 3
    K = np.array([[0, 0, 0], [1, 0, 0], [0, 3, 0], [2, 0, -1], [0, -2, 0], [1, 1, 0], [3, 0, 5]])
    got = F[tuple(np.mod(K, n).T)]
    # aliasing of the hat-function factors on 64 points: below 3e-4 of C_2^2
    np.testing.assert_allclose(got, sig.coeff(K), rtol=0, atol=3e-4)
    assert abs(sig.coeff(np.array([[1, 1, 0]]))[0]) == 0.0
    # Parseval: the grid mean of f^2 is ||f||^2 up to the grid's aliasing
    assert abs(np.mean(sig.value(X).real ** 2) - sig.norm2()) < 1e-3
    # error of the empty approximation is 1; of the exact coefficients on I,
    # sqrt(1 - sum_I |f^_k|^2 / ||f||^2)
    assert abs(sig.rel_l2_error(np.zeros((0, 3), dtype=np.int64), np.zeros(0)) - 1.0) < 1e-15
    e = sig.rel_l2_error(K, sig.coeff(K))
    want = math.sqrt(1 - float(np.sum(np.abs(sig.coeff(K)) ** 2)) / sig.norm2())
    assert abs(e - want) < 1e-14


def test_dimension_incremental_run_on_the_function():
    """Algorithm 3 on a 4-variate instance (N = 8, s = 20, 60, 150,
    s_local = 2 s, r = 3): the coefficients it returns are the exact ones up to the aliasing
    of the coefficients it does not capture (|f^_k| ~ (4 / (9 pi))^4 ~ 4e-4
    just outside the box for the order-4 factor), and the L2 error falls as s
    grows."""
    sig = B.signal(W.bspline_function(4, 8, [[0, 2], [1, 3]], [4, 6]))
    errs = []
    for s in (20, 60, 150):
        res = sfft.sfft(sig, s, 2 * s, 3, 10, 1e-12, "abs", seed=5)
        fk = sig.coeff(res.freqs)
        assert np.max(np.abs(res.coeffs - fk)) < 1e-3
        errs.append(sig.rel_l2_error(res.freqs, res.coeffs))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 1e-3
