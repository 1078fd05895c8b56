"""Pins for the oracle's lattice algorithms (Section 2.1, Eq. 2.2, Algorithms
1 and 2, the Section 4.1 aliasing identity and the adjoint)."""

import math
from fractions import Fraction

import numpy as np
import pytest
import sympy

from oracle import lattice, philox


def _rand_set(rng, n, t, N):
    J = np.unique(rng.integers(-N, N + 1, size=(3 * n, t)), axis=0)
    rng.shuffle(J)
    J = J[:n]
    return J[np.lexsort(J.T[::-1])]


def test_unique_mask_matches_pairwise_definition():
    """Reconstruction property of Section 2.1 checked pair by pair."""
    rng = np.random.default_rng(0)
    for trial in range(40):
        t = int(rng.integers(1, 5))
        J = _rand_set(rng, int(rng.integers(2, 40)), t, 6)
        M = int(sympy.prime(int(rng.integers(3, 30))))
        z = rng.integers(1, M, size=t)
        np.testing.assert_array_equal(lattice.unique_mask(J, z, M),
                                      lattice.unique_mask_bruteforce(J, z, M))


def test_lmax_matches_section_3_2_form():
    """Algorithm 1 with c = 2, gamma = 1/2 gives the lattice count that the
    complexity discussion of Section 3.2 writes as ceil(2 ln n + 2 ln 2)."""
    for n in [1, 2, 3, 7, 20, 400, 4225, 65000, 325000, 10**6, 6_500_000]:
        Lmax, lam = lattice.lmax_lambda(n)
        assert Lmax == math.ceil(2 * math.log(n) + 2 * math.log(2))
        assert lam == 2 * (n - 1)


def test_prime_set_against_library():
    """Eq. 2.2: the Lmax smallest primes above lambda (checked with sympy's
    primality routines) when injectivity is automatic (p > expansion)."""
    rng = np.random.default_rng(1)
    J = _rand_set(rng, 500, 3, 32)
    Lmax, lam = lattice.lmax_lambda(J.shape[0])
    ps = lattice.prime_set(J, lam, Lmax)
    want = []
    p = int(lam)
    while len(want) < Lmax:
        p = sympy.nextprime(p)
        want.append(p)
    assert ps == want


def test_prime_set_skips_non_injective():
    """J = {0, 5} in Z^1: lambda = 2, Lmax = 3; 5 maps both to 0 and is not in
    P^J, so the set is {3, 7, 11}."""
    J = np.array([[0], [5]])
    Lmax, lam = lattice.lmax_lambda(2)
    assert (Lmax, lam) == (3, 2.0)
    assert lattice.prime_set(J, lam, Lmax) == [3, 7, 11]


def test_node_count_bruteforce():
    """|Lambda| = 1 - L + sum M_l for distinct primes and z in [1, M-1]^t,
    counted as distinct exact rational points."""
    rng = np.random.default_rng(2)
    J = _rand_set(rng, 12, 2, 5)
    ml = lattice.construct(J, seed=3, t=2, attempt=0)
    pts = set()
    for M, z in zip(ml.M, ml.z):
        for j in range(M):
            pts.add(tuple(Fraction(int(j * zz % M), M) for zz in z))
    assert len(pts) == ml.nodes()


def test_construct_covers_and_satisfies_condition_2_1():
    rng = np.random.default_rng(3)
    for t in (1, 2, 3):
        J = _rand_set(rng, 60, t, 8)
        ml = lattice.search(J, seed=11, t=t, b=10)
        assert ml.covered
        assert ml.L <= lattice.lmax_lambda(J.shape[0])[0]
        union = np.zeros(J.shape[0], dtype=bool)
        for M, z, IL in zip(ml.M, ml.z, ml.unique):
            assert sympy.isprime(M) and M > 2 * (J.shape[0] - 1)
            assert np.all(z >= 1) and np.all(z <= M - 1)
            np.testing.assert_array_equal(IL, lattice.unique_mask_bruteforce(J, z, M))
            union |= IL
        assert union.all()
        assert len(set(ml.M)) == ml.L


def test_construct_uses_philox_vectors():
    J = np.array([[1, 2], [3, -4], [0, 0], [5, 5]])
    ml = lattice.construct(J, seed=42, t=2, attempt=1)
    for l, (M, z) in enumerate(zip(ml.M, ml.z)):
        np.testing.assert_array_equal(z, philox.zvec(42, 2, l, 1, M))


def test_direct_dft_equals_library_fft():
    """t = 1, z = 1, J = all residues: Algorithm 2 with L = 1 is the plain
    length-M DFT with factor 1/M (textbook special case)."""
    rng = np.random.default_rng(4)
    for M in (2, 3, 5, 17, 101):
        y = rng.standard_normal(M) + 1j * rng.standard_normal(M)
        got = lattice.lattice_dft_direct(y, M, np.arange(M))
        np.testing.assert_allclose(got, np.fft.fft(y) / M, rtol=0, atol=1e-14)


def _planted(rng, s, t_total, N):
    freqs = _rand_set(rng, s, t_total, N)
    coeffs = rng.standard_normal(freqs.shape[0]) + 1j * rng.standard_normal(freqs.shape[0])
    return freqs, coeffs


@pytest.mark.parametrize("dft", ["direct", "fft"])
def test_reconstruct_evaluate_identity(dft):
    """Algorithm 2 is a left inverse of the lattice evaluation on a covered J."""
    rng = np.random.default_rng(5)
    J = _rand_set(rng, 80, 3, 7)
    ml = lattice.search(J, seed=5, t=3)
    assert ml.covered
    c = rng.standard_normal(J.shape[0]) + 1j * rng.standard_normal(J.shape[0])
    ys = lattice.evaluate(J, ml, c, "eval", dft)
    got, counter = lattice.reconstruct(J, ml, ys, dft)
    assert np.all(counter >= 1)
    np.testing.assert_allclose(got, c, rtol=0, atol=1e-12)


def test_evaluate_is_polynomial_at_nodes():
    """EVAL mode equals p(x) = sum_k c_k e^{2 pi i k.x} at x = j z / M mod 1."""
    rng = np.random.default_rng(6)
    J = _rand_set(rng, 15, 2, 4)
    ml = lattice.search(J, seed=6, t=2)
    c = rng.standard_normal(J.shape[0]) + 1j * rng.standard_normal(J.shape[0])
    ys = lattice.evaluate(J, ml, c, "eval", "fft")
    for M, z, y in zip(ml.M, ml.z, ys):
        for j in range(M):
            x = np.array([(j * int(zz)) % M / M for zz in z])
            want = np.sum(c * np.exp(2j * np.pi * (J @ x)))
            assert abs(y[j] - want) < 1e-12


def test_aliasing_identity_projected_coefficients():
    """Section 4.1: with a reconstructing multiple lattice for J at step t,
    Algorithm 2 applied to samples of p returns, for every k in J, the
    projected coefficient sum_{h: h_(1..t) = k} c_h e^{2 pi i h_(>t).x'}."""
    from oracle import sfft
    import workloads as W

    rng = np.random.default_rng(7)
    sig = W.planted_signal(4, 3, 30, seed=7, model="u1_10")
    t = 2
    heads = np.unique(sig.freqs[:, :t].astype(np.int64), axis=0)
    extra = _rand_set(rng, 20, t, 3)
    J = np.unique(np.concatenate([heads, extra]), axis=0)
    ml = lattice.search(J, seed=8, t=t)
    assert ml.covered
    x = rng.uniform(0, 1, 4)
    for dft in ("direct", "fft"):
        ys = sfft.sample_lattice(sig, t, ml, x, dft)
        got, _ = lattice.reconstruct(J, ml, ys, dft)
        want = np.zeros(J.shape[0], dtype=complex)
        for h, ch in zip(sig.freqs.astype(np.int64), sig.coeffs):
            idx = np.nonzero(np.all(J == h[:t], axis=1))[0]
            want[idx] += ch * np.exp(2j * np.pi * np.dot(h[t:], x[t:]))
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_adjoint_identity_and_dense_matrix():
    """<R y, c> = <y, R^H c>, and R written entry by entry matches Algorithm 2."""
    rng = np.random.default_rng(9)
    J = _rand_set(rng, 40, 2, 6)
    ml = lattice.search(J, seed=9, t=2)
    R = lattice.dense_reconstruct_matrix(J, ml)
    y = rng.standard_normal(R.shape[1]) + 1j * rng.standard_normal(R.shape[1])
    c = rng.standard_normal(R.shape[0]) + 1j * rng.standard_normal(R.shape[0])
    ys = np.split(y, np.cumsum(ml.M)[:-1])
    Ry, _ = lattice.reconstruct(J, ml, ys, "direct")
    np.testing.assert_allclose(Ry, R @ y, rtol=0, atol=1e-13)
    RHc = np.concatenate(lattice.evaluate(J, ml, c, "adjoint", "direct"))
    np.testing.assert_allclose(RHc, R.conj().T @ c, rtol=0, atol=1e-13)
    lhs = np.vdot(c, Ry)
    rhs = np.vdot(RHc, y)
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_uncovered_candidate_gets_zero():
    """A candidate that no lattice covers gets p~ = 0 and counter 0."""
    J = np.array([[0], [3], [6]])
    ml = lattice.MultiLattice(M=[3], z=[np.array([1])], unique=[lattice.unique_mask(J, [1], 3)],
                              covered=False, attempts=1)
    assert not ml.unique[0].any()
    got, counter = lattice.reconstruct(J, ml, [np.ones(3, dtype=complex)], "fft")
    assert np.all(counter == 0) and np.all(got == 0)


def _redraw_property_holds(J, ml) -> bool:
    """The redraw rule (the remark after Algorithm 1), checked pair by pair:
    every kept lattice, collision-free set recomputed by the pairwise
    definition, holds a frequency that no earlier lattice covers."""
    covered = np.zeros(J.shape[0], dtype=bool)
    for M, z, IL in zip(ml.M, ml.z, ml.unique):
        brute = lattice.unique_mask_bruteforce(J, z, M)
        if not np.array_equal(brute, IL) or not (brute & ~covered).any():
            return False
        covered |= brute
    return True


def test_redraw_rule_every_lattice_adds_a_frequency():
    rng = np.random.default_rng(31)
    redraws = 0
    for trial in range(40):
        t = int(rng.integers(1, 4))
        J = _rand_set(rng, int(rng.integers(2, 60)), t, 7)
        ml = lattice.construct(J, seed=trial, t=t, attempt=0, redraw=True)
        assert _redraw_property_holds(J, ml)
        # condition (2.1): the union is J whenever the search reports coverage
        if ml.covered:
            assert np.logical_or.reduce([lattice.unique_mask_bruteforce(J, z, M)
                                         for M, z in zip(ml.M, ml.z)]).all()
        plain = lattice.construct(J, seed=trial, t=t, attempt=0)
        redraws += int(not _redraw_property_holds(J, plain))
    # the rule changes something on these sizes (plain searches keep idle lattices)
    assert redraws > 0


def test_redraw_rule_agrees_with_plain_search_until_the_first_idle_lattice():
    """Both searches draw z_L from the same counters; they part only where
    the plain search keeps a lattice that adds nothing."""
    rng = np.random.default_rng(32)
    for trial in range(30):
        J = _rand_set(rng, int(rng.integers(5, 80)), 2, 9)
        a = lattice.construct(J, seed=100 + trial, t=2, attempt=0)
        b = lattice.construct(J, seed=100 + trial, t=2, attempt=0, redraw=True)
        covered = np.zeros(J.shape[0], dtype=bool)
        for L in range(min(a.L, b.L)):
            assert a.M[L] == b.M[L]
            if not (a.unique[L] & ~covered).any():
                break
            np.testing.assert_array_equal(a.z[L], b.z[L])
            covered |= a.unique[L]


def test_redraw_rule_needs_fewer_lattices():
    """Over many searches the rule never needs more lattices in total and
    saves some (the paper reports 2-10 % fewer samples with it, Section 5.1)."""
    rng = np.random.default_rng(33)
    La = Lb = 0
    for trial in range(60):
        J = _rand_set(rng, int(rng.integers(20, 400)), 3, 12)
        La += lattice.search(J, seed=trial, t=3).L
        Lb += lattice.search(J, seed=trial, t=3, redraw=True).L
    assert Lb < La


def test_redraw_property_catches_a_wrong_rule():
    """Planted mistake: a rule that redraws while the lattice does add a
    frequency (the condition inverted) violates the pinned property."""
    rng = np.random.default_rng(34)
    caught = False
    for trial in range(20):
        J = _rand_set(rng, 40, 2, 7)
        n = J.shape[0]
        Lmax, lam = lattice.lmax_lambda(n)
        primes = lattice.prime_set(J, lam, Lmax)
        covered = np.zeros(n, dtype=bool)
        Ms, zs, us = [], [], []
        for L in range(1, Lmax + 1):
            r = 0
            while True:
                z = philox.zvec(trial, 2, L - 1, 0, primes[L - 1], redraw=r)
                IL = lattice.unique_mask(J, z, primes[L - 1])
                if not (IL & ~covered).any() or r == 3:   # inverted condition
                    break
                r += 1
            covered |= IL
            Ms.append(primes[L - 1]), zs.append(z), us.append(IL)
            if covered.all():
                break
        bad = lattice.MultiLattice(Ms, zs, us, bool(covered.all()), 1)
        caught |= not _redraw_property_holds(J, bad)
    assert caught
