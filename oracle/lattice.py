"""Rank-1 and multiple rank-1 lattices (oracle side).

Sections 2.1 and 4.1 of Kaemmerer, Potts, Volkmer.  Frequencies are rows of
an int64 array J [n, t]; a lattice is (M, z) with M prime and z in Z^t; its
nodes are x_j = j z / M mod 1, j = 0..M-1.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import philox


# ----------------------------------------------------------------------------
# Section 2.1: residues and the reconstruction property
# ----------------------------------------------------------------------------

def residues(J: np.ndarray, z: np.ndarray, M: int) -> np.ndarray:
    """k . z mod M for every row k of J, canonical in [0, M) (exact int64:
    |k_j| <= 2^7, z_j < 2^31, t <= 64 keeps |k . z| < 2^44)."""
    J = np.asarray(J, dtype=np.int64)
    z = np.asarray(z, dtype=np.int64)
    return np.mod(J @ z, np.int64(M))


def unique_mask(J: np.ndarray, z: np.ndarray, M: int) -> np.ndarray:
    """I_l of Algorithm 1 / Algorithm 2: the k in J whose residue k.z mod M no
    other h in J shares (condition (2.1) for a single lattice)."""
    r = residues(J, z, M)
    counts = np.bincount(r, minlength=M)
    return counts[r] == 1


def unique_mask_bruteforce(J: np.ndarray, z: np.ndarray, M: int) -> np.ndarray:
    """The same set by the definition: pairwise comparison of k.z and h.z mod M
    (Section 2.1 reconstruction property).  O(n^2); for tiny sets."""
    J = [tuple(int(v) for v in row) for row in np.asarray(J)]
    zz = [int(v) for v in z]
    res = [sum(a * b for a, b in zip(k, zz)) % M for k in J]
    out = np.ones(len(J), dtype=bool)
    for a in range(len(J)):
        for b in range(len(J)):
            if a != b and res[a] == res[b]:
                out[a] = False
                break
    return out


# ----------------------------------------------------------------------------
# Eq. (2.2): the prime set P^I_{lambda, Lmax}
# ----------------------------------------------------------------------------

def is_prime(p: int) -> bool:
    if p < 2:
        return False
    if p % 2 == 0:
        return p == 2
    f = 3
    while f * f <= p:
        if p % f == 0:
            return False
        f += 2
    return True


def injective_mod(J: np.ndarray, p: int) -> bool:
    """Membership test of P^I: the componentwise map k -> k mod p is injective
    on J (Section 2.1, definition of P^I)."""
    J = np.asarray(J, dtype=np.int64)
    if J.shape[0] <= 1:
        return True
    red = np.mod(J, p)
    return np.unique(red, axis=0).shape[0] == J.shape[0]


def prime_set(J: np.ndarray, lam: float, Lmax: int) -> list[int]:
    """The Lmax smallest primes p > lam with p in P^J (Eq. 2.2)."""
    out: list[int] = []
    p = int(math.floor(lam)) + 1
    while len(out) < Lmax:
        if is_prime(p) and injective_mod(J, p):
            out.append(p)
        p += 1
    return out


def lmax_lambda(n: int, c: float = 2.0, gamma: float = 0.5) -> tuple[int, float]:
    """Algorithm 1, first two steps: Lmax = ceil(c^2/(c-1)^2 (ln n - ln gamma)/2)
    and lambda = c (n - 1)."""
    Lmax = math.ceil(c * c / ((c - 1.0) * (c - 1.0)) * (math.log(n) - math.log(gamma)) / 2.0)
    return int(Lmax), c * (n - 1)


# ----------------------------------------------------------------------------
# Algorithm 1: randomized reconstructing multiple rank-1 lattice
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class MultiLattice:
    M: list[int]                 # lattice sizes (distinct primes), L entries
    z: list[np.ndarray]          # generating vectors, L entries of int64 [t]
    unique: list[np.ndarray]     # I_l as boolean masks over J
    covered: bool                # union of the I_l equals J
    attempts: int                # searches used (1..b)

    @property
    def L(self) -> int:
        return len(self.M)

    def counter(self) -> np.ndarray:
        return np.sum(np.stack(self.unique), axis=0).astype(np.int64)

    def nodes(self) -> int:
        """|Lambda| = 1 - L + sum M_l (Section 2.1; node 0 is shared and, for z
        in [1, M-1]^t and distinct primes, no other node coincides)."""
        return 1 - self.L + int(sum(self.M))


REDRAW_CAP = 64   # replacement draws per lattice in the redraw rule


def construct(J: np.ndarray, seed: int, t: int, attempt: int, c: float = 2.0,
              gamma: float = 0.5, redraw: bool = False) -> MultiLattice:
    """One run of Algorithm 1 on J (rows in Z^t): primes from Eq. (2.2); for
    L = 1..Lmax draw z_L uniformly in [1, M_L - 1]^t, determine I_L, update the
    covered set and stop once it equals J.

    redraw=True applies the rule of the original construction that the remark
    after Algorithm 1 describes: while the new I_L holds no frequency that
    the earlier lattices leave uncovered, z_L is drawn again (at most
    REDRAW_CAP times; after that the last draw is kept)."""
    n = J.shape[0]
    Lmax, lam = lmax_lambda(n, c, gamma)
    primes = prime_set(J, lam, Lmax)
    covered = np.zeros(n, dtype=bool)
    Ms, zs, us = [], [], []
    for L in range(1, Lmax + 1):
        M = primes[L - 1]
        r = 0
        while True:
            z = philox.zvec(seed, t, L - 1, attempt, M, redraw=r)
            IL = unique_mask(J, z, M)
            if not redraw or (IL & ~covered).any() or r == REDRAW_CAP:
                break
            r += 1
        covered |= IL
        Ms.append(M)
        zs.append(z)
        us.append(IL)
        if covered.all():
            return MultiLattice(Ms, zs, us, True, attempt + 1)
    return MultiLattice(Ms, zs, us, False, attempt + 1)


def search(J: np.ndarray, seed: int, t: int, b: int = 10, c: float = 2.0,
           gamma: float = 0.5, redraw: bool = False) -> MultiLattice:
    """Step 2b of Algorithm 3: Algorithm 1 with c = 2, gamma = 0.5, repeated
    until condition (2.1) holds, b searches in total.  After b failed searches
    the last one is used; its uncovered candidates get no coefficient.
    redraw: the redraw rule (see construct)."""
    ml = None
    for attempt in range(b):
        ml = construct(J, seed, t, attempt, c, gamma, redraw)
        if ml.covered:
            return ml
    return ml


# ----------------------------------------------------------------------------
# Algorithm 2: inverse multiple rank-1 lattice FFT
# ----------------------------------------------------------------------------

def lattice_dft_direct(y: np.ndarray, M: int, rr: np.ndarray) -> np.ndarray:
    """(1/M) sum_{j=0}^{M-1} y_j exp(-2 pi i j r / M) at the residues rr, as a
    direct sum with the phase index j r reduced mod M in exact integers."""
    rr = np.asarray(rr, dtype=np.int64)
    out = np.zeros(rr.shape[0], dtype=np.complex128)
    j = np.arange(M, dtype=np.int64)
    step = max(1, 4_000_000 // max(M, 1))
    for a in range(0, rr.shape[0], step):
        ph = np.mod(np.outer(rr[a:a + step], j), M).astype(np.float64) / M
        out[a:a + step] = (np.exp(-2j * np.pi * ph) @ y) / M
    return out


def lattice_dft_fft(y: np.ndarray, M: int, rr: np.ndarray) -> np.ndarray:
    """The same values through a library FFT of length M (numpy pocketfft)."""
    return (np.fft.fft(y) / M)[np.asarray(rr, dtype=np.int64)]


def reconstruct(J: np.ndarray, ml: MultiLattice, ys: list[np.ndarray], dft: str = "fft"):
    """Algorithm 2.  ys[l] holds the M_l samples on lattice l (node j at
    position j).  Returns (p~ over J, counter).  Candidates no lattice covers
    keep p~ = 0 and counter = 0 (no division)."""
    n = J.shape[0]
    acc = np.zeros(n, dtype=np.complex128)
    counter = np.zeros(n, dtype=np.int64)
    f = lattice_dft_direct if dft == "direct" else lattice_dft_fft
    for M, z, IL, y in zip(ml.M, ml.z, ml.unique, ys):
        idx = np.nonzero(IL)[0]
        if idx.size == 0:
            continue
        r = residues(J[idx], z, M)
        acc[idx] += f(np.asarray(y, dtype=np.complex128), M, r)
        counter[idx] += 1
    out = np.zeros(n, dtype=np.complex128)
    ok = counter > 0
    out[ok] = acc[ok] / counter[ok]
    return out, counter


# ----------------------------------------------------------------------------
# Lattice evaluation (Section 4.1 aliasing derivation) and the adjoint of Alg. 2
# ----------------------------------------------------------------------------

def evaluate(J: np.ndarray, ml: MultiLattice, c: np.ndarray, mode: str = "eval",
             dft: str = "fft") -> list[np.ndarray]:
    """mode "eval":    y_{l,j} = sum_{k in J} c_k exp(2 pi i j (k.z_l mod M_l)/M_l),
                       i.e. p(x) = sum c_k e^{2 pi i k.x} at the lattice nodes.
       mode "adjoint": y_{l,j} = sum_{k in I_l} c_k / (counter_k M_l)
                                 * exp(2 pi i j (k.z_l mod M_l)/M_l),
                       the conjugate transpose of the map y -> p~ of Algorithm 2."""
    c = np.asarray(c, dtype=np.complex128)
    counter = ml.counter()
    out = []
    for M, z, IL in zip(ml.M, ml.z, ml.unique):
        r = residues(J, z, M)
        if mode == "eval":
            w = c
            sel = np.ones(J.shape[0], dtype=bool)
        else:
            sel = IL & (counter > 0)
            w = np.zeros_like(c)
            w[sel] = c[sel] / (counter[sel] * M)
        if dft == "direct":
            j = np.arange(M, dtype=np.int64)
            ph = np.mod(np.outer(j, r[sel]), M).astype(np.float64) / M
            out.append(np.exp(2j * np.pi * ph) @ w[sel])
        else:
            B = np.zeros(M, dtype=np.complex128)
            np.add.at(B, r[sel], w[sel])
            out.append(np.fft.ifft(B) * M)
    return out


def dense_reconstruct_matrix(J: np.ndarray, ml: MultiLattice) -> np.ndarray:
    """The matrix R [n, sum M_l] of Algorithm 2 written out entry by entry:
    R[k, (l, j)] = [k in I_l] / (counter_k M_l) * exp(-2 pi i j r_l(k) / M_l)."""
    counter = ml.counter()
    cols = []
    for M, z, IL in zip(ml.M, ml.z, ml.unique):
        r = residues(J, z, M)
        j = np.arange(M, dtype=np.int64)
        ph = np.mod(np.outer(r, j), M).astype(np.float64) / M
        w = np.where(IL & (counter > 0), 1.0 / (np.maximum(counter, 1) * M), 0.0)
        cols.append(w[:, None] * np.exp(-2j * np.pi * ph))
    return np.concatenate(cols, axis=1)
