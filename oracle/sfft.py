"""Algorithm 3 (MLFFT): dimension-incremental sparse FFT over multiple rank-1
lattices (oracle side).

Readings of passages the paper leaves open (also listed in the design notes):
  * every 1-D detection DFT carries the factor 1/K_t (step 1 has it; step 2a
    and Eq. 4.2 drop it; Eq. 4.2 only holds with it);
  * thresholds compare squared magnitudes: key = re*re + im*im (no fused
    multiply-add), kept when key >= theta^2 * max key of the pass (relative
    mode) or key >= theta^2 (absolute mode, the paper's delta);
  * "(up to) s-largest": descending key, ties to the smaller candidate id
    (lexicographic rank of the frequency); candidates that no lattice covers
    are never selected;
  * generating vectors are drawn from [1, M-1]^t (z in Z^t at step t);
  * b is the total number of lattice searches (default 10);
  * node 0 is shared by all lattices: one noise value for it;
  * the union over the r~ passes is capped only through each pass's s~;
  * the output coefficients are those of the single pass at t = d.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import lattice, philox


# ----------------------------------------------------------------------------
# Sampling the planted polynomial (the black box p of Algorithm 3)
# ----------------------------------------------------------------------------

def _phase_weights(freqs: np.ndarray, coeffs: np.ndarray, x: np.ndarray, comps) -> np.ndarray:
    """c_h * exp(2 pi i sum_{j in comps} h_j x_j) for every planted h."""
    comps = list(comps)
    if not comps:
        return coeffs.astype(np.complex128).copy()
    phi = freqs[:, comps].astype(np.float64) @ x[comps]
    phi = phi - np.floor(phi)
    return coeffs * np.exp(2j * np.pi * phi)


def sample_line(sig, t: int, x: np.ndarray, K: int, dft: str = "fft") -> np.ndarray:
    """p(x_1', .., x_{t-1}', l/K, x_{t+1}', .., x_d') for l = 0..K-1 (t is 1-based).
    A signal given in the spatial domain (sig.value, e.g. the Section 5.3
    function) is evaluated at the nodes directly."""
    if hasattr(sig, "value"):
        X = np.tile(np.asarray(x, dtype=np.float64), (K, 1))
        X[:, t - 1] = np.arange(K, dtype=np.float64) / K
        return sig.value(X)
    others = [j for j in range(sig.d) if j != t - 1]
    w = _phase_weights(sig.freqs, sig.coeffs, x, others)
    ht = sig.freqs[:, t - 1].astype(np.int64)
    if dft == "direct":
        l = np.arange(K, dtype=np.float64)
        return np.exp(2j * np.pi * np.outer(l, ht.astype(np.float64)) / K) @ w
    B = np.zeros(K, dtype=np.complex128)
    np.add.at(B, np.mod(ht, K), w)
    return np.fft.ifft(B) * K


def sample_lattice(sig, t: int, ml: lattice.MultiLattice, x: np.ndarray,
                   dft: str = "fft") -> list[np.ndarray]:
    """p(j z_l / M_l mod 1, x_{t+1}', .., x_d') for every lattice l and node j.
    "direct" evaluates p(x) = sum_h c_h e^{2 pi i h.x} at each node; "fft" uses
    the aliasing identity of Section 4.1 (bin h_{1..t}.z_l mod M_l, weight
    c_h e^{2 pi i h_{>t}.x'}) and a length-M_l inverse library FFT.  A
    spatial-domain signal (sig.value) is evaluated at the nodes directly."""
    if hasattr(sig, "value"):
        out = []
        for M, z in zip(ml.M, ml.z):
            X = np.tile(np.asarray(x, dtype=np.float64), (M, 1))
            j = np.arange(M, dtype=np.int64)
            X[:, :t] = np.mod(np.outer(j, np.asarray(z, dtype=np.int64)), M).astype(np.float64) / M
            out.append(sig.value(X))
        return out
    w = _phase_weights(sig.freqs, sig.coeffs, x, range(t, sig.d))
    head = sig.freqs[:, :t].astype(np.int64)
    out = []
    for M, z in zip(ml.M, ml.z):
        if dft == "direct":
            j = np.arange(M, dtype=np.int64)
            nodes = np.mod(np.outer(j, z), M).astype(np.float64) / M       # [M, t]
            ph = nodes @ head.T.astype(np.float64)                         # [M, s]
            ph = ph - np.floor(ph)
            out.append(np.exp(2j * np.pi * ph) @ w)
        else:
            B = np.zeros(M, dtype=np.complex128)
            np.add.at(B, lattice.residues(head, z, M), w)
            out.append(np.fft.ifft(B) * M)
    return out


def line_noise(seed: int, t: int, i: int, K: int, sigma: float) -> np.ndarray:
    g1, g2 = philox.normal_pairs(seed, philox.NOISE_LINE, t, np.arange(K, dtype=np.uint64), 0, i)
    return sigma / math.sqrt(2.0) * (g1 + 1j * g2)


def lattice_noise(seed: int, t: int, i: int, ml: lattice.MultiLattice, sigma: float):
    """eta_{l,j} = sigma/sqrt(2) (g1 + i g2) (Section 5.2); node 0 is one node of
    the multiple lattice, so all lattices see the same eta_{.,0}."""
    out = []
    for l, M in enumerate(ml.M):
        j = np.arange(M, dtype=np.uint64)
        ll = np.where(j == 0, 0, l).astype(np.uint64)
        g1, g2 = philox.normal_pairs(seed, philox.NOISE_LAT, t, j, ll, i)
        out.append(sigma / math.sqrt(2.0) * (g1 + 1j * g2))
    return out


# ----------------------------------------------------------------------------
# Thresholded "(up to) s-largest" selection (steps 1, 2a, 2e)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Selection:
    chosen: np.ndarray      # sorted candidate ids
    thr: float              # squared threshold used
    gap_rank: float         # relative gap between the s-th and (s+1)-th eligible keys (inf if none)
    gap_thr: float          # smallest relative distance of a key to the threshold


def select(p: np.ndarray, cap: int, theta: float, theta_mode: str,
           eligible: np.ndarray | None = None) -> Selection:
    re, im = p.real, p.imag
    key = re * re + im * im
    if eligible is None:
        eligible = np.ones(p.shape[0], dtype=bool)
    key = np.where(eligible, key, 0.0)
    if theta_mode == "rel":
        thr = (theta * theta) * (float(key.max()) if key.size else 0.0)
    else:
        thr = theta * theta
    ok = eligible & (key >= thr)
    idx = np.nonzero(ok)[0]
    order = idx[np.lexsort((idx, -key[idx]))]
    chosen = np.sort(order[:cap])
    gap_rank = math.inf
    if order.size > cap and cap > 0:
        a, b = key[order[cap - 1]], key[order[cap]]
        gap_rank = (a - b) / max(a, 1e-300)
    elig_keys = key[eligible]
    if elig_keys.size and thr > 0:
        gap_thr = float(np.min(np.abs(elig_keys - thr)) / thr)
    else:
        gap_thr = math.inf
    return Selection(chosen, thr, gap_rank, gap_thr)


# ----------------------------------------------------------------------------
# Algorithm 3
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class StepStats:
    t: int
    I_t: int                 # |I^(t)| from the 1-D detection
    n_candidates: int        # |J_t|
    L: int
    sum_M: int
    attempts: int
    covered: bool
    samples: int             # samples used at this increment (lines + lattices)
    min_gap_rank: float
    min_gap_thr: float


@dataclasses.dataclass
class SfftResult:
    freqs: np.ndarray        # int64 [n, d], lexicographic
    coeffs: np.ndarray       # complex128 [n]
    samples: int
    steps: list[StepStats]
    lines: list[np.ndarray]  # I^(t) per t (sorted k values)


def line_coefficients(y: np.ndarray, N: int) -> np.ndarray:
    """p~_{t,k} = (1/K) sum_{l=0}^{K-1} y_l exp(-2 pi i l k / K) for k = -N..N
    (K = 2N+1), as a direct sum with l k reduced mod K in integers."""
    K = 2 * N + 1
    k = np.arange(-N, N + 1, dtype=np.int64)
    l = np.arange(K, dtype=np.int64)
    ph = np.mod(np.outer(np.mod(k, K), l), K).astype(np.float64) / K
    return (np.exp(-2j * np.pi * ph) @ y) / K


def anchor(seed: int, purpose: int, t: int, d: int, i: int, zero: bool) -> np.ndarray:
    """The anchor x' of pass i (Algorithm 3 steps 1, 2a and 2c): Philox
    uniforms, or all zeros in the deterministic variant the paper remarks on
    in Section 3 (same-sign real or imaginary parts, r = 1)."""
    if zero:
        return np.zeros(d)
    return philox.uniform(seed, purpose, t, np.arange(d, dtype=np.uint64), 0, i)


def detect_1d(sig, t: int, seed: int, r: int, s_local: int, theta: float, theta_mode: str,
              dft: str = "fft", zero_anchors: bool = False):
    """Steps 1 and 2a: r random lines through the t-th coordinate; length-K_t
    DFT with factor 1/K_t; union of the (up to) s_local largest values above
    the threshold.  Returns (sorted k values, min rank gap, min threshold gap)."""
    N, d = sig.N, sig.d
    K = 2 * N + 1
    chosen = np.zeros(K, dtype=bool)
    gr, gt = math.inf, math.inf
    k = np.arange(-N, N + 1, dtype=np.int64)
    for i in range(r):
        x = anchor(seed, philox.ANCHOR_LINE, t, d, i, zero_anchors)
        y = sample_line(sig, t, x, K, dft)
        if sig.sigma > 0:
            y = y + line_noise(seed, t, i, K, sig.sigma)
        p = line_coefficients(y, N)
        sel = select(p, s_local, theta, theta_mode)
        chosen[sel.chosen] = True
        gr, gt = min(gr, sel.gap_rank), min(gt, sel.gap_thr)
    return k[chosen], gr, gt


def candidates(prefix: np.ndarray, last: np.ndarray) -> np.ndarray:
    """J_t = I^(1..t-1) x I^(t) (the full box Gamma makes the intersection a
    no-op); candidate id = p * |I^(t)| + q keeps lexicographic order."""
    npre, nq = prefix.shape[0], last.shape[0]
    J = np.empty((npre * nq, prefix.shape[1] + 1), dtype=np.int64)
    J[:, :-1] = np.repeat(prefix, nq, axis=0)
    J[:, -1] = np.tile(last, npre)
    return J


def lattice_pass(sig, t: int, seed: int, i: int, J: np.ndarray, ml: lattice.MultiLattice,
                 cap: int, theta: float, theta_mode: str, eligible: np.ndarray, dft: str = "fft",
                 zero_anchors: bool = False):
    """Steps 2c-2e of Algorithm 3 for detection iteration i: sample p along
    the multiple rank-1 lattice (anchor x'_{t+1..d} of pass i), reconstruct
    every p~_k by Algorithm 2 and select the (up to) cap largest above the
    threshold.  Returns (p~, Selection)."""
    x = anchor(seed, philox.ANCHOR_LAT, t, sig.d, i, zero_anchors)
    ys = sample_lattice(sig, t, ml, x, dft)
    if sig.sigma > 0:
        ys = [y + e for y, e in zip(ys, lattice_noise(seed, t, i, ml, sig.sigma))]
    p, _ = lattice.reconstruct(J, ml, ys, dft)
    return p, select(p, cap, theta, theta_mode, eligible)


def _lattice_pass_job(args):
    return lattice_pass(*args)


def sfft(sig, s: int, s_local: int, r: int, b: int, theta: float, theta_mode: str,
         seed: int, dft: str = "fft", t_stop: int | None = None, zero_anchors: bool = False,
         rep_map=map, redraw: bool = False) -> SfftResult:
    """Algorithm 3.  t_stop (optional) ends the run after that dimension
    increment (a bounded sample of the work; the result is then the
    projected set I^(1..t_stop)).  zero_anchors: every anchor x' is 0 (the
    deterministic variant of the remark in Section 3).  rep_map applies the
    independent detection iterations of an increment (default: the builtin
    map, one after another; a process pool's map runs them side by side with
    the same arithmetic).  redraw: Algorithm 1 with the redraw rule of the
    remark after it (see lattice.construct)."""
    d = sig.d
    if d < 2:
        raise ValueError("the dimension-incremental method needs d >= 2")
    K = 2 * sig.N + 1
    steps: list[StepStats] = []
    lines = []
    I1, gr, gt = detect_1d(sig, 1, seed, r, s_local, theta, theta_mode, dft, zero_anchors)
    lines.append(I1)
    samples = r * K
    prefix = I1.reshape(-1, 1)
    coeffs = np.zeros(0, dtype=np.complex128)
    for t in range(2, d + 1):
        if t_stop is not None and t > t_stop:
            break
        It, gr, gt = detect_1d(sig, t, seed, r, s_local, theta, theta_mode, dft, zero_anchors)
        lines.append(It)
        rt, st = (r, s_local) if t < d else (1, s)
        J = candidates(prefix, It)
        n = J.shape[0]
        step_samples = r * K
        if n == 0:
            prefix = np.zeros((0, t), dtype=np.int64)
            steps.append(StepStats(t, It.size, 0, 0, 0, 0, True, step_samples, gr, gt))
            samples += step_samples
            continue
        ml = lattice.search(J, seed, t, b, redraw=redraw)
        eligible = ml.counter() > 0
        detected = np.zeros(n, dtype=bool)
        p = None
        jobs = [(sig, t, seed, i, J, ml, st, theta, theta_mode, eligible, dft, zero_anchors) for i in range(rt)]
        for p, sel in rep_map(_lattice_pass_job, jobs):
            detected[sel.chosen] = True
            gr, gt = min(gr, sel.gap_rank), min(gt, sel.gap_thr)
            step_samples += ml.nodes()
        prefix = J[detected]
        if t == d:
            coeffs = p[detected]
        steps.append(StepStats(t, It.size, n, ml.L, int(sum(ml.M)), ml.attempts, ml.covered,
                               step_samples, gr, gt))
        samples += step_samples
    return SfftResult(prefix, coeffs, samples, steps, lines)
