"""The double-float FFT mode (butterflies as FP32 pairs on the FP32 pipes)
against the oracle, at the same bar as the FP64 path: integer work and
detected sets bit-exact, coefficients within 1e-10 relative error."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
import workloads as W
from oracle import lattice, sfft

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()


def _rand_set(rng, n, t, N):
    J = np.unique(rng.integers(-N, N + 1, size=(int(1.5 * n) + 8, t)), axis=0)
    rng.shuffle(J)
    J = J[:n]
    return J[np.lexsort(J.T[::-1])].astype(np.int64)


def _normwise(got, want):
    return np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300)


SETS = [(7, 1, 4), (333, 3, 6), (1500, 4, 8), (9000, 5, 9), (40000, 6, 10)]


@pytest.mark.parametrize("n,t,N", SETS)
def test_df_reconstruct_and_adjoint(n, t, N):
    rng = np.random.default_rng(300 + n)
    J = _rand_set(rng, n, t, N)
    pl = P.plan_search(J, seed=n, fft="df")
    ml = lattice.search(J, seed=n, t=t)
    y = rng.standard_normal((2, pl.sum_M)) + 1j * rng.standard_normal((2, pl.sum_M))
    got = pl.reconstruct(torch.from_numpy(y).cuda()).cpu().numpy()
    c = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    gotb = pl.evaluate(torch.from_numpy(c).cuda(), P.MR1L_ADJOINT).cpu().numpy()
    for h in range(2):
        want, _ = lattice.reconstruct(J, ml, np.split(y[h], np.cumsum(ml.M)[:-1]), "fft")
        assert _normwise(got[h], want) < RTOL
        wantb = np.concatenate(lattice.evaluate(J, ml, c[h], "adjoint", "fft"))
        assert _normwise(gotb[h], wantb) < RTOL


@pytest.mark.parametrize("M", [1_300_021, 3_000_017, 16_700_003])
def test_df_large_lattice(M):
    I = np.arange(-30000, 30000).reshape(-1, 1)
    pl = P.plan(I, [M], [[7919]], fft="df")
    rng = np.random.default_rng(2)
    y = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    got = pl.reconstruct(torch.from_numpy(y).cuda()).cpu().numpy()
    ml = lattice.MultiLattice([M], [np.array([7919])], [lattice.unique_mask(I, [7919], M)], True, 1)
    want, _ = lattice.reconstruct(I, ml, [y], "fft")
    assert _normwise(got, want) < RTOL


def _pair(name, seed, **kw):
    sig, p = W.workload(name, seed)
    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=seed, b=p["b"],
                         freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma, batch_reps=True, fft="df", **kw)
    ref = sfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=seed,
                    t_stop=kw.get("t_stop"))
    return out, ref


def _assert_equal(out, ref):
    for st, rs in zip(out.steps, ref.steps):
        assert (st["n_line"], st["n_cand"], st["L"], st["attempts"], st["samples"]) == \
            (rs.I_t, rs.n_candidates, rs.L, rs.attempts, rs.samples)
    np.testing.assert_array_equal(out.freqs, ref.freqs)
    assert out.samples == ref.samples
    if ref.coeffs.size:
        assert np.max(np.abs(out.coeffs - ref.coeffs) / np.abs(ref.coeffs)) < RTOL


@pytest.mark.parametrize("seed", [1, 2])
def test_df_sfft_tiny(seed):
    _assert_equal(*_pair("tiny_d3", seed))


def test_df_sfft_plain_d10():
    _assert_equal(*_pair("plain_d10", 1))


@pytest.mark.slow
def test_df_sfft_large_first_increments():
    _assert_equal(*_pair("large_d25", 1, t_stop=3))
