"""Parity of the CUDA path with the CPU oracle, element by element.

Integer work (residues, collision masks, lattice choice, detected sets) must
match bit-exactly; fp64 coefficients within 1e-10 relative error."""

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
    scale = max(np.max(np.abs(want)), 1e-300)
    return np.max(np.abs(got - want)) / scale


# sizes chosen so that P spans the one-CTA path (P <= 4096) and the 4-step
# path, with ragged candidate counts
SETS = [(1, 1, 3), (7, 1, 4), (50, 2, 5), (333, 3, 6), (1500, 4, 8), (9000, 5, 9), (40000, 6, 10)]


@pytest.mark.parametrize("n,t,N", SETS)
def test_plan_search_bitexact(n, t, N):
    rng = np.random.default_rng(n)
    J = _rand_set(rng, n, t, N)
    ml = lattice.search(J, seed=n + 7, t=t)
    pl = P.plan_search(J, seed=n + 7)
    assert pl.L == ml.L and list(pl.M) == ml.M
    np.testing.assert_array_equal(pl.z, np.stack(ml.z))
    masks, res = pl.masks()
    want_mask = np.zeros(J.shape[0], dtype=np.uint64)
    for l, IL in enumerate(ml.unique):
        want_mask |= IL.astype(np.uint64) << np.uint64(l)
    np.testing.assert_array_equal(masks, want_mask)
    for l, (M, z) in enumerate(zip(ml.M, ml.z)):
        np.testing.assert_array_equal(res[l], lattice.residues(J, z, M))
    assert pl.n_uncovered == int(np.sum(ml.counter() == 0))
    assert pl.nodes == ml.nodes()


@pytest.mark.parametrize("n,t,N", SETS)
def test_reconstruct_parity(n, t, N):
    rng = np.random.default_rng(100 + n)
    J = _rand_set(rng, n, t, N)
    pl = P.plan_search(J, seed=n)
    ml = lattice.search(J, seed=n, t=t)
    nrhs = 3
    y = rng.standard_normal((nrhs, pl.sum_M)) + 1j * rng.standard_normal((nrhs, pl.sum_M))
    got = pl.reconstruct(torch.from_numpy(y).cuda()).cpu().numpy()
    for h in range(nrhs):
        want, _ = lattice.reconstruct(J, ml, np.split(y[h], np.cumsum(ml.M)[:-1]), "fft")
        assert _normwise(got[h], want) < RTOL


@pytest.mark.parametrize("n,t,N", SETS)
@pytest.mark.parametrize("mode", [P.MR1L_EVAL, P.MR1L_ADJOINT])
def test_evaluate_parity(n, t, N, mode):
    rng = np.random.default_rng(200 + n)
    J = _rand_set(rng, n, t, N)
    pl = P.plan_search(J, seed=n)
    ml = lattice.search(J, seed=n, t=t)
    c = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    got = pl.evaluate(torch.from_numpy(c).cuda(), mode).cpu().numpy()
    for h in range(2):
        want = np.concatenate(lattice.evaluate(J, ml, c[h], "eval" if mode == P.MR1L_EVAL else "adjoint", "fft"))
        assert _normwise(got[h], want) < RTOL


def test_reconstruct_direct_tier_small():
    """Against the direct-sum oracle (no library FFT anywhere)."""
    rng = np.random.default_rng(3)
    J = _rand_set(rng, 120, 3, 5)
    pl = P.plan_search(J, seed=9)
    ml = lattice.search(J, seed=9, t=3)
    y = rng.standard_normal(pl.sum_M) + 1j * rng.standard_normal(pl.sum_M)
    got = pl.reconstruct(torch.from_numpy(y).cuda()).cpu().numpy()
    want, _ = lattice.reconstruct(J, ml, np.split(y, np.cumsum(ml.M)[:-1]), "direct")
    assert _normwise(got, want) < RTOL


def test_given_lattice_plan_and_uncovered():
    """mr1l_plan with explicit lattices, one frequency left uncovered: its
    coefficient is 0; MR1L_STRICT refuses the plan."""
    J = np.array([[0], [3], [6], [1]])
    M, z = [3], [[1]]
    pl = P.plan(J, M, z)
    assert pl.n_uncovered == 3
    y = torch.ones(3, dtype=torch.complex128, device="cuda")
    got = pl.reconstruct(y).cpu().numpy()
    ml = lattice.MultiLattice([3], [np.array([1])], [lattice.unique_mask(J, [1], 3)], False, 1)
    want, _ = lattice.reconstruct(J, ml, [np.ones(3, dtype=complex)], "direct")
    np.testing.assert_allclose(got, want, atol=1e-15)
    with pytest.raises(P.Mr1lError) as e:
        P.plan(J, M, z, strict=True)
    assert e.value.code == P.MR1L_E_NOT_RECONSTRUCTING


@pytest.mark.parametrize("M", [2, 5, 7, 13, 2039, 2053, 4093, 4099])
def test_small_and_boundary_primes(M):
    """One lattice of prime size M: Bluestein lengths 3, 12, 16, 32 (the
    one-CTA path), 4096 (its largest), 6144, 8192 and 12288 (the smallest
    4-step lengths), with every residue class occupied (I = 0..M-1, z = 1)
    against the direct-sum oracle, forward and both evaluation modes."""
    I = np.arange(M).reshape(-1, 1)
    pl = P.plan(I, [M], [[1]], strict=True)
    ml = lattice.MultiLattice([M], [np.array([1])], [np.ones(M, dtype=bool)], True, 1)
    rng = np.random.default_rng(M)
    y = rng.standard_normal((2, M)) + 1j * rng.standard_normal((2, M))
    c = rng.standard_normal((2, M)) + 1j * rng.standard_normal((2, M))
    got = pl.reconstruct(torch.from_numpy(y).cuda()).cpu().numpy()
    ge = pl.evaluate(torch.from_numpy(c).cuda(), P.MR1L_EVAL).cpu().numpy()
    ga = pl.evaluate(torch.from_numpy(c).cuda(), P.MR1L_ADJOINT).cpu().numpy()
    for h in range(2):
        want, _ = lattice.reconstruct(I, ml, [y[h]], "direct")
        assert _normwise(got[h], want) < RTOL
        assert _normwise(ge[h], np.concatenate(lattice.evaluate(I, ml, c[h], "eval", "direct"))) < RTOL
        assert _normwise(ga[h], np.concatenate(lattice.evaluate(I, ml, c[h], "adjoint", "direct"))) < RTOL


@pytest.mark.parametrize("M", [1_300_021, 2_000_003, 3_000_017, 8_000_009, 10_000_019, 16_700_003])
def test_large_single_lattice_4step(M):
    """One lattice per case, chosen so that the Bluestein length is 3 * 2^20,
    2^22, 3 * 2^21 (one-column tiles), 2^24, 3 * 2^23 (single 6144-element
    columns, 768-thread CTAs) and 2^25 (the largest: single 8192-element rows,
    1024-thread CTAs), against numpy's FFT."""
    assert lattice.is_prime(M)
    I = np.arange(-30000, 30000).reshape(-1, 1)
    pl = P.plan(I, [M], [[7919]])
    rng = np.random.default_rng(1)
    y = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    got = pl.reconstruct(torch.from_numpy(y).cuda()).cpu().numpy()
    ml = lattice.MultiLattice([M], [np.array([7919])], [lattice.unique_mask(I, [7919], M)], True, 1)
    want, _ = lattice.reconstruct(I, ml, [y], "fft")
    assert _normwise(got, want) < RTOL
    yb = pl.evaluate(torch.from_numpy(want).cuda(), P.MR1L_ADJOINT).cpu().numpy()
    wantb = np.concatenate(lattice.evaluate(I, ml, want, "adjoint", "fft"))
    assert _normwise(yb[0] if yb.ndim > 1 else yb, wantb) < RTOL


@pytest.mark.parametrize("M", [1_300_021, 2_000_003])
@pytest.mark.parametrize("width", [300, 30000])
def test_large_lattice_evaluation(M, width):
    """Lattice evaluation through the 4-step passes, with Bluestein lengths
    3 * 2^20 and 3 * 2^21 (a 48 KB column tile): few candidates leave every
    column of the padded input with a handful of non-zeros (the direct column
    transform), many leave dozens per column (the column FFT)."""
    I = np.arange(-width, width).reshape(-1, 1)
    pl = P.plan(I, [M], [[7919]])
    ml = lattice.MultiLattice([M], [np.array([7919])], [lattice.unique_mask(I, [7919], M)], True, 1)
    rng = np.random.default_rng(M + width)
    c = rng.standard_normal(I.shape[0]) + 1j * rng.standard_normal(I.shape[0])
    got = pl.evaluate(torch.from_numpy(c).cuda(), P.MR1L_EVAL).cpu().numpy()
    want = np.concatenate(lattice.evaluate(I, ml, c, "eval", "fft"))
    assert _normwise(got[0] if got.ndim > 1 else got, want) < RTOL


def _sfft_pair(name, seed, batch=False):
    sig, p = W.workload(name, seed)
    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=seed, b=p["b"],
                         freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma, batch_reps=batch)
    ref = sfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=seed)
    return sig, out, ref


def _assert_sfft_equal(out, ref):
    for st, rs in zip(out.steps, ref.steps):
        assert st["n_line"] == rs.I_t and st["n_cand"] == rs.n_candidates
        assert st["L"] == rs.L and st["attempts"] == rs.attempts and st["covered"] == rs.covered
        assert st["samples"] == rs.samples
    np.testing.assert_array_equal(out.freqs, ref.freqs)
    assert out.samples == ref.samples
    rel = np.abs(out.coeffs - ref.coeffs) / np.abs(ref.coeffs)
    assert rel.size == 0 or rel.max() < RTOL


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_sfft_tiny_d3_parity(seed):
    sig, out, ref = _sfft_pair("tiny_d3", seed)
    _assert_sfft_equal(out, ref)
    np.testing.assert_array_equal(out.freqs, sig.freqs.astype(np.int64))


def test_sfft_plain_d10_parity():
    """The full d = 10, N = 32, s = 1000, 40 dB, r = 5 workload."""
    sig, out, ref = _sfft_pair("plain_d10", 1)
    assert min(s.min_gap_rank for s in ref.steps) > 1e-9, "degenerate seed (near tie)"
    _assert_sfft_equal(out, ref)


@pytest.mark.parametrize("seed", [1, 2])
def test_sfft_zero_anchors_parity(seed):
    """The deterministic variant (anchors 0, r = 1) on coefficients with
    positive real parts, noiseless and at 30 dB, against the oracle."""
    for snr in (None, 30.0):
        sig = W.planted_signal(5, 8, 80, seed=seed, model="posre", snr_db=snr)
        out = P.sfft_dimincr(5, 8, 80, 1, 1e-12, "abs", seed=seed, freqs=sig.freqs, coeffs=sig.coeffs,
                             sigma=sig.sigma, zero_anchors=True)
        ref = sfft.sfft(sig, 80, 80, 1, 10, 1e-12, "abs", seed=seed, zero_anchors=True)
        assert min(st.min_gap_rank for st in ref.steps) > 1e-9, "degenerate seed (near tie)"
        _assert_sfft_equal(out, ref)
        if snr is None:
            np.testing.assert_array_equal(out.freqs, sig.freqs.astype(np.int64))


def test_sfft_smallest_box():
    """N = 1 (frequencies in {-1, 0, 1}^6, K = 3 line samples): half of the
    box planted."""
    sig = W.planted_signal(6, 1, 360, seed=3, model="u1_10")
    out = P.sfft_dimincr(6, 1, 360, 2, 1e-12, "rel", seed=3, freqs=sig.freqs, coeffs=sig.coeffs)
    ref = sfft.sfft(sig, 360, 360, 2, 10, 1e-12, "rel", seed=3)
    _assert_sfft_equal(out, ref)
    np.testing.assert_array_equal(out.freqs, sig.freqs.astype(np.int64))


def test_sfft_batched_reps_identical():
    sig, out, ref = _sfft_pair("tiny_d3", 5, batch=True)
    _assert_sfft_equal(out, ref)


def test_sfft_callback_sampler_matches_planted():
    """A user sampler (here: the planted polynomial evaluated on the host and
    copied to the device) gives the same result as the built-in one."""
    import ctypes
    sig, p = W.workload("tiny_d3", 6)
    cudart = None
    for name in ("libcudart.so", "/usr/local/cuda/lib64/libcudart.so", "libcudart.so.13"):
        try:
            cudart = ctypes.CDLL(name)
            break
        except OSError:
            continue
    if cudart is None:
        pytest.skip("libcudart not loadable through ctypes")

    def sampler(req, y_ptr, stream_ptr):
        x = np.ctypeslib.as_array(req.anchors, shape=(req.d,)).copy()
        if req.kind == P.SFFT_REQ_LINE:
            vals = sfft.sample_line(sig, req.t, x, req.K, "direct")
        else:
            Ms = np.ctypeslib.as_array(req.M, shape=(req.L,)).tolist()
            zs = np.ctypeslib.as_array(req.z, shape=(req.L * req.t,)).reshape(req.L, req.t)
            ml = lattice.MultiLattice(Ms, list(zs), [], True, 1)
            vals = np.concatenate(sfft.sample_lattice(sig, req.t, ml, x, "fft"))
        buf = np.ascontiguousarray(vals.astype(np.complex128))
        rc = cudart.cudaMemcpy(ctypes.c_void_p(y_ptr), buf.ctypes.data_as(ctypes.c_void_p),
                               ctypes.c_size_t(buf.nbytes), 1)
        return rc

    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=6, b=p["b"],
                         sampler=sampler)
    ref = sfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=6)
    _assert_sfft_equal(out, ref)


def test_sfft_nothing_detected():
    """Absolute threshold above every coefficient: empty output, no failure."""
    sig, p = W.workload("tiny_d3", 7)
    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], 1e6, "abs", seed=7, freqs=sig.freqs, coeffs=sig.coeffs)
    ref = sfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], 1e6, "abs", seed=7)
    assert out.freqs.shape == (0, 3) and ref.freqs.shape[0] == 0
    assert out.samples == ref.samples


def test_sfft_d2_and_caps():
    """d = 2 (a single lattice increment) with a cap below the support size."""
    sig = W.planted_signal(2, 20, 60, seed=8)
    out = P.sfft_dimincr(2, 20, 25, 2, 1e-12, "rel", seed=8, freqs=sig.freqs, coeffs=sig.coeffs)
    ref = sfft.sfft(sig, 25, 25, 2, 10, 1e-12, "rel", seed=8)
    _assert_sfft_equal(out, ref)
    assert out.freqs.shape[0] == 25


def test_batched_plans_match_single_calls():
    """mr1l_reconstruct_batch / mr1l_evaluate_batch over plans of different
    sizes (one listed twice) give exactly the single-call results."""
    rng = np.random.default_rng(77)
    plans, ys, cs = [], [], []
    for n, t, N in [(50, 2, 5), (1500, 4, 8), (9000, 5, 9)]:
        J = _rand_set(rng, n, t, N)
        pl = P.plan_search(J, seed=n)
        plans.append(pl)
        ys.append(torch.from_numpy(rng.standard_normal((2, pl.sum_M)) + 1j * rng.standard_normal((2, pl.sum_M))).cuda())
        cs.append(torch.from_numpy(rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))).cuda())
    plans.append(plans[1])
    ys.append(ys[1] * 2)
    cs.append(cs[1] * 2)
    got = P.reconstruct_batch(plans, ys)
    gote = P.evaluate_batch(plans, cs, P.MR1L_ADJOINT)
    torch.cuda.synchronize()
    for pl, y, c, g, ge in zip(plans, ys, cs, got, gote):
        np.testing.assert_array_equal(g.cpu().numpy(), pl.reconstruct(y).cpu().numpy())
        np.testing.assert_array_equal(ge.cpu().numpy(), pl.evaluate(c, P.MR1L_ADJOINT).cpu().numpy())


@pytest.mark.parametrize("n,t,N", [(7, 1, 4), (50, 2, 5), (333, 3, 6), (1500, 4, 8), (9000, 5, 9)])
def test_plan_search_redraw_bitexact(n, t, N):
    """Algorithm 1 with the redraw rule (the remark after it): the same
    lattices, generating vectors and collision-free sets as the oracle."""
    rng = np.random.default_rng(n + 1)
    J = _rand_set(rng, n, t, N)
    for seed in range(3):
        ml = lattice.search(J, seed=seed, t=t, redraw=True)
        pl = P.plan_search(J, seed=seed, redraw=True)
        assert pl.L == ml.L and list(pl.M) == ml.M
        np.testing.assert_array_equal(pl.z, np.stack(ml.z))
        masks, _ = pl.masks()
        want_mask = np.zeros(J.shape[0], dtype=np.uint64)
        for l, IL in enumerate(ml.unique):
            want_mask |= IL.astype(np.uint64) << np.uint64(l)
        np.testing.assert_array_equal(masks, want_mask)


@pytest.mark.parametrize("name,seed", [("tiny_d3", 11), ("tiny_d3", 12)])
def test_sfft_redraw_parity(name, seed):
    sig, p = W.workload(name, seed)
    out = P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=seed, b=p["b"],
                         freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma, redraw=True)
    ref = sfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=seed, redraw=True)
    _assert_sfft_equal(out, ref)


def test_sfft_redraw_parity_d6():
    """A six-dimensional planted signal (noisy) with the redraw rule, and
    its sample count at most the plain rule's."""
    sig = W.planted_signal(6, 12, 150, seed=13, model="u1_10", snr_db=30.0)
    out = P.sfft_dimincr(6, 12, 150, 3, 1e-12, "rel", seed=13, freqs=sig.freqs, coeffs=sig.coeffs,
                         sigma=sig.sigma, redraw=True, batch_reps=True)
    ref = sfft.sfft(sig, 150, 150, 3, 10, 1e-12, "rel", seed=13, redraw=True)
    _assert_sfft_equal(out, ref)


@pytest.mark.parametrize("density", [0.003, 0.03, 0.1, 0.3])
@pytest.mark.parametrize("fft", ["f64", "df"])
def test_evaluate_sparse_coefficients(density, fft):
    """Lattice evaluation of sparse coefficient vectors, where the evaluation
    column pass sums the few non-zeros of each column directly (plain sums
    for one or two, the split by n1 mod 8 for three to 24, the column FFT in
    tiles holding a denser column): against the oracle, normwise and at
    every sample that a single coefficient would make non-zero."""
    rng = np.random.default_rng(int(density * 1e4))
    J = _rand_set(rng, 40000, 6, 10)
    pl = P.plan_search(J, seed=41, fft=fft)
    ml = lattice.search(J, seed=41, t=6)
    c = np.zeros((2, J.shape[0]), dtype=np.complex128)
    for h in range(2):
        k = rng.random(J.shape[0]) < density
        c[h, k] = rng.standard_normal(k.sum()) + 1j * rng.standard_normal(k.sum())
    got = pl.evaluate(torch.from_numpy(c).cuda(), P.MR1L_EVAL).cpu().numpy()
    for h in range(2):
        want = np.concatenate(lattice.evaluate(J, ml, c[h], "eval", "fft"))
        assert _normwise(got[h], want) < RTOL
