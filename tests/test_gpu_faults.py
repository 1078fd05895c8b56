"""Failures made on the host, never on the GPU: a user sampler that reports an
error (Algorithm 3 treats the function as a black box it can only sample),
and device allocations that fail (injected in the library's host-side block
allocator).  Each must come back as its status code, leave no device block
outstanding, and leave the library usable: the next solve still matches the
oracle."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
import workloads as W
from oracle import lattice, sfft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()
    yield
    P.inject_alloc_failure(-1)


def _cudart():
    for name in ("libcudart.so", "/usr/local/cuda/lib64/libcudart.so", "libcudart.so.13"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcudart not loadable through ctypes")


def _outstanding():
    torch.cuda.synchronize()
    return P.pool_stats(torch.cuda.current_device())["outstanding"]


def _tiny():
    sig, p = W.workload("tiny_d3", 3)
    return sig, p


def _solve_planted(sig, p, seed=3):
    return P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=seed, b=p["b"],
                          freqs=sig.freqs, coeffs=sig.coeffs, sigma=sig.sigma)


def _assert_matches_oracle(out, sig, p, seed=3):
    ref = sfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=seed)
    np.testing.assert_array_equal(out.freqs, ref.freqs)
    assert np.max(np.abs(out.coeffs - ref.coeffs) / np.abs(ref.coeffs)) < 1e-10
    assert out.samples == ref.samples


@pytest.mark.parametrize("fail_kind,fail_t", [(P.SFFT_REQ_LINE, 2), (P.SFFT_REQ_LATTICE, 2),
                                              (P.SFFT_REQ_LATTICE, 3)])
def test_sampler_error(fail_kind, fail_t):
    """A callback that returns non-zero at a chosen request: MR1L_E_SAMPLER,
    a message naming the request, nothing leaked; the next solve is exact."""
    cudart = _cudart()
    sig, p = _tiny()
    calls = []

    def sampler(req, y_ptr, stream_ptr):
        calls.append((req.kind, req.t))
        if req.kind == fail_kind and req.t == fail_t:
            return 7
        x = np.ctypeslib.as_array(req.anchors, shape=(req.d,)).copy()
        if req.kind == P.SFFT_REQ_LINE:
            vals = sfft.sample_line(sig, req.t, x, req.K, "fft")
        else:
            Ms = np.ctypeslib.as_array(req.M, shape=(req.L,)).tolist()
            zs = np.ctypeslib.as_array(req.z, shape=(req.L * req.t,)).reshape(req.L, req.t)
            ml = lattice.MultiLattice(Ms, list(zs), [], True, 1)
            vals = np.concatenate(sfft.sample_lattice(sig, req.t, ml, x, "fft"))
        buf = np.ascontiguousarray(vals.astype(np.complex128))
        return cudart.cudaMemcpy(ctypes.c_void_p(y_ptr), buf.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_size_t(buf.nbytes), 1)

    before = _outstanding()
    with pytest.raises(P.Mr1lError) as e:
        P.sfft_dimincr(sig.d, sig.N, p["s"], p["r"], p["theta"], p["theta_mode"], seed=3, b=p["b"],
                       sampler=sampler)
    assert e.value.code == P.MR1L_E_SAMPLER
    assert ("line request" if fail_kind == P.SFFT_REQ_LINE else "lattice request") in str(e.value)
    assert f"t = {fail_t}" in str(e.value)
    assert calls[-1] == (fail_kind, fail_t)
    assert _outstanding() == before
    _assert_matches_oracle(_solve_planted(sig, p), sig, p)


def test_injected_allocation_failures_in_sfft():
    """The k-th device allocation of a solve fails, for k spread over the
    whole run: MR1L_E_NOMEM (or success once k exceeds the run's count),
    every block returned, and the library still exact afterwards."""
    sig, p = _tiny()
    failed = 0
    for after in (0, 1, 2, 5, 9, 14, 20, 30, 45, 70, 100, 1000):
        before = _outstanding()
        P.inject_alloc_failure(after)
        try:
            out = _solve_planted(sig, p)
        except P.Mr1lError as e:
            assert e.code == P.MR1L_E_NOMEM
            assert "injected" in str(e)
            failed += 1
        else:
            _assert_matches_oracle(out, sig, p)
        finally:
            P.inject_alloc_failure(-1)
        assert _outstanding() == before, f"blocks leaked after a failure at request {after}"
    assert failed >= 5
    _assert_matches_oracle(_solve_planted(sig, p), sig, p)


def test_injected_allocation_failure_in_plan_and_transform():
    """Plan construction and a transform whose allocation fails report
    MR1L_E_NOMEM; the plan stays usable for the next transform."""
    rng = np.random.default_rng(4)
    J = np.unique(rng.integers(-6, 7, size=(900, 3)), axis=0)
    before = _outstanding()
    P.inject_alloc_failure(0)
    with pytest.raises(P.Mr1lError) as e:
        P.plan_search(J, seed=5)
    assert e.value.code == P.MR1L_E_NOMEM
    P.inject_alloc_failure(-1)
    assert _outstanding() == before
    pl = P.plan_search(J, seed=5)
    y = torch.from_numpy(rng.standard_normal((3, pl.sum_M)) + 1j * rng.standard_normal((3, pl.sum_M))).cuda()
    P.inject_alloc_failure(0)   # the transform's scratch grows for three right-hand sides
    with pytest.raises(P.Mr1lError) as e:
        pl.reconstruct(y)
    assert e.value.code == P.MR1L_E_NOMEM
    P.inject_alloc_failure(-1)
    got = pl.reconstruct(y).cpu().numpy()
    ml = lattice.search(J.astype(np.int64), seed=5, t=3)
    for h in range(3):
        want, _ = lattice.reconstruct(J.astype(np.int64), ml, np.split(y[h].cpu().numpy(), np.cumsum(ml.M)[:-1]))
        assert np.max(np.abs(got[h] - want)) / np.max(np.abs(want)) < 1e-10
