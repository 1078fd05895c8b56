"""The thresholded "(up to) s-largest" selection of Algorithm 3 (steps 1, 2a
and 2e) through the C ABI (sfft_select) against the oracle's selection, on
values built so that keys tie exactly: equal keys at the cut (the smaller
index wins), keys exactly at the threshold (kept: the comparison is >=),
all keys equal, caps above the eligible count, indices no lattice covers.
Both kernels are covered: segments of at most 65536 values (one CTA per
segment) and longer ones (the multi-CTA digit passes)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
from oracle import sfft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()


def _check(p: np.ndarray, cap: int, theta: float, mode: str, eligible=None):
    """GPU union of the per-row selections == the oracle's, bit for bit."""
    p = np.atleast_2d(p)
    want = np.zeros(p.shape[1], dtype=bool)
    for row in p:
        sel = sfft.select(row, cap, theta, mode, eligible)
        want[sel.chosen] = True
    el = None if eligible is None else torch.from_numpy(eligible.astype(np.uint8)).cuda()
    got = P.select(torch.from_numpy(np.ascontiguousarray(p)).cuda(), cap, theta, mode, eligible=el)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy().astype(bool), want)
    return want


SIZES = [1, 37, 4096, 65536, 65537, 200003]


@pytest.mark.parametrize("n", SIZES)
def test_ties_at_the_cut(n):
    """Integer values: many keys equal, the cut falls inside a class of equal
    keys, so the smaller indices of that class must be taken."""
    rng = np.random.default_rng(n)
    p = (rng.integers(-3, 4, size=(3, n)) + 1j * rng.integers(-3, 4, size=(3, n))).astype(np.complex128)
    for cap in (1, max(1, n // 7), max(1, n // 2), n, n + 5):
        want = _check(p, cap, 0.0, "abs")
        if cap < n:
            assert want.sum() >= min(cap, n)


@pytest.mark.parametrize("n", SIZES)
def test_all_keys_equal(n):
    p = np.full((2, n), 3 - 4j, dtype=np.complex128)
    for cap in (1, 2, max(1, n // 3), n):
        want = _check(p, cap, 1e-12, "rel")
        assert want.sum() == min(cap, n) and want[:min(cap, n)].all()


@pytest.mark.parametrize("n", SIZES)
def test_keys_exactly_at_the_threshold(n):
    """|p|^2 = 25 exactly at an absolute theta = 5 and at a relative theta =
    1/2 with max key 100: those keys are kept, 24 is not."""
    rng = np.random.default_rng(n + 1)
    vals = np.array([5 + 0j, 3 + 4j, 4 - 3j, 4 + 2.8284271247461903j, 10 + 0j, 1 + 1j])
    p = rng.choice(vals, size=(2, n)).astype(np.complex128)
    p[:, 0] = 10.0  # max key 100 in every row
    for cap in (n, max(1, n // 4)):
        _check(p, cap, 5.0, "abs")
        _check(p, cap, 0.5, "rel")


@pytest.mark.parametrize("n", [50, 65536, 100000])
def test_ineligible_and_cap_above_count(n):
    rng = np.random.default_rng(n + 2)
    p = (rng.standard_normal((4, n)) + 1j * rng.standard_normal((4, n))).astype(np.complex128)
    eligible = rng.random(n) < 0.3
    for cap in (1, int(eligible.sum()) // 2 + 1, int(eligible.sum()), n):
        want = _check(p, cap, 1e-12, "rel", eligible)
        assert not want[~eligible].any()
    # a relative threshold that leaves fewer keys than the cap
    _check(p, n, 0.9, "rel", eligible)


def test_cap_zero_and_empty():
    p = torch.ones((2, 10), dtype=torch.complex128, device="cuda")
    assert int(P.select(p, 0, 0.0, "abs").sum()) == 0
    flags = torch.zeros(10, dtype=torch.uint8, device="cuda")
    flags[3] = 1
    P.select(p, 2, 0.0, "abs", flags=flags)   # OR-ed into the given flags
    assert flags.cpu().tolist() == [1, 1, 0, 1, 0, 0, 0, 0, 0, 0]
