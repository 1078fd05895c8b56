"""The planted sampler's measurement noise (Section 5.2) on the GPU against
the oracle's Philox4x32-10 + Box-Muller draws, value by value."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
from oracle import lattice, sfft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()


@pytest.mark.parametrize("seed,t,rep", [(1, 2, 0), (77, 9, 4), (2**40 + 3, 25, 9)])
def test_lattice_noise_matches_oracle(seed, t, rep):
    M = [130003, 130021, 7, 2]
    got = P.lattice_noise(seed, t, rep, M, 1.7).cpu().numpy()
    ml = lattice.MultiLattice(M, [np.zeros(1)] * len(M), [], True, 1)
    want = np.concatenate(sfft.lattice_noise(seed, t, rep, ml, 1.7))
    # shared node 0
    offs = np.concatenate([[0], np.cumsum(M)[:-1]])
    assert np.all(got[offs] == got[0])
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-3)
    assert err.max() < 1e-13, err.max()
    # the moments of the complex Gaussian: E|eta|^2 = sigma^2
    assert abs(np.mean(np.abs(got) ** 2) / 1.7**2 - 1.0) < 0.02
