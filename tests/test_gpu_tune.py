"""The tile tuner: the first 4-step transform of each (P, mode, arithmetic)
times the candidate tilings and keeps the fastest; every tiling must give the
same output bit for bit, so results with and without tuning are identical."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
from oracle import lattice

pytestmark = pytest.mark.gpu

CANDS = {1024, 2048, 4096}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()
    yield
    P.tune_enable(True)


@pytest.mark.parametrize("fft", ["f64", "df"])
@pytest.mark.parametrize("M,width", [(3001, 1000), (130003, 20000), (1_300_021, 20000)])
def test_tuned_tiles_give_identical_bits(fft, M, width):
    """Bluestein lengths 3 * 2^11 (P1 = 96: the row tile must divide it),
    2^18 and 3 * 2^20: default tiles (tuning off) against the trial run
    (whose output comes from the last candidate tiling) and against the
    cached choice."""
    I = np.arange(-width, width).reshape(-1, 1)
    z = 7919 if M > 7919 else 1723
    rng = np.random.default_rng(M)
    y = torch.from_numpy(rng.standard_normal((2, M)) + 1j * rng.standard_normal((2, M))).cuda()
    c = torch.from_numpy(rng.standard_normal((2, I.shape[0])) + 1j * rng.standard_normal((2, I.shape[0]))).cuda()

    P.tune_reset()
    P.tune_enable(False)
    pl = P.plan(I, [M], [[z]], fft=fft)
    a = pl.reconstruct(y).cpu().numpy()
    ae = pl.evaluate(c, P.MR1L_EVAL).cpu().numpy()
    assert P.tune_read() == []

    P.tune_enable(True)
    pl2 = P.plan(I, [M], [[z]], fft=fft)
    b = pl2.reconstruct(y).cpu().numpy()
    be = pl2.evaluate(c, P.MR1L_EVAL).cpu().numpy()
    cc = pl2.reconstruct(y).cpu().numpy()
    ce = pl2.evaluate(c, P.MR1L_EVAL).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, cc)
    np.testing.assert_array_equal(ae, be)
    np.testing.assert_array_equal(ae, ce)

    table = P.tune_read()
    modes = {(e["P"], e["mode"], e["df"]) for e in table}
    Pn = {3001: 3 * 2**11, 130003: 2**18, 1_300_021: 3 * 2**20}[M]
    df = int(fft == "df")
    assert {(Pn, "filter", df), (Pn, "recon", df), (Pn, "eval", df)} <= modes
    for e in table:
        assert e["col_tile"] in CANDS and e["row_tile"] in CANDS
        assert e["col_ms"] > 0 and e["row_ms"] > 0

    # and the tuned transform still matches the oracle
    ml = lattice.MultiLattice([M], [np.array([z])], [lattice.unique_mask(I, [z], M)], True, 1)
    want, _ = lattice.reconstruct(I, ml, [y[0].cpu().numpy()], "fft")
    assert np.max(np.abs(b[0] - want)) / np.max(np.abs(want)) < 1e-10


def test_forced_tiles_from_the_environment(tmp_path):
    """MR1L_TILES fixes the tiles (read once per process): a child process
    with forced 4096-element column and 1024-element row tiles gives the same
    bits as this process."""
    import subprocess
    import sys
    M = 1_300_021
    I = np.arange(-20000, 20000).reshape(-1, 1)
    rng = np.random.default_rng(5)
    y = rng.standard_normal((1, M)) + 1j * rng.standard_normal((1, M))
    np.save(tmp_path / "y.npy", y)
    pl = P.plan(I, [M], [[7919]])
    want = pl.reconstruct(torch.from_numpy(y).cuda()).cpu().numpy()
    code = (
        "import numpy as np, torch, paper_1711_05152_gb300 as P\n"
        f"y = np.load(r'{tmp_path / 'y.npy'}')\n"
        "I = np.arange(-20000, 20000).reshape(-1, 1)\n"
        f"pl = P.plan(I, [{M}], [[7919]])\n"
        "np.save(r'%s', pl.reconstruct(torch.from_numpy(y).cuda()).cpu().numpy())\n"
        "assert P.tune_read() == []\n" % (tmp_path / "got.npy"))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MR1L_TILES="4096,1024", PYTHONPATH=root)
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=root, timeout=300)
    np.testing.assert_array_equal(np.load(tmp_path / "got.npy"), want)
