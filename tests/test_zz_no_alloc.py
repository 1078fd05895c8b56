"""mr1l_reconstruct_noalloc: Algorithm 2 for callers that cannot allocate
device memory while they run (their device memory is owned by another
allocator or budget, or they cannot afford the synchronisation an allocation
may cause).  Its result must equal mr1l_reconstruct's (and the CPU oracle's);
it is called twice in a row with different inputs, since every call reuses
the same fixed scratch, and the second call must take no device memory."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
from oracle import lattice

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def test_reconstruct_noalloc_matches_reconstruct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = P.lib()
    rng = np.random.default_rng(21)
    J = np.unique(rng.integers(-8, 9, size=(4000, 4)), axis=0)[:3000]
    pl = P.plan_search(J, seed=22)
    ml = lattice.search(J.astype(np.int64), seed=22, t=J.shape[1])
    assert list(pl.M) == ml.M
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream().cuda_stream
    nrhs = 2
    for call in range(2):
        y = torch.from_numpy(rng.standard_normal((nrhs, pl.sum_M)) + 1j * rng.standard_normal((nrhs, pl.sum_M)))
        y = y.cuda()
        want = pl.reconstruct(y)
        got = torch.full_like(want, complex(np.nan, np.nan))
        torch.cuda.synchronize()
        pool0, free0 = P.pool_stats(dev), torch.cuda.mem_get_info()[0]
        rc = lib.mr1l_reconstruct_noalloc(pl._h, ctypes.c_void_p(y.data_ptr()), nrhs,
                                          ctypes.c_void_p(got.data_ptr()), ctypes.c_void_p(stream))
        assert rc == P.MR1L_OK
        torch.cuda.synchronize()
        if call == 1:
            # the first call may load the library's device code and commit the
            # fixed array; from then on a call takes no device memory at all
            assert P.pool_stats(dev) == pool0
            assert torch.cuda.mem_get_info()[0] == free0
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.max(np.abs(g - w)) / np.max(np.abs(w)) < RTOL, f"call {call}"
        # and against the CPU oracle's Algorithm 2 on the first right-hand side
        ref, _ = lattice.reconstruct(J.astype(np.int64), ml, np.split(y[0].cpu().numpy(), np.cumsum(ml.M)[:-1]))
        assert np.max(np.abs(g[0] - ref)) / np.max(np.abs(ref)) < RTOL, f"call {call} against the oracle"


def test_reconstruct_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(23)
    J = np.unique(rng.integers(-20, 21, size=(40000, 3)), axis=0)[:30000]
    pl = P.plan_search(J, seed=24)
    y = torch.zeros((8, pl.sum_M), dtype=torch.complex128, device="cuda")
    out = torch.zeros((8, pl.nI), dtype=torch.complex128, device="cuda")
    with pytest.raises(P.Mr1lError) as e:
        pl.reconstruct_noalloc(y, out)
    assert e.value.code == P.MR1L_E_INVAL
    assert "fixed maximum" in str(e.value)
