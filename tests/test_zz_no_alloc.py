"""mr1l_reconstruct_noalloc: Algorithm 2 for callers that cannot allocate
device memory while they run (their device memory is owned by another
allocator or budget, or they cannot afford the synchronisation an allocation
may cause).  Its result must equal mr1l_reconstruct's; it is called twice in
a row with different inputs, since every call reuses the same fixed scratch."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def test_reconstruct_noalloc_matches_reconstruct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = P.lib()
    rng = np.random.default_rng(21)
    J = np.unique(rng.integers(-8, 9, size=(4000, 4)), axis=0)[:3000]
    pl = P.plan_search(J, seed=22)
    stream = torch.cuda.current_stream().cuda_stream
    nrhs = 2
    for call in range(2):
        y = torch.from_numpy(rng.standard_normal((nrhs, pl.sum_M)) + 1j * rng.standard_normal((nrhs, pl.sum_M)))
        y = y.cuda()
        want = pl.reconstruct(y)
        got = torch.full_like(want, complex(np.nan, np.nan))
        rc = lib.mr1l_reconstruct_noalloc(pl._h, ctypes.c_void_p(y.data_ptr()), nrhs,
                                          ctypes.c_void_p(got.data_ptr()), ctypes.c_void_p(stream))
        assert rc == P.MR1L_OK
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.max(np.abs(g - w)) / np.max(np.abs(w)) < RTOL, f"call {call}"


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
