"""The C ABI library loads and exports every entry point its header declares,
and rejects invalid arguments on the host (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

import paper_1711_05152_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(P.LIB_PATH):
        from paper_1711_05152_gb300 import build
        build.build()
    return P.lib()


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|long long)\s+(\w+)\s*\(", src, flags=re.M)
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "mr1l_reconstruct" in names and "sfft_dimincr" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    for n in P.EXPORTS:
        assert n in names


def test_version(lib):
    assert lib.mr1l_version() >= 100


@pytest.mark.parametrize("I,M,z,msg", [
    ([[0], [0]], [5], [[1]], "distinct"),
    ([[0], [1]], [6], [[1]], "prime"),
    ([[0], [1]], [5], [[5]], "z_l"),
    ([[0], [1]], [5, 5], [[1], [2]], "distinct"),
    ([[40000], [1]], [5], [[1]], "2^15"),
])
def test_plan_rejects_invalid(lib, I, M, z, msg):
    with pytest.raises(P.Mr1lError) as e:
        P.plan(np.array(I), M, z, stream=0)
    assert e.value.code == P.MR1L_E_INVAL
    assert msg in str(e.value)


def test_sfft_rejects_invalid(lib):
    with pytest.raises(P.Mr1lError) as e:
        P.sfft_dimincr(1, 4, 3, 1, 1e-12, freqs=np.zeros((1, 1)), coeffs=[1.0], stream=0)
    assert e.value.code == P.MR1L_E_INVAL
    with pytest.raises(P.Mr1lError) as e:
        P.sfft_dimincr(3, 5000, 3, 1, 1e-12, freqs=np.zeros((1, 3)), coeffs=[1.0], stream=0)
    assert e.value.code == P.MR1L_E_INVAL


def test_null_plan_is_rejected(lib):
    rc = lib.mr1l_reconstruct(None, None, 1, None, None)
    assert rc == P.MR1L_E_INVAL
    buf = ctypes.create_string_buffer(256)
    assert lib.mr1l_last_error(buf, 256) == P.MR1L_E_INVAL
    assert b"plan is null" in buf.value


def test_tile_tuner_host_controls(lib):
    P.tune_reset()
    assert P.tune_read() == []
    P.tune_enable(False)
    P.tune_enable(True)
    assert lib.mr1l_tune_read(None, 0) == P.MR1L_E_INVAL


@pytest.mark.parametrize("groups,orders,msg", [
    ([[0, 1]], [9], "orders"),
    ([[0, 1]], [1], "orders"),
])
def test_bspline_sampler_rejects_invalid(lib, groups, orders, msg):
    import workloads as W
    f = W.bspline_function(3, 4, groups, orders)
    with pytest.raises(P.Mr1lError) as e:
        P.sfft_dimincr(3, 4, 10, 1, 1e-12, "abs", function=f, stream=0)
    assert e.value.code == P.MR1L_E_INVAL and msg in str(e.value)


def test_theorem_params(lib):
    """The theorem of Section 4: r = ceil(2 supp (ln 3 + ln d + ln supp - ln eps)),
    b = ceil((ln 3 + ln d - ln eps) / ln 2); d = 5, supp = 1000, eps = 0.01 by hand:
    ln 3 + ln 5 + ln 1000 - ln 0.01 = ln(1.5e6) = 14.2209..., so r = 28442;
    ln 3 + ln 5 - ln 0.01 = ln 1500 = 7.3132..., / ln 2 = 10.55, so b = 11."""
    assert P.theorem_params(5, 1000, 0.01) == (28442, 11)
    r1, b1 = P.theorem_params(10, 1000, 0.01)
    r2, b2 = P.theorem_params(10, 1000, 0.001)
    assert r2 > r1 and b2 >= b1
    with pytest.raises(P.Mr1lError):
        P.theorem_params(5, 1000, 1.5)


def test_output_tensor_checks():
    """Output tensors written through raw pointers are refused unless they
    have exactly the expected shape, dtype and device (checked on the host,
    before any launch)."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cpu")
    P.check_out(torch.empty((2, 5), dtype=torch.complex128), (2, 5), dev)
    with pytest.raises(ValueError, match="shape"):
        P.check_out(torch.empty((2, 4), dtype=torch.complex128), (2, 5), dev)
    with pytest.raises(ValueError, match="shape"):
        P.check_out(torch.empty((1, 5), dtype=torch.complex128), (2, 5), dev)
    with pytest.raises(TypeError):
        P.check_out(torch.empty((2, 5), dtype=torch.complex64), (2, 5), dev)
    with pytest.raises(TypeError):
        P.check_out(torch.empty((5, 2), dtype=torch.complex128).t(), (2, 5), dev)
    with pytest.raises(ValueError, match="expected cuda"):
        P.check_out(torch.empty((2, 5), dtype=torch.complex128), (2, 5), torch.device("cuda", 0))


def test_pool_stats_and_injection_controls(lib):
    """The block-cache counters and the allocation-failure injector are host
    calls: they work without a GPU."""
    st = P.pool_stats(63)
    assert st == {"outstanding": 0, "cached": 0, "mallocs": 0}
    P.inject_alloc_failure(5)
    P.inject_alloc_failure(-1)
    with pytest.raises(P.Mr1lError):
        P.inject_alloc_failure(-2)
    with pytest.raises(P.Mr1lError):
        P.pool_stats(-1)
