"""bench.py's host-side helpers (no GPU): the Section 5.3 L2 error it reports
for Table 5.7 against the oracle's evaluator, and the paper fixtures it reads."""

import importlib.util
import os
import sys

import numpy as np

import workloads as W
from oracle import bspline as B
from oracle import sfft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    # registered under its own name, so that spawned workers can import it
    if "bench" in sys.modules:
        return sys.modules["bench"]
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules["bench"] = mod
    spec.loader.exec_module(mod)
    return mod


def test_l2_error_matches_the_oracle():
    bench = _bench()
    desc = W.bspline_function(4, 8, [[0, 2], [1, 3]], [4, 6])
    ref = sfft.sfft(B.signal(desc), 60, 120, 3, 10, 1e-12, "abs", seed=5)
    got = bench._bspline_l2_error(desc, ref)
    want = B.signal(desc).rel_l2_error(ref.freqs, ref.coeffs)
    assert abs(got - want) < 1e-14 * max(want, 1.0)
    empty = type("R", (), {"freqs": np.zeros((0, 4), dtype=np.int64), "coeffs": np.zeros(0)})()
    assert abs(bench._bspline_l2_error(desc, empty) - 1.0) < 1e-15


def test_paper_fixtures_parse():
    bench = _bench()
    t51 = bench._paper_rows("paper_table_5_1.txt")
    assert len(t51) == 18 and t51[0][:3] == [5.0, 1000.0, 4525799.0]
    assert len(bench._paper_rows("paper_table_5_2.txt")) == 15
    assert len(bench._paper_rows("paper_table_5_4.txt")) == 18
    t57 = bench._paper_rows("paper_table_5_7.txt")
    assert len(t57) == 13 and t57[-1][:3] == [64.0, 10000.0, 2639274025.0]


def test_all_cores_oracle_leg_runs():
    """The all-cores CPU leg (spawned single-threaded oracle processes, one
    signal each) on the d = 3 workload with two processes: every process
    finishes, and the rate is scaled by the timed job's coefficients per
    sample."""
    bench = _bench()
    sig, p = W.workload("tiny_d3", 1)
    ref = sfft.sfft(sig, p["s"], p["s_local"], p["r"], p["b"], p["theta"], p["theta_mode"], seed=1)
    wl = type("WL", (), {"seeds": [1]})()
    out = bench.oracle_sample_all_cores("tiny_d3", wl, [ref], cores=2, t_stop=3)
    assert out["cores"] == 2 and out["kind"] == "oracle" and out["value"] > 0
    assert "seeds 1..2" in out["sample"]
