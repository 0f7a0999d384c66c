"""The stored fixed objective targets (tests/golden/dstar_*.txt, written by
tests/golden/make_dstar.py from the FP64 oracle) are well formed: D_best is
the smaller finite long-run objective of JMM and BMM, both runs had nearly
stopped descending, and the workload's initial objective lies far above."""
import math
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

from make_dstar import WORKLOADS, read_dstar  # noqa: E402

import oracle as O  # noqa: E402
from paper_2106_15214_gb300 import inputs  # noqa: E402


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_stored_targets_are_consistent(name):
    d = read_dstar(name)
    assert d is not None, f"tests/golden/dstar_{name}.txt missing"
    assert d["workload"] == name and d["iterations"] == WORKLOADS[name][1]
    finite = [v for v in (d["D_jmm"], d["D_bmm"]) if math.isfinite(v)]
    assert finite and d["D_best"] == min(finite)
    for key in ("rel_jmm", "rel_bmm"):
        assert 0.0 <= d[key] < 1e-4          # monotone (MM) and nearly stationary at the end of the run
    p = getattr(inputs, WORKLOADS[name][0])()
    d0 = O.D_beta(p.V, p.W0 @ p.H0, p.beta)
    assert d0 > d["D_best"] * 1.01
