"""Host-side pieces of bench.py that need no GPU: the serving request stream."""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2312_11801_gb300 import instances as I  # noqa: E402


def test_serve_requests_structure():
    reqs = bench.serve_requests(I, 40, 100, 2000, seed=3)
    assert [q["id"] for q in reqs] == list(range(40))
    grown = [q for q in reqs if q["parent"] >= 0]
    assert 10 <= len(grown) <= 30 and reqs[0]["parent"] == -1
    for q in grown:
        parent = reqs[q["parent"]]
        assert q["parent"] < q["id"]
        n0 = parent["prob"].n
        assert q["prob"].n == n0 + max(1, math.ceil(0.01 * n0))
        # the parent's vertices keep their indices and edges (warm-start setting)
        pc, cc = parent["prob"], q["prob"]
        for i in range(0, n0, max(1, n0 // 7)):
            old = set(pc.C_col[pc.C_rowptr[i]:pc.C_rowptr[i + 1]].tolist()) - {i}
            new = set(cc.C_col[cc.C_rowptr[i]:cc.C_rowptr[i + 1]].tolist()) - {i}
            assert old <= new
    fresh = [q["prob"].n for q in reqs if q["parent"] < 0]
    assert min(fresh) >= 100 and max(fresh) <= 2000


def test_percentile_helper():
    assert bench._pct([], 50) is None
    assert bench._pct([1.0, 2.0, 3.0], 50) == 2.0
    assert abs(bench._pct(list(np.arange(101.0)), 99) - 99.0) < 1e-12
