"""The failure path of the library's bounded device-side waits, without a GPU fault.

Every wait of a staged Gram-Schmidt tile on its bulk copies is bounded: when it runs out
the kernel records USBS_ETIMEOUT, waits (bounded) for copies still in flight, releases its
barriers and returns.  usbs_selftest_tile_wait runs that wait alone: with no copy issued
(a barrier that nothing completes) it must report USBS_ETIMEOUT; the device must stay usable,
so a second call that delivers the copy, and then an eigen solve, run clean.
"""
import time

import numpy as np
import pytest

from paper_2312_11801_gb300 import instances as I
from tests.gpu_util import gpu_modules

pytestmark = pytest.mark.gpu


def test_tile_wait_runs_out_and_the_device_stays_usable():
    torch, U = gpu_modules()
    t0 = time.perf_counter()
    rc = U.usbs_selftest_tile_wait(0)
    waited = time.perf_counter() - t0
    assert rc == U.USBS_ETIMEOUT, rc
    assert waited < 30.0, waited              # bounded: two waits of about 0.1 s each
    assert U.usbs_selftest_tile_wait(1) == U.USBS_OK
    prob = I.maxcut_er(300, 6.0, 1)
    with U.usbs_create(prob, precision=1) as ctx:
        evals, _, info = U.usbs_extreme_eigs(ctx, want_vecs=False)
    assert np.all(np.isfinite(evals)) and info["cycles"] >= 1
