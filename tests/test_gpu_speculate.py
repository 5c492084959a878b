"""Speculative Lanczos cycles: a cycle first runs without the masked deflation passes of its
blocks and runs again with them when a first pass met a deficient column.  The results must
equal, bit for bit, those of cycles that always run the masked passes (USBS_NO_SPECULATE=1)."""
import os

import numpy as np
import pytest

from paper_2312_11801_gb300 import instances as I
from tests._graphs import named_problem
from tests.gpu_util import gpu_modules

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    return gpu_modules()


def _run(U, prob, precision, speculate, steps):
    if speculate:
        os.environ.pop("USBS_NO_SPECULATE", None)
    else:
        os.environ["USBS_NO_SPECULATE"] = "1"
    try:
        with U.usbs_create(prob, precision=precision, lanczos_basis=32, rho=0.1) as ctx:
            out = [U.usbs_step(ctx) for _ in range(steps)]
            w, v, info = U.usbs_extreme_eigs(ctx)
    finally:
        os.environ.pop("USBS_NO_SPECULATE", None)
    return out, w, v, info


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["K64", "er200"])
def test_speculative_cycles_are_exact(mods, case, precision):
    torch, U = mods
    # K64: two distinct eigenvalues, so an 8-column block Krylov space stops growing at 9
    # columns and every cycle meets deficient columns; er200: no deflation after the start
    prob = named_problem("K64") if case == "K64" else I.maxcut_er(200, 6.0, 7)
    s_steps, s_w, s_v, s_info = _run(U, prob, precision, True, 5)
    p_steps, p_w, p_v, p_info = _run(U, prob, precision, False, 5)
    assert p_info["reruns"] == 0
    if case == "K64":
        assert s_info["reruns"] > 0
    for a, b in zip(s_steps, p_steps):
        for key in ("f_y", "cx", "trx", "lambda_max", "relgap", "relinf", "descent", "matvecs"):
            assert a[key] == b[key], (key, a[key], b[key])
    np.testing.assert_array_equal(s_w, p_w)
    np.testing.assert_array_equal(s_v, p_v)
    assert s_info["cycles"] == p_info["cycles"] and s_info["matvecs"] == p_info["matvecs"]
