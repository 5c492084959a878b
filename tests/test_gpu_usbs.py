"""USBS iterations and solves through the C ABI against the FP64 oracle and closed forms."""
import json
import math
import os

import numpy as np
import pytest

from oracle.usbs import USBSOracle
from paper_2312_11801_gb300 import instances as I
from tests._graphs import named_graph
from tests.gpu_util import gpu_modules

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def mods():
    return gpu_modules()


def _golden():
    return json.load(open(os.path.join(HERE, "golden", "oracle_solves.json")))


def test_step_trajectory_matches_oracle_fp64(mods):
    """Per-iteration f(y), <C,X>, tr X, lambda_max and descent flags of Algorithm 1."""
    torch, U = mods
    prob = I.maxcut_er(120, 6.0, 3)
    ora = USBSOracle(prob, k=8)
    ora.cold_start()
    with U.usbs_create(prob, precision=0, lanczos_restarts=300, lanczos_tol=1e-12) as ctx:
        for t in range(12):
            g = U.usbs_step(ctx)
            o = ora.step()
            assert g["descent"] == int(o["descent"]), t
            for key_g, key_o in [("f_y", "f_y"), ("cx", "cx"), ("trx", "trX"),
                                 ("lambda_max", "lambda_max"), ("f_hat", "f_hat")]:
                assert abs(g[key_g] - o[key_o]) <= 1e-6 * (1 + abs(o[key_o])), (t, key_g, g[key_g], o[key_o])


def test_step_trajectory_with_inequalities_fp64(mods):
    """Alternating maximisation (I not empty): same iterates as the oracle."""
    torch, U = mods
    prob = I.clustering_sdp(200, 800, 1)
    ora = USBSOracle(prob, k=8)
    ora.cold_start()
    with U.usbs_create(prob, precision=0, lanczos_restarts=300, lanczos_tol=1e-12) as ctx:
        for t in range(6):
            g = U.usbs_step(ctx)
            o = ora.step()
            assert g["n_alt"] == o["n_alt"], t
            assert g["descent"] == int(o["descent"]), t
            for key_g, key_o in [("f_y", "f_y"), ("cx", "cx"), ("trx", "trX"), ("relinf", "relinf")]:
                assert abs(g[key_g] - o[key_o]) <= 1e-6 * (1 + abs(o[key_o])), (t, key_g, g[key_g], o[key_o])


_GOLDEN_PROBLEMS = {
    "er800_d6_s0": lambda: I.maxcut_er(800, 6.0, 0),
    "er120_d6_s3": lambda: I.maxcut_er(120, 6.0, 3),
    "rgg400_d10_s5": lambda: I.maxcut_rgg(400, 10.0, seed=5),
    "clust200_e800_s1": lambda: I.clustering_sdp(200, 800, 1),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(_GOLDEN_PROBLEMS))
def test_solve_matches_oracle(mods, name, precision):
    """A GPU solve to both gates <= 1e-3 against a long FP64 oracle solve of the same
    problem (rho = 0.1, up to 5000 iterations).  Every dual value f(y) bounds the optimum
    from above (App. E) and a near-feasible primal value approaches it from below, so
    each side's dual bound must lie above the other side's primal value, and the two
    primal values must agree within the sum of the two gaps (scaled units, 1 + |.|)."""
    torch, U = mods
    gold = _golden()[name]
    prob = _GOLDEN_PROBLEMS[name]()
    with U.usbs_create(prob, precision=precision, rho=gold["rho"], max_iters=3000) as ctx:
        res = U.usbs_solve(ctx, tol=1e-3)
    last = res["last"]
    assert res["converged"], (res["iters"], last["relgap"], last["relinf"])
    assert last["relgap"] <= 1e-3 and last["relinf"] <= 1e-3
    cx, f = last["cx"], last["f_y"]
    cx_o, f_o = gold["cx_scaled"], gold["f_scaled"]
    slack_g = 1e-3 * (1 + abs(cx))
    slack_o = max(gold["relgap"], gold["relinf"]) * (1 + abs(cx_o))
    assert f >= cx_o - slack_o - slack_g, (f, cx_o)
    assert f_o >= cx - slack_g - slack_o, (f_o, cx)
    assert abs(cx - cx_o) <= 2 * (slack_g + slack_o), (cx, cx_o)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,value", [
    ("K32", 32 * 32 / 4), ("C33", 16.5 * (1 + math.cos(math.pi / 33))), ("torus8", 128.0)])
def test_closed_form_maxcut(mods, name, value, precision):
    torch, U = mods
    if name == "torus8":
        prob = I.maxcut_torus(8, signed=False)       # bipartite: SDP = |E| = 128
    else:
        n, i, j, w = named_graph(name)
        prob = I.maxcut_from_edges(n, i, j, w, name=name)
    with U.usbs_create(prob, precision=precision, max_iters=3000, rho=0.1,
                       ipm_mu_tol=1e-10, lanczos_restarts=50) as ctx:
        res = U.usbs_solve(ctx, tol=1e-5)
    last = res["last"]
    slack = 1.01 * max(last["relgap"], 1e-5) * (1 + abs(last["cx"])) * prob.n * 1.0
    c_scale = float(np.sqrt(np.sum(prob.C_val ** 2)))
    slack *= c_scale
    assert last["dual_bound"] >= value * (1 - (1e-9 if precision == 0 else 1e-5))
    assert abs(last["objective"] - value) <= max(slack, 2e-4 * value), (last, value)
