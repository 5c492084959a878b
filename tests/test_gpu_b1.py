"""The model value of App. B.1 by its interior point method on the GPU.

f^_t(y~) = <b, y~> + max over the model set {alpha (eta Xbar / tr Xbar + V S V^T): eta >= 0,
S >= 0, eta + tr S <= 1} of <C - A*(y~), X> is a linear SDP over that set.  With
usbs_params.model_value_ipm = 1 the library solves it by the App. B.1 IPM (the App. B.2
Newton iteration with the quadratic terms removed) and uses that value in the descent test;
the closed form (the maximum over the set's vertices) is reported beside it.  The two must
agree to the IPM's stopping accuracy, and the iterates must follow the oracle's, whose model
value is the closed form.
"""
import numpy as np
import pytest

from oracle.usbs import USBSOracle
from paper_2312_11801_gb300 import instances as I
from tests.gpu_util import gpu_modules

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    return gpu_modules()


@pytest.mark.parametrize("name,k_c,k_p", [("er120", 8, 0), ("clust200", 8, 0), ("er120", 6, 2)])
def test_b1_ipm_equals_closed_form_along_the_oracle_trajectory(mods, name, k_c, k_p):
    torch, U = mods
    prob = I.maxcut_er(120, 6.0, 3) if name == "er120" else I.clustering_sdp(200, 800, 1)
    ora = USBSOracle(prob, k=k_c, k_p=k_p, ipm_mu_tol=1e-10)   # the same subproblem accuracy
    ora.cold_start()
    with U.usbs_create(prob, precision=0, k_c=k_c, k_p=k_p, model_value_ipm=1, ipm_mu_tol=1e-10,
                       lanczos_restarts=300, lanczos_tol=1e-12) as ctx:
        for t in range(10):
            g = U.usbs_step(ctx)
            o = ora.step()
            # an IPM stopped at mu < 1e-10 has a duality gap of about 2 (k + 2) mu
            assert abs(g["f_hat"] - g["f_hat_closed"]) <= 1e-7 * (1 + abs(g["f_hat_closed"])), (t, g)
            assert g["ipm_iters_b1"] > 0
            assert g["descent"] == int(o["descent"]), t
            for kg, ko in [("f_y", "f_y"), ("cx", "cx"), ("f_hat", "f_hat")]:
                assert abs(g[kg] - o[ko]) <= 1e-6 * (1 + abs(o[ko])), (t, kg, g[kg], o[ko])


@pytest.mark.parametrize("precision", [0, 1])
def test_b1_ipm_solve_reaches_the_bipartite_value(mods, precision):
    """A whole solve with the IPM model value reaches |E| on the bipartite torus."""
    torch, U = mods
    prob = I.maxcut_torus(8, signed=False)
    with U.usbs_create(prob, precision=precision, model_value_ipm=1, rho=0.1, max_iters=2000,
                       lanczos_restarts=50) as ctx:
        res = U.usbs_solve(ctx, tol=1e-4)
    last = res["last"]
    e = 2.0 * prob.n
    assert res["converged"], res
    assert abs(last["objective"] - e) <= 1e-3 * e and last["dual_bound"] >= e * (1 - 1e-5)
