"""Pins for oracle/ipm.py: the App. B.2 IPM and the App. B.1 model value."""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import ipm as P
from oracle.svec import svec, smat, svec_dim


def _data(k, seed, scale=1.0, m=40):
    rng = np.random.default_rng(seed)
    K = svec_dim(k)
    G = rng.standard_normal((m, K + 1)) * scale
    Qfull = G.T @ G
    Q11, q12, q22 = Qfull[:K, :K], Qfull[:K, K], float(Qfull[K, K])
    h1 = rng.standard_normal(K) * 3 * scale
    h2 = float(rng.standard_normal()) * 3 * scale
    return Q11, q12, q22, h1, h2


def _reference_min(Q11, q12, q22, h1, h2, k, has_eta=True, starts=12, seed=0):
    """Same program solved by SLSQP over S = L L^T (independent method)."""
    rng = np.random.default_rng(seed)
    tri = np.tril_indices(k)
    nL = len(tri[0])

    def unpack(x):
        L = np.zeros((k, k)); L[tri] = x[:nL]
        return L @ L.T, (x[nL] if has_eta else 0.0)

    def obj(x):
        S, eta = unpack(x)
        return P.quad_objective(Q11, q12, q22, h1, h2, S, eta)

    cons = [{"type": "ineq", "fun": lambda x: 1.0 - np.trace(unpack(x)[0]) - unpack(x)[1]}]
    bounds = [(None, None)] * nL + ([(0.0, 1.0)] if has_eta else [])
    best = np.inf
    for _ in range(starts):
        x0 = rng.standard_normal(nL + (1 if has_eta else 0)) * 0.3
        if has_eta:
            x0[-1] = abs(x0[-1])
        r = so.minimize(obj, x0, method="SLSQP", bounds=bounds, constraints=cons,
                        options={"ftol": 1e-14, "maxiter": 2000})
        if r.success or r.status == 8:
            S, eta = unpack(r.x)
            if 1.0 - np.trace(S) - eta >= -1e-9:
                best = min(best, r.fun)
    return best


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (2, 2), (3, 3)])
@pytest.mark.parametrize("has_eta", [True, False])
def test_ipm_quad_matches_independent_solver(k, seed, has_eta):
    Q11, q12, q22, h1, h2 = _data(k, seed)
    sol = P.ipm_quad(Q11, q12, q22, h1, h2, k, has_eta=has_eta, mu_tol=1e-10)
    val = P.quad_objective(Q11, q12, q22, h1, h2, sol["S"], sol["eta"])
    ref = _reference_min(Q11, q12, q22, h1, h2, k, has_eta)
    assert abs(val - ref) <= 1e-6 * (1 + abs(ref)), (val, ref)
    # strict feasibility of the returned point
    assert np.linalg.eigvalsh(sol["S"]).min() > 0
    assert 1 - np.trace(sol["S"]) - sol["eta"] > 0


def test_ipm_kkt_and_central_path_identities():
    """At exit the first-order conditions of eq. linearized_system2 hold up to mu, and
    the three complementarity products of eq. barrier_param_est are all O(mu)."""
    k = 3
    Q11, q12, q22, h1, h2 = _data(k, 7)
    sol = P.ipm_quad(Q11, q12, q22, h1, h2, k, mu_tol=1e-9)
    S, T, eta, zeta, omega = sol["S"], sol["T"], sol["eta"], sol["zeta"], sol["omega"]
    v = svec(np.eye(k))
    F1 = Q11 @ svec(S) + eta * q12 + h1 - svec(T) + omega * v
    F2 = q12 @ svec(S) + eta * q22 + h2 - zeta + omega
    scale = np.abs(Q11).max() + np.abs(h1).max()
    assert np.linalg.norm(F1) <= 1e-6 * scale
    assert abs(F2) <= 1e-6 * scale
    slack = 1 - np.trace(S) - eta
    prods = [np.sum(S * T) / k, eta * zeta, omega * slack]
    assert all(0 < p_ <= 50 * sol["mu"] + 1e-12 for p_ in prods), (prods, sol["mu"])
    assert np.linalg.eigvalsh(T).min() > 0


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("has_eta", [True, False])
def test_model_value_ipm_b1_equals_closed_form(seed, has_eta):
    """App. B.1 solved by the IPM equals the vertex formula of the model value."""
    rng = np.random.default_rng(seed)
    k, alpha = 4, 2.0
    Z = rng.standard_normal((k, k)); Z = (Z + Z.T) / 2
    if seed % 3 == 0:
        Z -= 5 * np.eye(k)           # all candidates negative: maximum at X = 0
    xbar_term = float(rng.standard_normal())
    bdy = float(rng.standard_normal())
    closed = P.model_value_closed_form(bdy, alpha, Z, has_eta, xbar_term)
    g1 = -alpha * svec(Z)
    g2 = -alpha * xbar_term
    sol = P.ipm_linear(g1, g2, k, has_eta=has_eta, mu_tol=1e-11)
    via_ipm = bdy - (g1 @ svec(sol["S"]) + sol["eta"] * g2)
    assert abs(via_ipm - closed) <= 1e-8 * (1 + abs(closed))
