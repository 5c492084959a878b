"""The synthetic QAP relaxation (App. E, QAP, eq. qap_sdp) built by instances.qap_sdp:
every permutation is a feasible point priced at minus its QAP cost, and the oracle's dual
bound stays above all of them (weak duality)."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.usbs import USBSOracle
from paper_2312_11801_gb300 import instances as I


def _perm_point(nq, perm):
    Pi = np.eye(nq)[list(perm)]                 # Pi[i, perm[i]] = 1
    v = np.concatenate([[1.0], Pi.flatten(order="F")])   # vec stacks columns
    return Pi, np.outer(v, v)


def _A_of(prob, X):
    out = np.zeros(prob.m)
    np.add.at(out, prob.A_con, prob.A_val * X[prob.A_i, prob.A_j])
    return out


@pytest.mark.parametrize("nq,seed", [(4, 0), (5, 1)])
def test_permutations_are_feasible_and_priced(nq, seed):
    prob = I.qap_sdp(nq, seed)
    W, D = prob.meta["W"], prob.meta["D"]
    C = sp.csr_matrix((prob.C_val, prob.C_col, prob.C_rowptr), shape=(prob.n, prob.n)).toarray()
    assert np.allclose(C, C.T)
    eq = prob.is_ineq == 0
    for perm in itertools.permutations(range(nq)):
        Pi, X = _perm_point(nq, perm)
        ax = _A_of(prob, X)
        assert np.allclose(ax[eq], prob.b[eq], atol=1e-12)
        assert np.all(ax[~eq] <= prob.b[~eq] + 1e-12)
        assert abs(np.trace(X) - prob.trace) <= 1e-12
        assert abs(np.sum(C * X) + np.trace(W @ Pi @ D @ Pi.T)) <= 1e-9


def test_oracle_dual_bound_covers_every_permutation():
    """f(y) >= SDP value >= <C, X_Pi> for every permutation and every y in Y: checked at
    each of 60 oracle iterations."""
    nq = 4
    prob = I.qap_sdp(nq, 0)
    W, D = prob.meta["W"], prob.meta["D"]
    best = max(-np.trace(W @ np.eye(nq)[list(p)] @ D @ np.eye(nq)[list(p)].T)
               for p in itertools.permutations(range(nq)))
    o = USBSOracle(prob, k=4, rho=0.1)
    o.cold_start()
    for _ in range(60):
        o.step()
        assert o.dual_bound() >= best - 1e-9 * abs(best)


def test_qap_rounding_recovers_a_permutation_point():
    """App. E rounding: with the sketch of X_Pi itself (a rank-one primal) the top column of
    U is +-[1; vec(Pi)] / |.|, and the Hungarian projection returns Pi at its QAP cost."""
    from oracle.nystrom import nystrom_reconstruct, qap_cost, qap_round
    nq = 5
    prob = I.qap_sdp(nq, 2)
    W, D = prob.meta["W"], prob.meta["D"]
    perm = (3, 0, 4, 1, 2)
    Pi, X = _perm_point(nq, perm)
    psi = np.random.default_rng(5).standard_normal((prob.n, nq))
    U, lam = nystrom_reconstruct(X @ psi, psi)
    cost, k, Pr = qap_round(U[:, :1], W, D)
    np.testing.assert_array_equal(Pr, Pi)
    assert cost == qap_cost(W, D, Pi)
    assert abs(lam[0] - (1 + nq)) <= 1e-9 * (1 + nq)


def test_qap_rounding_never_beats_the_optimum():
    from oracle.nystrom import qap_round
    nq = 5
    prob = I.qap_sdp(nq, 1)
    W, D = prob.meta["W"], prob.meta["D"]
    opt = min(np.trace(W @ np.eye(nq)[list(p)] @ D @ np.eye(nq)[list(p)].T)
              for p in itertools.permutations(range(nq)))
    U = np.linalg.qr(np.random.default_rng(6).standard_normal((prob.n, 6)))[0]
    cost, _, Pi = qap_round(U, W, D)
    assert np.allclose(Pi.sum(0), 1) and np.allclose(Pi.sum(1), 1)
    assert cost >= opt - 1e-9
