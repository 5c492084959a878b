"""Pins for oracle/usbs.py (Algorithm 1, Sec. 4, App. C, App. E) by closed forms,
brute force, certificates and the invariants the paper states."""
import math

import numpy as np
import pytest

from oracle import usbs as U
from oracle.svec import svec
from paper_2312_11801_gb300 import instances as I
from tests._graphs import brute_force_maxcut, load_sdp_values, named_graph, named_problem

PINS = ["K4", "K5", "K6", "C5", "C7", "C8", "K3,3", "K2,4", "petersen", "Q3"]


@pytest.mark.parametrize("name", PINS)
def test_maxcut_closed_forms(name, golden_dir):
    n, val = load_sdp_values(f"{golden_dir}/maxcut_sdp_values.txt")[name]
    o = U.USBSOracle(named_problem(name), k=8)
    o.solve(tol=1e-5, max_iters=300)
    # weak duality: f(y) is an upper bound of the SDP value for every y in Y
    assert o.dual_bound() >= val * (1 - 1e-9)
    assert abs(o.objective() - val) <= 3e-5 * val
    assert abs(o.dual_bound() - val) <= 3e-5 * val


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_cut_below_sdp_below_eigen_bound(seed):
    rng = np.random.default_rng(seed)
    n = 14
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < 0.35
    i, j = iu[keep], ju[keep]
    w = rng.random(len(i)) + 0.1
    prob = I.maxcut_from_edges(n, i, j, w)
    o = U.USBSOracle(prob, k=8, rho=0.1, ipm_mu_tol=1e-10)
    hist = o.solve(tol=1e-5, max_iters=120)
    cut = brute_force_maxcut(n, i, j, w)
    # the gap reached, |f - <C,X>| <= relgap (1 + |<C,X>|) in scaled units, unscaled
    slack = 1.01 * hist[-1]["relgap"] * (1 + abs(o.state.cx)) * o.sp.c_scale * o.sp.tau
    assert hist[-1]["relgap"] <= 1e-4
    L = np.zeros((n, n))
    for a, b_, ww in zip(i, j, w):
        L[a, a] += ww; L[b_, b_] += ww; L[a, b_] -= ww; L[b_, a] -= ww
    eig_bound = n / 4 * np.linalg.eigvalsh(L)[-1]
    assert cut <= o.dual_bound() + 1e-9
    assert cut <= o.objective() + slack
    assert o.dual_bound() <= eig_bound + slack


def _dense_A(prob):
    """Dense A_c from the COO convention, written independently of the oracle."""
    m, n = prob.m, prob.n
    A = np.zeros((m, n, n))
    for c, i, j, v in zip(prob.A_con, prob.A_i, prob.A_j, prob.A_val):
        if i == j:
            A[c, i, i] += v
        else:
            A[c, i, j] += v / 2
            A[c, j, i] += v / 2
    return A


def _tiny_clustering(n=12, e=20, seed=3):
    return I.clustering_sdp(n, e, seed)


def test_clustering_primal_dual_certificate():
    """Equality + inequality SDP: a near-feasible primal and a feasible dual whose
    values agree pin the optimum (no closed form exists for this family)."""
    prob = _tiny_clustering()
    o = U.USBSOracle(prob, k=8, rho=1.0, ipm_mu_tol=1e-10, dense_track=True)
    hist = o.solve(tol=1e-6, max_iters=150)
    assert hist[-1]["relgap"] <= 1e-6 and hist[-1]["relinf"] <= 1e-6
    st, s = o.state, o.sp
    A = _dense_A(prob)
    C = s.C.toarray()
    X = st.Xbar
    AX = np.einsum("cij,ij->c", A, X)
    infeas = np.linalg.norm(AX - np.where(s.ineq, np.minimum(AX, s.b), s.b))
    assert infeas <= 1e-5
    assert np.linalg.eigvalsh(X).min() >= -1e-10
    Z = C - np.einsum("c,cij->ij", st.y, A)
    dual = 2.0 * max(np.linalg.eigvalsh(Z)[-1], 0) + s.b @ st.y
    assert np.all(st.y[s.ineq] >= 0)
    assert abs(dual - np.sum(C * X)) <= 1e-5
    assert abs(dual - st.f_y) <= 1e-9


def _run_invariants(prob, iters, psi=None):
    o = U.USBSOracle(prob, k=6, psi=psi, dense_track=True)
    o.cold_start()
    s = o.sp
    A = _dense_A(prob)
    C = s.C.toarray()
    f_prev = o.state.f_y
    out = []
    for _ in range(iters):
        info = o.step()
        st = o.state
        yc, nu = info["y_cand"], info["nu"]
        # Sec. 3 "Feasibility of the candidate": y_I >= 0 and <y, nu> = 0
        assert np.all(yc[s.ineq] >= 0)
        assert abs(yc @ nu) <= 1e-10 * (1 + np.abs(yc).sum() * np.abs(nu).max())
        # minorant (eq. minorant_cond) and non-negative predicted decrease
        assert info["f_hat"] <= info["f_cand"] + 1e-7
        assert info["f_old"] - info["f_hat"] >= -1e-6
        # implicit primal (App. C) equals the dense recomputation
        X = st.Xbar
        assert abs(st.cx - np.sum(C * X)) <= 1e-12 * (1 + abs(st.cx))
        assert abs(st.tr - np.trace(X)) <= 1e-12
        np.testing.assert_allclose(st.ax, np.einsum("cij,ij->c", A, X), atol=1e-13)
        if psi is not None:
            np.testing.assert_allclose(st.P, X @ psi.astype(np.float64), atol=1e-12)
        # f(y_t) is non-increasing
        assert st.f_y <= f_prev + 1e-15
        f_prev = st.f_y
        out.append(info)
    return out


def test_invariants_clustering_with_inequalities():
    prob = _tiny_clustering(14, 30, 5)
    psi = I.gaussian_psi(prob.n, 4, seed=9)
    hist = _run_invariants(prob, 25, psi)
    assert any(h["n_alt"] > 1 for h in hist)         # the alternation actually ran
    assert any(h["descent"] for h in hist) and any(not h["descent"] for h in hist)


def test_invariants_maxcut():
    prob = I.maxcut_er(30, 5, seed=4)
    _run_invariants(prob, 20, I.gaussian_psi(30, 5, seed=2))


def test_scaling_invariance():
    """Scaling C by a constant scales the optimum by the same constant (App. E scaling)."""
    p1 = named_problem("C5")
    p2 = named_problem("C5")
    p2.C_val = p2.C_val * 7.0
    o1, o2 = U.USBSOracle(p1), U.USBSOracle(p2)
    o1.solve(tol=1e-6, max_iters=50)
    o2.solve(tol=1e-6, max_iters=50)
    assert abs(o2.objective() - 7 * o1.objective()) <= 1e-9 * o2.objective()


def test_warm_start_padding_keeps_sketch_exact():
    parent = I.maxcut_rgg(40, 6.0, seed=1)
    child = I.grow_rgg(parent, 0.05, seed=2)
    psi = I.gaussian_psi(parent.n, 4, seed=3)
    o = U.USBSOracle(parent, k=6, psi=psi, dense_track=True, rho=1.0, ipm_mu_tol=1e-10)
    o.solve(tol=1e-6, max_iters=200)
    psi2 = I.extend_psi(psi, child.n, seed=4)
    w = U.warm_start(o, child, psi2)
    s = o.sp.tau / w.sp.tau
    Xpad = np.zeros((child.n, child.n))
    Xpad[:parent.n, :parent.n] = s * o.state.Xbar
    np.testing.assert_allclose(w.state.P, Xpad @ psi2.astype(np.float64), atol=1e-13)
    assert abs(w.state.tr - np.trace(Xpad)) <= 1e-13
    np.testing.assert_allclose(w.state.ax, np.diag(Xpad), atol=1e-13)
    assert abs(w.state.cx - np.sum(w.sp.C.toarray() * Xpad)) <= 1e-12
    hw = w.solve(tol=1e-7, max_iters=3)
    cold = U.USBSOracle(child, k=6, rho=1.0, ipm_mu_tol=1e-10)
    hc = cold.solve(tol=1e-7, max_iters=3)
    # the padded, rescaled state starts near the grown problem's optimum (Sec. 5.1)
    assert hw[-1]["relgap"] + hw[-1]["relinf"] < 0.5 * (hc[-1]["relgap"] + hc[-1]["relinf"])
    cold.solve(tol=1e-7, max_iters=100)
    w.solve(tol=1e-7, max_iters=100)
    assert abs(w.objective() - cold.objective()) <= 2e-4 * cold.objective()


def test_planted_wrong_sign_of_N_is_caught(monkeypatch):
    """The printed sign nu_I <= 0 yields negative candidate duals on inequality rows."""
    monkeypatch.setattr(U, "proj_N", lambda sp_, u: np.where(sp_.ineq, np.minimum(u, 0.0), 0.0))
    prob = _tiny_clustering(14, 30, 5)
    o = U.USBSOracle(prob, k=6)
    o.cold_start()
    broke = False
    for _ in range(10):
        info = o.step()
        yc, nu = info["y_cand"], info["nu"]
        broke |= bool(abs(yc @ nu) > 1e-8)
    assert broke


def test_planted_dropped_half_in_adjoint_is_caught(monkeypatch):
    """A*(y) without the 1/2 on off-diagonal entries breaks the dense certificate."""
    def bad(sp_, y):
        import scipy.sparse as sps
        w = y[sp_.con] * sp_.aval
        off = sp_.ai != sp_.aj
        rows = np.concatenate([sp_.ai[~off], sp_.ai[off], sp_.aj[off]])
        cols = np.concatenate([sp_.aj[~off], sp_.aj[off], sp_.ai[off]])
        vals = np.concatenate([w[~off], w[off], w[off]])
        return sps.csr_matrix((vals, (rows, cols)), shape=(sp_.n, sp_.n))
    monkeypatch.setattr(U, "A_adjoint", bad)
    with pytest.raises(AssertionError):
        test_clustering_primal_dual_certificate()
