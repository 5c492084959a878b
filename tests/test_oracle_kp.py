"""Pins of the oracle's past-information columns (k_p > 0; Sec. 3, eqs.
model_update_eigendecomposition, x_bar_def, v_next_def) by closed forms and by the
invariants the paper states for the model update."""
import numpy as np
import pytest

from oracle import usbs as U
from paper_2312_11801_gb300 import instances as I
from tests._graphs import load_sdp_values, named_problem


def _dense_A(prob):
    A = np.zeros((prob.m, prob.n, prob.n))
    for c, i, j, v in zip(prob.A_con, prob.A_i, prob.A_j, prob.A_val):
        if i == j:
            A[c, i, i] += v
        else:
            A[c, i, j] += 0.5 * v
            A[c, j, i] += 0.5 * v
    return A


@pytest.mark.parametrize("name,k_c,k_p", [("K5", 4, 1), ("C7", 4, 2), ("petersen", 5, 3), ("K3,3", 3, 1)])
def test_closed_forms_with_past_columns(name, k_c, k_p, golden_dir):
    """The theorem of Sec. 3 holds for every k_p >= 0: the solve reaches the known SDP
    value from both sides."""
    n, val = load_sdp_values(f"{golden_dir}/maxcut_sdp_values.txt")[name]
    o = U.USBSOracle(named_problem(name), k=k_c, k_p=k_p)
    o.solve(tol=1e-5, max_iters=400)
    assert o.state.V.shape[1] == k_c + k_p
    assert o.dual_bound() >= val * (1 - 1e-9)
    assert abs(o.objective() - val) <= 3e-5 * val
    assert abs(o.dual_bound() - val) <= 3e-5 * val


@pytest.mark.parametrize("k_p", [1, 3])
def test_model_update_invariants(k_p):
    """Dense tracking on a 24-vertex graph, every step:
    - V_t has k_c + k_p orthonormal columns and spans V_{t-1} Q_p (past information kept);
    - X_{t+1} = eta Xbar_t + V_t S V_t^T and Xbar_{t+1} = X_{t+1} - V_t Q_p L_p Q_p^T V_t^T
      with (Q_p, L_p) the k_p largest eigenpairs of S (eq. model_update_eigendecomposition);
    - Xbar is PSD; the implicit <C, Xbar>, tr Xbar, A Xbar and the sketch equal their dense
      values; the gates are those of the primal iterate X_{t+1}."""
    prob = I.maxcut_er(24, 5, seed=6)
    psi = I.gaussian_psi(24, 4, seed=3)
    k_c = 4
    o = U.USBSOracle(prob, k=k_c, k_p=k_p, psi=psi, dense_track=True)
    o.cold_start()
    s = o.sp
    A = _dense_A(prob)
    C = s.C.toarray()
    for _ in range(25):
        V0 = o.state.V.copy()
        Xbar0 = o.state.Xbar.copy()
        info = o.step()
        st = o.state
        S, eta = info["S"], info["eta"]
        lam, Q = np.linalg.eigh(0.5 * (S + S.T))
        Qp, Lp = Q[:, -k_p:], lam[-k_p:]
        X_it = eta * Xbar0 + V0 @ S @ V0.T
        np.testing.assert_allclose(st.X, X_it, atol=1e-12)
        np.testing.assert_allclose(st.Xbar, X_it - (V0 @ Qp * Lp) @ (V0 @ Qp).T, atol=1e-11)
        assert st.V.shape == (prob.n, k_c + k_p)
        np.testing.assert_allclose(st.V.T @ st.V, np.eye(k_c + k_p), atol=1e-12)
        W = V0 @ Qp
        assert np.linalg.norm(W - st.V @ (st.V.T @ W)) <= 1e-10
        assert np.linalg.eigvalsh(st.Xbar).min() >= -1e-10
        assert abs(st.cx - np.sum(C * st.Xbar)) <= 1e-12 * (1 + abs(st.cx))
        assert abs(st.tr - np.trace(st.Xbar)) <= 1e-12
        np.testing.assert_allclose(st.ax, np.einsum("cij,ij->c", A, st.Xbar), atol=1e-13)
        np.testing.assert_allclose(st.P, st.Xbar @ psi.astype(np.float64), atol=1e-12)
        ax_it = np.einsum("cij,ij->c", A, X_it)
        relinf = np.linalg.norm(ax_it - s.b) / (1 + np.linalg.norm(s.b))
        assert abs(info["relinf"] - relinf) <= 1e-12
        assert abs(info["cx"] - np.sum(C * X_it)) <= 1e-12 * (1 + abs(info["cx"]))


def test_k_p_zero_is_the_default_path():
    """k_p = 0 keeps Xbar = X and V_{t+1} = [v_1..v_kc]: identical iterates."""
    prob = I.maxcut_er(40, 5, seed=2)
    a = U.USBSOracle(prob, k=6)
    b = U.USBSOracle(prob, k=6, k_p=0)
    a.cold_start()
    b.cold_start()
    for _ in range(10):
        ia, ib = a.step(), b.step()
        assert ia["f_y"] == ib["f_y"] and ia["cx"] == ib["cx"]


def test_planted_full_S_into_Xbar_is_caught(monkeypatch):
    """If Xbar absorbed all of S (the k_p = 0 rule) while V still kept V Q_p, the
    model-update invariants fail: Xbar_{t+1} must leave out V Q_p L_p Q_p^T V^T."""
    real = U.split_past

    def planted(S, k_p):
        Qp, _, _ = real(S, k_p)
        lam, Q = np.linalg.eigh(0.5 * (S + S.T))
        return Qp, Q, lam
    monkeypatch.setattr(U, "split_past", planted)
    with pytest.raises(AssertionError):
        test_model_update_invariants(1)
