"""Small FP64 subproblems of a USBS iteration (App. B).

Test infrastructure only (see ``oracle/__init__``).

``ipm_quad`` is the primal-dual path-following method of App. B.2 for
eq. compressed_subprob_2:

    minimise   1/2 s^T Q11 s + eta q12^T s + 1/2 eta^2 q22 + h1^T s + eta h2
    subject to eta >= 0,  S >= 0 (PSD),  1 - v^T s - eta >= 0,

with s = svec(S), v = svec(I).  Each Newton step solves eq. delta_S_linear_system2
for svec(dS) and back-substitutes the eliminated unknowns (derived from the
linearised system below eq. linearized_system2):

    d_eta   = (kappa1 a - c) / (kappa1 kappa2 + 1)
    d_omega = (kappa2 c + a) / (kappa1 kappa2 + 1)
    svec(dT) = mu svec(S^-1) - svec(T) - (T (x)_s S^-1) svec(dS)
    d_zeta  = mu / eta - zeta - (zeta / eta) d_eta

with a = -F2 + mu/eta - zeta - q12^T ds and c = mu/omega + v^T s + eta - 1 + v^T ds.

App. B.1 (the program whose value is the model value) is the same method with
Q11 = 0, q12 = 0, q22 = 0, h1 = g1, h2 = g2: ``ipm_linear``.

Readings where App. B is silent (each is listed in the design notes):
* start point S = I/(2k), eta = 1/4, T = I, zeta = omega = 1 ("arbitrary strictly
  feasible" in App. B.1);
* backtracking halves delta from 1 until S, T are positive definite (Cholesky) and
  eta, zeta, omega and the trace slack are positive, then takes 0.95 delta;
* at most 100 Newton steps; stop once mu < mu_tol (1e-7 as in App. B.1);
* every call starts from the fixed point above (no warm start across alternations);
* when tr(Xbar) = 0 the eta block does not exist: eta is fixed at 0 and the eta,
  zeta rows are dropped, and mu is estimated with 2(k+1) in place of 2(k+2).
"""
import numpy as np

from .svec import skron, smat, svec


def _is_pd(A):
    try:
        np.linalg.cholesky(A)
        return True
    except np.linalg.LinAlgError:
        return False


def ipm_quad(Q11, q12, q22, h1, h2, k, has_eta=True, mu_tol=1e-7, max_iter=100):
    """App. B.2 IPM.  Returns dict(S, eta, T, zeta, omega, mu, iters)."""
    v = svec(np.eye(k))
    S = np.eye(k) / (2 * k)
    T = np.eye(k)
    eta = 0.25 if has_eta else 0.0
    zeta = 1.0
    omega = 1.0
    denom = 2.0 * (k + 2) if has_eta else 2.0 * (k + 1)

    def slack_of(S_, eta_):
        return 1.0 - np.trace(S_) - eta_

    def mu_est(S_, T_, eta_, zeta_, omega_):
        val = np.sum(S_ * T_) + omega_ * slack_of(S_, eta_)
        if has_eta:
            val += eta_ * zeta_
        return val / denom

    mu = mu_est(S, T, eta, zeta, omega)
    it = 0
    for it in range(1, max_iter + 1):
        Sinv = np.linalg.inv(S)
        Sinv = 0.5 * (Sinv + Sinv.T)
        s, t = svec(S), svec(T)
        slack = slack_of(S, eta)
        TS = skron(T, Sinv)
        F1 = Q11 @ s + eta * q12 + h1 - t + omega * v
        kappa1 = slack / omega
        r3 = mu / omega - slack                     # mu/omega + v^T s + eta - 1
        rhs1 = -F1 + mu * svec(Sinv) - t
        if has_eta:
            F2 = q12 @ s + eta * q22 + h2 - zeta + omega
            kappa2 = zeta / eta + q22
            r2 = -F2 + mu / eta - zeta
            det = kappa1 * kappa2 + 1.0
            L = Q11 + TS - (np.outer(q12, kappa1 * q12 + v) + np.outer(v, q12 - kappa2 * v)) / det
            rhs = rhs1 - (q12 * (kappa1 * r2 - r3) + v * (kappa2 * r3 + r2)) / det
            ds = np.linalg.solve(L, rhs)
            a = r2 - q12 @ ds
            c = r3 + v @ ds
            deta = (kappa1 * a - c) / det
            domega = (kappa2 * c + a) / det
            dzeta = mu / eta - zeta - (zeta / eta) * deta
        else:
            L = Q11 + TS + np.outer(v, v) / kappa1
            rhs = rhs1 - v * (r3 / kappa1)
            ds = np.linalg.solve(L, rhs)
            domega = (r3 + v @ ds) / kappa1
            deta = dzeta = 0.0
        dt = mu * svec(Sinv) - t - TS @ ds
        dS, dT = smat(ds), smat(dt)
        delta = 1.0
        for _ in range(80):
            S_n, T_n = S + delta * dS, T + delta * dT
            eta_n, zeta_n, omega_n = eta + delta * deta, zeta + delta * dzeta, omega + delta * domega
            ok = (_is_pd(S_n) and _is_pd(T_n) and omega_n > 0 and slack_of(S_n, eta_n) > 0
                  and (not has_eta or (eta_n > 0 and zeta_n > 0)))
            if ok:
                break
            delta *= 0.5
        delta *= 0.95
        S = S + delta * dS
        T = T + delta * dT
        S = 0.5 * (S + S.T)
        T = 0.5 * (T + T.T)
        omega += delta * domega
        if has_eta:
            eta += delta * deta
            zeta += delta * dzeta
        gamma = 1.0 if delta <= 0.2 else 0.5 - 0.4 * delta * delta
        mu = min(mu, gamma * mu_est(S, T, eta, zeta, omega))
        if mu < mu_tol:
            break
    return {"S": S, "eta": eta, "T": T, "zeta": zeta, "omega": omega, "mu": mu, "iters": it}


def ipm_linear(g1, g2, k, has_eta=True, mu_tol=1e-7, max_iter=100):
    """App. B.1: minimise g1^T svec(S) + eta g2 over the same set (Q11 = q12 = q22 = 0)."""
    K = g1.shape[0]
    return ipm_quad(np.zeros((K, K)), np.zeros(K), 0.0, g1, g2, k, has_eta, mu_tol, max_iter)


def quad_objective(Q11, q12, q22, h1, h2, S, eta):
    s = svec(S)
    return 0.5 * s @ Q11 @ s + eta * (q12 @ s) + 0.5 * eta * eta * q22 + h1 @ s + eta * h2


def model_value_closed_form(b_dot_y, alpha, VZV, has_eta, xbar_term):
    """Model value f_hat_t(y) for a feasible y (App. B.1 without the IPM).

    The model set {alpha (eta_hat Xbar/tr Xbar + V S_hat V^T) : eta_hat + tr S_hat <= 1,
    eta_hat >= 0, S_hat >= 0} is the convex hull of 0, alpha Xbar/tr Xbar and
    alpha u u^T with u a unit vector in range(V); a linear function <Z, X> attains its
    maximum at one of these points, where it equals 0, alpha <Z, Xbar>/tr Xbar or
    alpha lambda_max(V^T Z V) (eq. max_eigenvalue_equiv).  Here VZV = V^T Z V and
    xbar_term = <Z, Xbar>/tr Xbar, Z = C - A*(y).
    """
    cands = [0.0, float(np.linalg.eigvalsh(0.5 * (VZV + VZV.T))[-1])]
    if has_eta:
        cands.append(float(xbar_term))
    return b_dot_y + alpha * max(cands)
