"""Plain FP64 USBS: Algorithm 1 with the implicit primal and the Nystrom sketch.

Test infrastructure only (see ``oracle/__init__``).

Follows, in this order, the paper's Sec. 3 (Algorithm 1, eq. pen-D, eqs. subspace_def
to v_next_def, dual_update, small_quad_sdp, dual_slack_update), Sec. 4 (sketch update),
App. B.2 (data Q11, q12, q22, h1, h2 of eq. compressed_subprob_2), App. C (implicit
<C, Xbar>, tr Xbar, A Xbar) and App. E (scaling ||C||_F = tr X* = 1, alpha = 2; gates of
eq. relative_error_tol with the bound of eq. objective_subopt_upper_bound).

The model set is read as X = alpha (eta_hat Xbar/tr Xbar + V S_hat V^T) with
eta_hat >= 0, S_hat >= 0 and eta_hat + tr S_hat <= 1: this is the normalisation that
reproduces the printed Q11, q12, q22, h1, h2 and the constraint 1 - v^T svec(S) - eta >= 0.
The IPM returns (eta_hat, S_hat); then eta = alpha eta_hat / tr Xbar and S = alpha S_hat.

The dual slack set is read as N = {nu : nu_I >= 0, nu_I' = 0}: that is the sign for
which the candidate of eq. dual_update equals proj_Y(y - (b - A X)/rho), is
complementary to nu and keeps y_I >= 0, as Sec. 3 states; the printed "nu_I <= 0" would
give y_I <= 0.

k_p = 0 by default (Xbar = X, V_{t+1} = [v_1..v_kc]), as in the configurations built.
With k_p > 0 (Sec. 3, eqs. model_update_eigendecomposition, x_bar_def, v_next_def) V has
k_c + k_p columns; S_{t+1} = Q_p L_p Q_p^T + Q_c L_c Q_c^T splits off its k_p largest
eigenpairs as past information, Xbar_{t+1} = eta Xbar_t + V Q_c L_c Q_c^T V^T takes only
the rest, and V_{t+1} is an orthonormal basis (QR) of [V Q_p, v_1..v_kc].  The primal
iterate X_{t+1} = eta Xbar_t + V S V^T then differs from Xbar_{t+1}; the gates and the
objective are X_{t+1}'s, the model and the sketch Xbar's.  The cold start takes the top
k_c + k_p eigenvectors of C as V_0.
"""
import dataclasses
import math

import numpy as np
import scipy.sparse as sp

from .eig import top_eigenpairs
from .ipm import ipm_quad, model_value_closed_form
from .svec import smat, svec, svec_dim, SQRT2


@dataclasses.dataclass
class ScaledProblem:
    n: int
    m: int
    C: sp.csr_matrix          # C / ||C||_F
    con: np.ndarray
    ai: np.ndarray
    aj: np.ndarray
    aval: np.ndarray
    b: np.ndarray             # b / tr X*
    ineq: np.ndarray          # bool
    c_scale: float            # ||C||_F
    tau: float                # tr X*


def scale_problem(prob):
    """App. E, eq. std_scaling: C <- C/||C||_F, b <- b / tr(X*) so X_s = X / tr(X*)."""
    n = prob.n
    c_scale = float(np.sqrt(np.sum(np.asarray(prob.C_val, dtype=np.float64) ** 2)))
    if c_scale == 0.0:
        c_scale = 1.0
    C = sp.csr_matrix((np.asarray(prob.C_val, dtype=np.float64) / c_scale,
                       np.asarray(prob.C_col), np.asarray(prob.C_rowptr)), shape=(n, n))
    tau = float(prob.trace)
    return ScaledProblem(n, prob.m, C, np.asarray(prob.A_con, np.int64),
                         np.asarray(prob.A_i, np.int64), np.asarray(prob.A_j, np.int64),
                         np.asarray(prob.A_val, np.float64),
                         np.asarray(prob.b, np.float64) / tau,
                         np.asarray(prob.is_ineq).astype(bool), c_scale, tau)


# ---- the linear maps A and A* (Sec. 2.1) ---------------------------------------------

def A_dense(sp_, X):
    """(A X)_c = sum over entries (c, i, j, v) of v X_ij."""
    return np.bincount(sp_.con, weights=sp_.aval * X[sp_.ai, sp_.aj], minlength=sp_.m)


def A_lowrank(sp_, V, S):
    """A(V S V^T): X_ij = V_i S V_j^T for each entry (App. C, constraint evaluation)."""
    Xij = np.einsum("ep,pq,eq->e", V[sp_.ai], S, V[sp_.aj])
    return np.bincount(sp_.con, weights=sp_.aval * Xij, minlength=sp_.m)


def A_adjoint(sp_, y):
    """A*(y) = sum_c y_c A_c as a sparse symmetric matrix."""
    w = y[sp_.con] * sp_.aval
    off = sp_.ai != sp_.aj
    rows = np.concatenate([sp_.ai[~off], sp_.ai[off], sp_.aj[off]])
    cols = np.concatenate([sp_.aj[~off], sp_.aj[off], sp_.ai[off]])
    vals = np.concatenate([w[~off], 0.5 * w[off], 0.5 * w[off]])
    return sp.csr_matrix((vals, (rows, cols)), shape=(sp_.n, sp_.n))


def slack_matrix(sp_, y):
    """C - A*(y), the dual slack matrix of (D)."""
    return (sp_.C - A_adjoint(sp_, y)).tocsr()


def G_matrix(sp_, V):
    """Rows g_c = svec(V^T A_c V) (App. B.2, the factors of Q11).

    An entry (c, i, j, v) contributes (v/2)(V_i^T V_j + V_j^T V_i), V_i being row i.
    """
    k = V.shape[1]
    Vi, Vj = V[sp_.ai], V[sp_.aj]
    E = np.empty((len(sp_.con), svec_dim(k)))
    p = 0
    for q in range(k):
        for r in range(q, k):
            term = 0.5 * sp_.aval * (Vi[:, r] * Vj[:, q] + Vj[:, r] * Vi[:, q])
            E[:, p] = term if r == q else SQRT2 * term
            p += 1
    agg = sp.csr_matrix((np.ones(len(sp_.con)), (sp_.con, np.arange(len(sp_.con)))),
                        shape=(sp_.m, len(sp_.con)))
    return np.asarray(agg @ E)


def proj_K(sp_, z):
    """Projection onto K = {z : z_I <= b_I, z_I' = b_I'} (Sec. 2.1)."""
    out = np.where(sp_.ineq, np.minimum(z, sp_.b), sp_.b)
    return out


def proj_Y(sp_, y):
    """Projection onto Y = {y : y_I >= 0}."""
    return np.where(sp_.ineq, np.maximum(y, 0.0), y)


def proj_N(sp_, u):
    """Projection onto N = {nu : nu_I >= 0, nu_I' = 0} (sign reading in module doc)."""
    return np.where(sp_.ineq, np.maximum(u, 0.0), 0.0)


# ---- state ----------------------------------------------------------------------------

def split_past(S, k_p):
    """eq. model_update_eigendecomposition: (Q_p, Q_c, L_c) with Q_p the eigenvectors of the
    k_p largest eigenvalues of S (past information) and (Q_c, L_c) the remaining pairs."""
    lam, Q = np.linalg.eigh(0.5 * (S + S.T))
    order = np.argsort(-lam, kind="stable")
    lam, Q = lam[order], Q[:, order]
    return Q[:, :k_p], Q[:, k_p:], lam[k_p:]


@dataclasses.dataclass
class State:
    y: np.ndarray
    V: np.ndarray
    f_y: float
    cx: float                 # <C, Xbar>
    tr: float                 # tr Xbar
    ax: np.ndarray            # A Xbar
    P: np.ndarray             # Xbar Psi (n x r), r may be 0
    Xbar: np.ndarray = None   # dense Xbar, only when tracked (tiny n)
    t: int = 0
    cx_it: float = 0.0        # <C, X_t> of the primal iterate (= cx when k_p = 0)
    ax_it: np.ndarray = None  # A X_t (= ax when k_p = 0)
    X: np.ndarray = None      # dense X_t, only when tracked


class USBSOracle:
    """One USBS instance (Algorithm 1), FP64.  k = k_c current eigenvectors, k_p past
    columns (default 0)."""

    def __init__(self, prob, k=8, rho=0.01, beta=0.25, alpha=2.0, psi=None,
                 ipm_mu_tol=1e-7, max_alt=50, alt_tol=1e-8, eig_tol=1e-10,
                 dense_track=False, seed=0, k_p=0):
        self.prob = prob
        self.sp = scale_problem(prob)
        k = min(k, prob.n)
        self.k, self.rho, self.beta, self.alpha = k, rho, beta, alpha
        self.k_p = max(0, min(int(k_p), prob.n - k))
        self.psi = None if psi is None else np.asarray(psi, dtype=np.float64)
        self.ipm_mu_tol, self.max_alt, self.alt_tol = ipm_mu_tol, max_alt, alt_tol
        self.eig_tol = eig_tol
        self.dense_track = dense_track
        self.seed = seed
        self.bnorm = float(np.linalg.norm(self.sp.b))
        self.state = None

    # f(y) of eq. pen-D for y in Y
    def eig_at(self, y, start=None):
        M = slack_matrix(self.sp, y)
        w, U = top_eigenpairs(M, self.k, start=start, tol=self.eig_tol, seed=self.seed)
        return w, U

    def f_value(self, lam_max, y):
        return self.alpha * max(lam_max, 0.0) + float(self.sp.b @ y)

    def cold_start(self):
        """y_0 = 0, Xbar_0 = 0 (tr Xbar_0 = 0), V_0 = top-(k_c + k_p) eigenvectors of C."""
        n, m = self.sp.n, self.sp.m
        y = np.zeros(m)
        if self.k_p:
            w, U = top_eigenpairs(slack_matrix(self.sp, y), self.k + self.k_p, tol=self.eig_tol,
                                  seed=self.seed)
        else:
            w, U = self.eig_at(y)
        r = 0 if self.psi is None else self.psi.shape[1]
        self.state = State(y=y, V=U, f_y=self.f_value(w[0], y), cx=0.0, tr=0.0,
                           ax=np.zeros(m), P=np.zeros((n, r)),
                           Xbar=np.zeros((n, n)) if self.dense_track else None,
                           cx_it=0.0, ax_it=np.zeros(m),
                           X=np.zeros((n, n)) if self.dense_track else None)
        return self.state

    def model_data(self, st):
        """V^T C V, G and the quadratic data of eq. compressed_subprob_2."""
        sp_, a, rho = self.sp, self.alpha, self.rho
        Vc = st.V.T @ (sp_.C @ st.V)
        Vc = 0.5 * (Vc + Vc.T)
        G = G_matrix(sp_, st.V)
        has_eta = st.tr > 0.0
        Q11 = (a * a / rho) * (G.T @ G)
        if has_eta:
            q12 = (a * a / (rho * st.tr)) * (G.T @ st.ax)
            q22 = (a * a / (rho * st.tr ** 2)) * float(st.ax @ st.ax)
        else:
            q12 = np.zeros(G.shape[1])
            q22 = 0.0
        return Vc, G, has_eta, Q11, q12, q22

    def linear_data(self, st, Vc, G, has_eta, nu):
        """h1, h2 of eq. compressed_subprob_2 with w = y_t - (b - nu)/rho."""
        a = self.alpha
        w = st.y - (self.sp.b - nu) / self.rho
        h1 = a * (G.T @ w - svec(Vc))
        h2 = a * (float(st.ax @ w) - st.cx) / st.tr if has_eta else 0.0
        return h1, h2

    def step(self):
        """One iteration of Algorithm 1.  Returns a dict of diagnostics."""
        st = self.state
        sp_, a, rho, k = self.sp, self.alpha, self.rho, self.k
        Vc, G, has_eta, Q11, q12, q22 = self.model_data(st)
        # alternating maximisation over (X, nu), eqs. small_quad_sdp / dual_slack_update
        nu = np.zeros(sp_.m)
        any_ineq = bool(np.any(sp_.ineq))
        n_alt = 0
        ipm_iters = 0
        kv = st.V.shape[1]                    # k_c + k_p columns
        for n_alt in range(1, self.max_alt + 1):
            h1, h2 = self.linear_data(st, Vc, G, has_eta, nu)
            sol = ipm_quad(Q11, q12, q22, h1, h2, kv, has_eta, self.ipm_mu_tol)
            ipm_iters += sol["iters"]
            S_hat, eta_hat = sol["S"], sol["eta"]
            if not any_ineq:
                break
            AX_t = a * ((eta_hat / st.tr) * st.ax if has_eta else 0.0) + a * (G @ svec(S_hat))
            nu_new = proj_N(sp_, sp_.b - AX_t - rho * st.y)
            done = np.linalg.norm(nu_new - nu) <= self.alt_tol * (1.0 + self.bnorm)
            nu = nu_new
            if done:
                break
        eta = a * eta_hat / st.tr if has_eta else 0.0
        S = a * S_hat
        # X_{t+1} = eta Xbar_t + V S V^T through its implicit quantities (App. C)
        AX = eta * st.ax + A_lowrank(sp_, st.V, S)
        CX = eta * st.cx + float(np.sum(Vc * S))
        trX = eta * st.tr + float(np.trace(S))
        # candidate, eq. dual_update in its projected form
        y_new = proj_Y(sp_, st.y - (sp_.b - AX) / rho)
        w, U = self.eig_at(y_new, start=st.V[:, :k])
        f_new = self.f_value(w[0], y_new)
        # model value f_hat_t(y_new) (App. B.1, closed form)
        VZV = Vc - smat(G.T @ y_new)
        xbar_term = (st.cx - float(st.ax @ y_new)) / st.tr if has_eta else 0.0
        f_hat = model_value_closed_form(float(sp_.b @ y_new), a, VZV, has_eta, xbar_term)
        f_old = st.f_y
        descent = self.beta * (f_old - f_hat) <= f_old - f_new
        if descent:
            st.y, st.f_y = y_new, f_new
        if st.X is not None:
            st.X = eta * st.Xbar + st.V @ S @ st.V.T
        st.cx_it, st.ax_it = CX, AX
        if self.k_p == 0:
            # model update with k_p = 0: Xbar_{t+1} = X_{t+1}; sketch; V_{t+1}
            if st.P.shape[1]:
                st.P = eta * st.P + st.V @ (S @ (st.V.T @ self.psi))
            if st.Xbar is not None:
                st.Xbar = eta * st.Xbar + st.V @ S @ st.V.T
            st.cx, st.tr, st.ax = CX, trX, AX
            st.V = U
        else:
            Qp, Qc, Lc = split_past(S, self.k_p)
            Sc = (Qc * Lc) @ Qc.T
            # eq. x_bar_def through its implicit quantities (App. C)
            st.cx = eta * st.cx + float(np.sum(Vc * Sc))
            st.tr = eta * st.tr + float(np.sum(Lc))
            st.ax = eta * st.ax + A_lowrank(sp_, st.V, Sc)
            if st.P.shape[1]:
                st.P = eta * st.P + st.V @ (Sc @ (st.V.T @ self.psi))
            if st.Xbar is not None:
                st.Xbar = eta * st.Xbar + st.V @ Sc @ st.V.T
            # eq. v_next_def: an orthonormal basis of [V Q_p, v_1..v_kc] by QR
            st.V, _ = np.linalg.qr(np.hstack([st.V @ Qp, U]))
        st.t += 1
        relgap, relinf = self.gates(st)
        return {"t": st.t, "descent": bool(descent), "f_y": st.f_y, "f_cand": f_new,
                "f_hat": f_hat, "f_old": f_old, "lambda_max": float(w[0]), "eigs": w,
                "cx": CX, "trX": trX, "eta": eta, "S": S, "eta_hat": eta_hat,
                "y_cand": y_new, "nu": nu, "n_alt": n_alt, "ipm_iters": ipm_iters,
                "relgap": relgap, "relinf": relinf, "AX": AX}

    def gates(self, st):
        """Relative suboptimality bound and relative infeasibility (App. E) of the primal
        iterate X_t, scaled units."""
        cx = st.cx_it if self.k_p else st.cx
        ax = st.ax_it if self.k_p else st.ax
        relgap = abs(st.f_y - cx) / (1.0 + abs(cx))
        relinf = float(np.linalg.norm(ax - proj_K(self.sp, ax))) / (1.0 + self.bnorm)
        return relgap, relinf

    def solve(self, tol=1e-3, max_iters=1000, callback=None):
        if self.state is None:
            self.cold_start()
        hist = []
        for _ in range(max_iters):
            info = self.step()
            hist.append(info)
            if callback:
                callback(info)
            if info["relgap"] <= tol and info["relinf"] <= tol:
                break
        return hist

    # results in the units of the unscaled problem
    def objective(self):
        cx = self.state.cx_it if self.k_p else self.state.cx
        return cx * self.sp.c_scale * self.sp.tau

    def dual_bound(self):
        return self.state.f_y * self.sp.c_scale * self.sp.tau


def warm_start(old: USBSOracle, new_prob, psi_new=None, **kw):
    """Warm start on a grown instance (Sec. 5.1: pad with zeros, rescale).

    Reading: y is unscaled with the old ||C||_F, zero-padded for the new rows and
    rescaled with the new one; the implicit primal (tr Xbar, A Xbar, P) is scaled by
    tau_old/tau_new and zero-padded; <C', Xbar'> adds the change of C on old-old
    entries, which must be diagonal with each X_ii fixed by a one-entry constraint
    (true for MaxCut growth); otherwise the implicit primal restarts at 0.  V and
    f(y) come from an eigen solve at the new y started from the padded V.
    """
    o = old.state
    osp = old.sp
    new = USBSOracle(new_prob, k=old.k, rho=old.rho, beta=old.beta, alpha=old.alpha,
                     psi=psi_new, ipm_mu_tol=old.ipm_mu_tol, max_alt=old.max_alt,
                     alt_tol=old.alt_tol, eig_tol=old.eig_tol, seed=old.seed, **kw)
    nsp = new.sp
    n0, m0 = osp.n, osp.m
    y = np.zeros(nsp.m)
    y[:m0] = o.y * osp.c_scale / nsp.c_scale
    s = osp.tau / nsp.tau
    Vpad = np.zeros((nsp.n, old.k))
    Vpad[:n0] = o.V
    ok = o.tr > 0.0
    # change of C restricted to old x old entries
    Cn = (nsp.C * nsp.c_scale).tocsr()[:n0, :n0]
    Co = (osp.C * osp.c_scale).tocsr()
    dC = (Cn - Co).tocoo()
    nz = np.abs(dC.data) > 0
    di, dj, dv = dC.row[nz], dC.col[nz], dC.data[nz]
    corr = 0.0
    if ok and np.any(di != dj):
        ok = False
    if ok and len(di):
        single = {}
        counts = np.bincount(osp.con, minlength=m0)
        for e in range(len(osp.con)):
            c = osp.con[e]
            if counts[c] == 1 and osp.ai[e] == osp.aj[e]:
                single[int(osp.ai[e])] = (c, osp.aval[e])
        for i, v in zip(di, dv):
            if int(i) not in single:
                ok = False
                break
            c, av = single[int(i)]
            corr += v * o.ax[c] / av
    r = 0 if psi_new is None else psi_new.shape[1]
    P = np.zeros((nsp.n, r))
    ax = np.zeros(nsp.m)
    if ok:
        # new constraints must only touch new vertices for A Xbar' = [A Xbar; 0]
        newc = nsp.con >= m0
        if np.any(newc & (nsp.ai < n0) & (nsp.aj < n0)):
            ok = False
    if ok:
        ax[:m0] = s * o.ax
        cx = s * (osp.c_scale * o.cx + corr) / nsp.c_scale
        tr = s * o.tr
        if r:
            P[:n0] = s * o.P
    else:
        cx, tr = 0.0, 0.0
    w, U = new.eig_at(y, start=Vpad)
    new.state = State(y=y, V=U, f_y=new.f_value(w[0], y), cx=cx, tr=tr, ax=ax, P=P)
    return new
