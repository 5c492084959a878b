"""Fixed-rank reconstruction of the primal from its Nystrom sketch, and MaxCut rounding.

Test infrastructure only (see ``oracle/__init__``).

App. C, eq. nystrom_approx: the sketch P = X Psi of the implicit primal and the test matrix
Psi give the Nystrom approximation X_hat = P (Psi^T P)^+ P^T, computed by the numerically
stable method the paper adopts (Tropp, Yurtsever, Udell and Cevher, "Fixed-rank
approximation of a positive-semidefinite matrix from streaming data", NeurIPS 2017,
Algorithm 3):

1. nu = sqrt(n) * eps(||P||_2), the spacing of the floating-point numbers at ||P||_2;
2. Y = P + nu Psi;
3. B = Psi^T Y, symmetrised, and its Cholesky factor B = R^T R (R upper triangular);
4. E = Y R^-1 and its thin singular value decomposition E = U Sigma W^T;
5. Lambda = max(Sigma^2 - nu I, 0), X_hat = U Lambda U^T.

App. E (MaxCut, rounding): every column u of U gives the cut sgn(u) (0 counted as +1);
the value of the sign vector z is <C, z z^T> = z^T C z in problem units, the MaxCut
objective (1/4) z^T L z when C = L/4; the best of the r columns is kept.

App. E (QAP, rounding): every column of U, its first entry dropped and the remaining nq^2
reshaped into an nq x nq matrix (vec stacks columns), is projected onto the permutation
matrices by the Hungarian method (a linear assignment maximising <M, Pi>); the permutation
of least QAP cost tr(W Pi D Pi^T) over the columns is kept.
"""
import numpy as np
import scipy.linalg as sla
import scipy.optimize as so
import scipy.sparse as sp


def nystrom_shift(P):
    """The shift nu = sqrt(n) eps(||P||_2), eps(x) the spacing of the sketch's own
    floating-point format at x: 2^(e - 24) for an FP32 sketch and 2^(e - 53) for an FP64
    one, x = f 2^e with f in [1/2, 1).  (The shift must cover the rounding of the stored
    sketch: with an FP32 sketch and the FP64 spacing, Psi^T (P + nu Psi) is indefinite.)"""
    n = P.shape[0]
    norm = float(np.linalg.norm(np.asarray(P, dtype=np.float64), 2))
    if norm == 0.0:
        return 0.0
    bits = 24 if np.asarray(P).dtype == np.float32 else 53
    _, e = np.frexp(norm)
    return float(np.sqrt(n) * np.ldexp(1.0, int(e) - bits))


def nystrom_reconstruct(P, Psi):
    """The reconstruction above: (U, lam) with X_hat = U diag(lam) U^T, lam descending, U n x r.
    The arithmetic is FP64 whatever the sketch's format; the shift follows the format."""
    nu = nystrom_shift(P)
    P = np.asarray(P, dtype=np.float64)
    Psi = np.asarray(Psi, dtype=np.float64)
    Y = P + nu * Psi
    B = Psi.T @ Y
    B = 0.5 * (B + B.T)
    R = sla.cholesky(B, lower=False)                    # B = R^T R
    E = sla.solve_triangular(R, Y.T, trans="T", lower=False).T   # E R = Y
    U, sig, _ = np.linalg.svd(E, full_matrices=False)
    lam = np.maximum(sig ** 2 - nu, 0.0)
    return U, lam


def nystrom_matrix(P, Psi):
    """X_hat as a dense matrix (small n only)."""
    U, lam = nystrom_reconstruct(P, Psi)
    return (U * lam) @ U.T


def sign_vector(u):
    """sgn with 0 -> +1."""
    return np.where(np.asarray(u) >= 0.0, 1.0, -1.0)


def rounding_values(C, U):
    """<C, z_k z_k^T> for z_k = sgn(U[:, k]), every column k (C sparse or dense, n x n)."""
    Z = sign_vector(U)
    CZ = C @ Z
    return np.einsum("ik,ik->k", Z, np.asarray(CZ))


def maxcut_round(C, U):
    """(best value, best column, its sign vector) over the columns of U."""
    vals = rounding_values(C, U)
    k = int(np.argmax(vals))
    return float(vals[k]), k, sign_vector(U[:, k])


def cut_weight(n, ei, ej, w, z):
    """Total weight of the edges whose ends z separates (each edge listed once)."""
    z = np.asarray(z)
    return float(np.sum(np.asarray(w)[z[np.asarray(ei)] != z[np.asarray(ej)]]))


def qap_cost(W, D, Pi):
    """tr(W Pi D Pi^T)."""
    return float(np.trace(W @ Pi @ D @ Pi.T))


def project_permutation(M):
    """The permutation matrix Pi maximising <M, Pi> (Hungarian method)."""
    nq = M.shape[0]
    rows, cols = so.linear_sum_assignment(-np.asarray(M, dtype=np.float64))
    Pi = np.zeros((nq, nq))
    Pi[rows, cols] = 1.0
    return Pi


def qap_round(U, W, D):
    """(least cost, its column, its permutation) over the columns of U ((nq^2 + 1) x r).
    An eigenvector is defined up to sign; each column is oriented so that its first entry,
    the one paired with X_00 = 1, is non-negative (for X = v v^T with v = [1; vec(B)] this
    gives +vec(B)) before that entry is dropped."""
    nq = W.shape[0]
    best = (np.inf, -1, None)
    for k in range(U.shape[1]):
        sgn = 1.0 if U[0, k] >= 0.0 else -1.0
        M = (sgn * U[1:, k]).reshape((nq, nq), order="F")
        Pi = project_permutation(M)
        c = qap_cost(W, D, Pi)
        if c < best[0]:
            best = (c, k, Pi)
    return best
