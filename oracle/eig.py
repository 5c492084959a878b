"""Extreme eigenpairs of the dual slack matrix C - A*(y) (Sec. 3, eq. pen-D; App. E).

Test infrastructure only (see ``oracle/__init__``).

The USBS step needs the top k_c eigenpairs of a symmetric matrix.  That result has a
plain definition, so the oracle computes it directly:

* ``jacobi_eigh``: cyclic Jacobi rotations on the dense matrix (textbook method,
  Golub and Van Loan Sec. 8.5), used for n <= 64;
* ``dense_top``: LAPACK ``eigh`` on the dense matrix for n <= 4096 (library primitive);
* ``block_lanczos_top``: block Lanczos with full (two-pass classical Gram-Schmidt)
  reorthogonalisation and thick restart, in FP64, for larger sparse matrices.  The
  paper runs thick-restart Lanczos (App. E: 32 inner iterations, at most 10
  restarts); the oracle instead runs to a residual tolerance.

All return eigenvalues in descending order and orthonormal eigenvectors as columns.
"""
import numpy as np
import scipy.linalg
import scipy.sparse as sp

DENSE_MAX_N = 4096
JACOBI_MAX_N = 16


def jacobi_eigh(A, tol=1e-15, max_sweeps=60):
    """All eigenpairs of a small dense symmetric matrix by cyclic Jacobi."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    scale = np.linalg.norm(A)
    for _ in range(max_sweeps):
        off = np.sqrt(max(np.sum(A * A) - np.sum(np.diag(A) ** 2), 0.0))
        if off <= tol * max(scale, 1e-300):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                if abs(tau) > 1e150:        # t -> 1/(2 tau) without overflow
                    t = 0.5 / tau
                else:
                    t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + np.sqrt(1.0 + tau * tau))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                colp, colq = A[:, p].copy(), A[:, q].copy()
                A[:, p], A[:, q] = c * colp - s * colq, s * colp + c * colq
                rowp, rowq = A[p, :].copy(), A[q, :].copy()
                A[p, :], A[q, :] = c * rowp - s * rowq, s * rowp + c * rowq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p], V[:, q] = c * vp - s * vq, s * vp + c * vq
    w = np.diag(A).copy()
    order = np.argsort(-w, kind="stable")
    return w[order], V[:, order]


def dense_top(A, k):
    n = A.shape[0]
    w, V = scipy.linalg.eigh(A, subset_by_index=[n - k, n - 1])
    return w[::-1].copy(), V[:, ::-1].copy()


def _orth_against(W, Q, rng, tiny):
    """Two passes of classical Gram-Schmidt of W against the columns of Q, then QR.

    Columns that vanish (rank deficiency, e.g. an exhausted Krylov space) are replaced
    by seeded random vectors orthogonal to Q and to the other columns; their rows of R
    are zero.
    """
    if Q.shape[1]:
        W = W - Q @ (Q.T @ W)
        W = W - Q @ (Q.T @ W)
    Qn, R = np.linalg.qr(W)
    for i in range(W.shape[1]):
        if abs(R[i, i]) <= tiny:
            z = rng.standard_normal(W.shape[0])
            base = np.hstack([Q, Qn[:, :i]])
            for _ in range(2):
                z = z - base @ (base.T @ z)
            Qn[:, i] = z / np.linalg.norm(z)
            R[i, :] = 0.0
    if W.shape[1] > 1:                  # re-orthonormalise the block itself
        Qn2, R2 = np.linalg.qr(Qn)
        Qn = Qn2 * np.sign(np.diag(R2))
    return Qn, R


def block_lanczos_top(matvec, n, k, X0=None, b=8, J=64, keep=None, tol=1e-10,
                      max_restarts=2000, seed=0):
    """Top-k eigenpairs of a symmetric operator by thick-restart block Lanczos (FP64).

    ``matvec(X)`` returns M X for an n x c array.  The basis holds J columns; after a
    Rayleigh-Ritz step on T = Q^T M Q the ``keep`` leading Ritz vectors and the
    normalised residual block start the next cycle.  A Ritz pair (theta, Q y)
    has residual ||R_res E^T y||, with R_res the R factor of the residual block.
    Stops when the top-k residuals are <= tol * max|theta|.
    Returns (evals, evecs, info).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    keep = keep if keep is not None else max(k, J - 4 * b)
    X = rng.standard_normal((n, b))
    if X0 is not None:
        c = min(b, X0.shape[1])
        X[:, :c] = X0[:, :c] + 1e-3 * X[:, :c]
    Q0, _ = _orth_against(X, np.zeros((n, 0)), rng, 0.0)
    blocks = [Q0]
    T = np.zeros((0, 0))
    n_matvec = 0
    norm_est = 0.0
    theta = Y = None
    for restart in range(max_restarts):
        while True:
            Qall = np.hstack(blocks)
            c0 = Qall.shape[1] - b
            W = matvec(blocks[-1])
            n_matvec += b
            H = Qall.T @ W
            W = W - Qall @ H
            H2 = Qall.T @ W
            W = W - Qall @ H2
            H = H + H2
            Tn = np.zeros((Qall.shape[1], Qall.shape[1]))
            Tn[:c0, :c0] = T
            Tn[:, c0:] = H
            Tn[c0:, :] = H.T
            T = 0.5 * (Tn + Tn.T)
            norm_est = max(norm_est, np.abs(np.linalg.eigvalsh(T)).max())
            Qnext, R = _orth_against(W, np.zeros((n, 0)), rng, 1e-13 * max(norm_est, 1e-300))
            if Qall.shape[1] + b <= J:
                # Q_next must also be orthogonal to the whole basis (it is in exact arithmetic)
                Qnext, _ = _orth_against(Qnext, Qall, rng, 0.0)
                blocks.append(Qnext)
            else:
                break
        Qall = np.hstack(blocks)
        w, Yf = np.linalg.eigh(T)
        order = np.argsort(-w, kind="stable")
        theta, Y = w[order], Yf[:, order]
        res = np.linalg.norm(R @ Y[-b:, :], axis=0)
        scale = max(np.abs(theta).max(), 1e-300)
        if np.all(res[:k] <= tol * scale):
            break
        # thick restart: Ritz vectors + residual block
        U = Qall @ Y[:, :keep]
        Qres, _ = _orth_against(Qnext, U, rng, 0.0)
        blocks = [U[:, i:i + 1] for i in range(keep)]
        blocks = [np.hstack(blocks), Qres]
        # the first "block" is the keep Ritz vectors; the projected matrix is diag(theta)
        T = np.diag(theta[:keep])
        # re-express the block list so that blocks[-1] is the residual block of width b
    evecs = Qall @ Y[:, :k]
    info = {"restarts": restart, "matvecs": n_matvec, "residuals": res[:k],
            "converged": bool(np.all(res[:k] <= tol * scale))}
    return theta[:k].copy(), evecs, info


def top_eigenpairs(M, k, start=None, tol=1e-10, seed=0):
    """Top-k eigenpairs (descending) of a symmetric sparse or dense matrix M."""
    n = M.shape[0]
    if n <= DENSE_MAX_N:
        A = M.toarray() if sp.issparse(M) else np.asarray(M)
        if n <= JACOBI_MAX_N:
            w, V = jacobi_eigh(A)
            return w[:k].copy(), V[:, :k].copy()
        return dense_top(A, k)
    w, V, _ = block_lanczos_top(lambda X: M @ X, n, k, X0=start, tol=tol, seed=seed)
    return w, V
