"""svec, U and the symmetric Kronecker product (App. B, preamble).

Test infrastructure only (see ``oracle/__init__``).

``svec`` stacks the lower triangle column by column, off-diagonal entries scaled by
sqrt(2), so that <A, B> = svec(A)^T svec(B).  ``vec`` stacks columns.  ``U`` maps
vec(A) to svec(A) for symmetric A and has orthonormal rows.  The symmetric Kronecker
product is defined by its action (G (x)_s H) svec(A) = 1/2 svec(H A G^T + G A H^T),
and equivalently by 1/2 U (G (x) H + H (x) G) U^T; the paper's implementation uses the
second form, and so does ``skron``.
"""
import math

import numpy as np

SQRT2 = math.sqrt(2.0)


def svec_dim(k):
    return k * (k + 1) // 2


def svec_index(i, j, k):
    """Position of entry (i, j), i >= j, in svec of a k x k matrix (0-based)."""
    if i < j:
        i, j = j, i
    return j * k - j * (j - 1) // 2 + (i - j)


def svec(A):
    k = A.shape[0]
    out = np.empty(svec_dim(k))
    p = 0
    for j in range(k):
        out[p] = A[j, j]
        p += 1
        for i in range(j + 1, k):
            out[p] = SQRT2 * A[i, j]
            p += 1
    return out


def smat(s):
    """Inverse of svec."""
    K = s.shape[0]
    k = int(round((math.sqrt(8 * K + 1) - 1) / 2))
    A = np.empty((k, k))
    p = 0
    for j in range(k):
        A[j, j] = s[p]
        p += 1
        for i in range(j + 1, k):
            A[i, j] = A[j, i] = s[p] / SQRT2
            p += 1
    return A


def vec(A):
    return A.reshape(-1, order="F").copy()


def U_matrix(k):
    """The (k(k+1)/2) x k^2 matrix with U vec(A) = svec(A) for symmetric A."""
    U = np.zeros((svec_dim(k), k * k))
    for j in range(k):
        for i in range(j, k):
            row = svec_index(i, j, k)
            for l in range(k):          # column index of vec entry a_{kk,l}
                for kk in range(k):
                    col = l * k + kk
                    if i == j == kk == l:
                        U[row, col] = 1.0
                    elif i != j and ((i == kk and j == l) or (i == l and j == kk)):
                        U[row, col] = 1.0 / SQRT2
    return U


def skron(G, H):
    """G (x)_s H = 1/2 U (G (x) H + H (x) G) U^T."""
    U = U_matrix(G.shape[0])
    return 0.5 * U @ (np.kron(G, H) + np.kron(H, G)) @ U.T


def skron_action(G, H, A):
    """(G (x)_s H) svec(A) = 1/2 svec(H A G^T + G A H^T)."""
    return 0.5 * svec(H @ A @ G.T + G @ A @ H.T)
