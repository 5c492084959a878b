"""Pins for oracle/eig.py: Jacobi and block Lanczos against LAPACK and closed forms."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import eig as E


@pytest.mark.parametrize("n", [2, 5, 16, 40])
def test_jacobi_matches_lapack(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)); A = A + A.T
    w, V = E.jacobi_eigh(A)
    np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(A))[::-1], atol=1e-12 * np.abs(w).max())
    np.testing.assert_allclose(A @ V, V * w, atol=1e-11 * np.abs(w).max())
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-12)


def test_jacobi_repeated_eigenvalue_complete_graph():
    n = 7
    L = n * np.eye(n) - np.ones((n, n))            # Laplacian of K_n: eigenvalues n (x n-1), 0
    w, V = E.jacobi_eigh(L)
    np.testing.assert_allclose(w, [n] * (n - 1) + [0.0], atol=1e-12)


def _sparse_sym(n, nnz_per_row, seed):
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n), nnz_per_row)
    cols = rng.integers(0, n, size=n * nnz_per_row)
    vals = rng.standard_normal(n * nnz_per_row)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return (A + A.T).tocsr()


def test_block_lanczos_matches_lapack():
    n, k = 1500, 8
    A = _sparse_sym(n, 4, 1)
    w, V, info = E.block_lanczos_top(lambda X: A @ X, n, k, tol=1e-11)
    ref = np.sort(np.linalg.eigvalsh(A.toarray()))[::-1][:k]
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    np.testing.assert_allclose(A @ V, V * w, atol=1e-8 * np.abs(ref).max())
    assert info["converged"]


def test_block_lanczos_finds_multiple_top_eigenvalue():
    n = 800
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = np.concatenate([[5.0, 5.0, 5.0], np.linspace(4.0, -3.0, n - 3)])
    A = (Q * d) @ Q.T
    w, V, info = E.block_lanczos_top(lambda X: A @ X, n, 5, tol=1e-11)
    np.testing.assert_allclose(w[:3], 5.0, atol=1e-9)
    np.testing.assert_allclose(w[3:], d[3:5], atol=1e-8)


def test_jacobi_vs_lanczos_small():
    n = 60
    A = _sparse_sym(n, 3, 4)
    wj, _ = E.jacobi_eigh(A.toarray())
    wl, _, _ = E.block_lanczos_top(lambda X: A @ X, n, 4, b=4, J=32, tol=1e-12)
    np.testing.assert_allclose(wl, wj[:4], atol=1e-10 * np.abs(wj).max())


def test_top_eigenpairs_dispatch():
    for n in (10, 100):
        A = _sparse_sym(n, 3, n)
        w, V = E.top_eigenpairs(A, 3)
        ref = np.sort(np.linalg.eigvalsh(A.toarray()))[::-1][:3]
        np.testing.assert_allclose(w, ref, atol=1e-11 * np.abs(ref).max())
