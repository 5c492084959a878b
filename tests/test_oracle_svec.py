"""Pins for oracle/svec.py (App. B preamble): svec, U, symmetric Kronecker product."""
import numpy as np
import pytest

from oracle import svec as SV


def _sym(rng, k):
    A = rng.standard_normal((k, k))
    return A + A.T


def test_U_matches_printed_example(golden_dir):
    U_paper = np.loadtxt(f"{golden_dir}/svec_U_k2.txt")
    np.testing.assert_allclose(SV.U_matrix(2), U_paper, atol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_svec_inner_product_and_U(k):
    rng = np.random.default_rng(k)
    A, B = _sym(rng, k), _sym(rng, k)
    # <A, B> = tr(AB) = svec(A)^T svec(B)
    assert np.isclose(np.trace(A @ B), SV.svec(A) @ SV.svec(B), rtol=1e-13)
    U = SV.U_matrix(k)
    np.testing.assert_allclose(U @ U.T, np.eye(SV.svec_dim(k)), atol=1e-14)     # orthonormal rows
    np.testing.assert_allclose(U @ SV.vec(A), SV.svec(A), atol=1e-13)
    np.testing.assert_allclose(U.T @ SV.svec(A), SV.vec(A), atol=1e-13)         # U^T U vec = vec
    np.testing.assert_allclose(SV.smat(SV.svec(A)), A, atol=1e-14)


def test_svec_order_is_column_wise_lower_triangle():
    A = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 5.0], [3.0, 5.0, 6.0]])
    r2 = np.sqrt(2.0)
    np.testing.assert_allclose(SV.svec(A), [1, r2 * 2, r2 * 3, 4, r2 * 5, 6])


@pytest.mark.parametrize("k", [2, 3, 4, 8])
def test_skron_two_definitions_agree(k):
    rng = np.random.default_rng(10 + k)
    G, H, A = rng.standard_normal((k, k)), rng.standard_normal((k, k)), _sym(rng, k)
    np.testing.assert_allclose(SV.skron(G, H) @ SV.svec(A), SV.skron_action(G, H, A),
                               rtol=1e-12, atol=1e-12)


def test_skron_of_pd_pair_is_symmetric_pd():
    rng = np.random.default_rng(3)
    k = 4
    X = rng.standard_normal((k, k)); T = X @ X.T + np.eye(k)
    Y = rng.standard_normal((k, k)); S = Y @ Y.T + np.eye(k)
    M = SV.skron(T, np.linalg.inv(S))
    np.testing.assert_allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(M).min() > 0


def test_planted_missing_sqrt2_is_caught(monkeypatch):
    """A dropped sqrt(2) in svec breaks the inner-product pin."""
    monkeypatch.setattr(SV, "SQRT2", 1.0)
    rng = np.random.default_rng(0)
    A, B = _sym(rng, 3), _sym(rng, 3)
    assert not np.isclose(np.trace(A @ B), SV.svec(A) @ SV.svec(B), rtol=1e-6)
