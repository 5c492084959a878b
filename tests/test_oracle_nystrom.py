"""Pins of the oracle's Nystrom reconstruction (App. C, eq. nystrom_approx) and MaxCut
rounding (App. E) against definitions and facts that do not come from the oracle itself."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.nystrom import (cut_weight, maxcut_round, nystrom_matrix, nystrom_reconstruct,
                            rounding_values, sign_vector)
from paper_2312_11801_gb300 import instances as I
from tests._graphs import named_graph


def _psd(n, spectrum, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * np.asarray(spectrum, dtype=np.float64)) @ Q.T


@pytest.mark.parametrize("n,k,r", [(60, 3, 8), (200, 8, 8), (150, 1, 16)])
def test_exact_for_rank_at_most_r(n, k, r):
    """A PSD matrix of rank k <= r is recovered exactly from X Psi (the Nystrom
    approximation equals X on its range): error at rounding level."""
    rng = np.random.default_rng(n + k)
    F = rng.standard_normal((n, k))
    X = F @ F.T
    Psi = rng.standard_normal((n, r))
    Xh = nystrom_matrix(X @ Psi, Psi)
    assert np.linalg.norm(Xh - X) <= 1e-9 * np.linalg.norm(X)


def test_matches_pseudo_inverse_definition():
    """eq. nystrom_approx written out with a pseudo-inverse: P (Psi^T P)^+ P^T."""
    n, r = 80, 12
    X = _psd(n, 0.9 ** np.arange(n), 3)
    Psi = np.random.default_rng(4).standard_normal((n, r))
    P = X @ Psi
    ref = P @ np.linalg.pinv(Psi.T @ P) @ P.T
    got = nystrom_matrix(P, Psi)
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


def test_output_is_psd_with_orthonormal_factor():
    n, r = 120, 10
    X = _psd(n, np.linspace(1.0, 0.0, n) ** 3, 5)
    Psi = np.random.default_rng(6).standard_normal((n, r))
    U, lam = nystrom_reconstruct(X @ Psi, Psi)
    assert U.shape == (n, r) and lam.shape == (r,)
    assert np.all(lam >= 0.0) and np.all(np.diff(lam) <= 0.0)
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-10)


def test_expected_nuclear_error_bound():
    """The fact of App. C (Tropp et al. 2017): E ||X - X_hat||_* <= (1 + r'/(r - r' - 1))
    ||X - [[X]]_r'||_* for r' < r - 1, with Gaussian Psi.  The sample mean over 60 test
    matrices stays below the bound (10 % allowance for the sampling error)."""
    n, r, rp = 100, 12, 5
    spectrum = 0.7 ** np.arange(n)
    X = _psd(n, spectrum, 7)
    tail = float(np.sum(spectrum[rp:]))
    bound = (1.0 + rp / (r - rp - 1)) * tail
    rng = np.random.default_rng(8)
    errs = []
    for _ in range(60):
        Psi = rng.standard_normal((n, r))
        D = X - nystrom_matrix(X @ Psi, Psi)
        errs.append(np.sum(np.abs(np.linalg.eigvalsh(0.5 * (D + D.T)))))
    assert np.mean(errs) <= 1.1 * bound, (np.mean(errs), bound)


def test_rounding_value_is_cut_weight():
    """With C = L/4, <C, z z^T> = (1/4) z^T L z is the weight of the cut z."""
    n, ei, ej, w = 40, *I.complete_graph_edges(40)
    w = np.random.default_rng(9).uniform(0.5, 2.0, len(ei))
    C = sp.csr_matrix((np.concatenate([-w / 4, -w / 4]), (np.concatenate([ei, ej]), np.concatenate([ej, ei]))),
                      shape=(n, n))
    deg = np.zeros(n)
    np.add.at(deg, ei, w)
    np.add.at(deg, ej, w)
    C = C + sp.diags(deg / 4)
    U = np.random.default_rng(10).standard_normal((n, 6))
    vals = rounding_values(C, U)
    for k in range(6):
        assert abs(vals[k] - cut_weight(n, ei, ej, w, sign_vector(U[:, k]))) <= 1e-12 * max(1.0, vals[k])


@pytest.mark.parametrize("name", ["C12", "K3,4", "petersen", "Q3"])
def test_rounding_against_brute_force(name):
    """The rounded cut never beats the maximum cut (brute force over all 2^n sign
    vectors), and on a bipartite graph the sign of the top eigenvector of the SDP
    optimum zz^T finds it."""
    n, ei, ej, w = named_graph(name)
    prob = I.maxcut_from_edges(n, ei, ej, w)
    C = sp.csr_matrix((prob.C_val, prob.C_col, prob.C_rowptr), shape=(n, n))
    best = 0.0
    for bits in itertools.product((-1.0, 1.0), repeat=n - 1):
        z = np.array((1.0,) + bits)
        best = max(best, cut_weight(n, ei, ej, w, z))
    rng = np.random.default_rng(11)
    U = np.linalg.qr(rng.standard_normal((n, 4)))[0]
    val, k, z = maxcut_round(C, U)
    assert val <= best + 1e-12
    if name in ("C12", "K3,4", "Q3"):            # bipartite: X* = z z^T, z the 2-colouring
        side = np.zeros(n)
        adj = [[] for _ in range(n)]
        for a, b in zip(ei, ej):
            adj[a].append(b)
            adj[b].append(a)
        side[:] = np.nan
        side[0] = 1.0
        stack = [0]
        while stack:
            a = stack.pop()
            for b in adj[a]:
                if np.isnan(side[b]):
                    side[b] = -side[a]
                    stack.append(b)
        Xs = np.outer(side, side)
        Psi = rng.standard_normal((n, 4))
        Ub, lam = nystrom_reconstruct(Xs @ Psi, Psi)
        val2, _, _ = maxcut_round(C, Ub)
        assert abs(val2 - best) <= 1e-9 and abs(best - float(np.sum(w))) <= 1e-12


def test_fp32_sketch_uses_fp32_shift():
    """A sketch stored in FP32 (as the GPU keeps it) of a rank-5 matrix.  With the FP64
    spacing in the shift, Psi^T (P + nu Psi) is indefinite (the FP32 rounding of P is far
    larger than the shift).  With the FP32 spacing the reconstruction goes through; the
    shift, about n times the rounding it has to cover, then biases the small eigenvalues
    down: the top eigenvalue within 1 % and X within 2 % (Frobenius)."""
    rng = np.random.default_rng(12)
    n, k, r = 2000, 5, 16
    F = rng.standard_normal((n, k)) * 0.5 ** np.arange(k)
    X = F @ F.T / n
    Psi = rng.standard_normal((n, r)).astype(np.float32)
    P = (X @ Psi.astype(np.float64)).astype(np.float32)
    U, lam = nystrom_reconstruct(P, Psi)
    Xh = (U * lam) @ U.T
    assert np.linalg.norm(Xh - X) <= 2e-2 * np.linalg.norm(X)
    assert abs(lam[0] - np.linalg.eigvalsh(X)[-1]) <= 1e-2 * lam[0]
    Pd = P.astype(np.float64)
    nu64 = float(np.sqrt(n) * np.spacing(np.linalg.norm(Pd, 2)))
    B = Psi.astype(np.float64).T @ (Pd + nu64 * Psi.astype(np.float64))
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() < 0.0


def test_planted_transposed_factor_is_caught(monkeypatch):
    """Solving E R^T = Y instead of E R = Y (a transposed Cholesky factor) breaks the exact
    recovery of a low-rank matrix."""
    import oracle.nystrom as NY
    real = NY.sla.solve_triangular

    def planted(a, b, trans=0, lower=False, **kw):
        return real(a, b, trans=0 if trans == "T" else "T", lower=lower, **kw)
    monkeypatch.setattr(NY.sla, "solve_triangular", planted)
    with pytest.raises(AssertionError):
        test_exact_for_rank_at_most_r(60, 3, 8)
