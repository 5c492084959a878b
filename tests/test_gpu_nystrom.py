"""Nystrom reconstruction of the primal and MaxCut rounding (App. C, eq. nystrom_approx;
App. E, rounding) through the C ABI, against the FP64 oracle and a closed form."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.nystrom import nystrom_reconstruct, rounding_values
from paper_2312_11801_gb300 import instances as I
from tests.gpu_util import gpu_modules

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    return gpu_modules()


def _C(prob):
    return sp.csr_matrix((prob.C_val, prob.C_col, prob.C_rowptr), shape=(prob.n, prob.n))


@pytest.mark.parametrize("precision", [0, 1])
def test_reconstruction_and_rounding_match_oracle(mods, precision):
    """n = 256, a power of two: the MaxCut trace n scales the sketch exactly, so the oracle
    run on the problem-unit sketch sees the GPU's own numbers.  Eigenvalues within 1e-9 of
    the largest; the top factor columns agree up to sign; every column's rounding value
    equals <C, z z^T> of the GPU's own sign vector."""
    torch, U_ = mods
    prob = I.maxcut_er(256, 6.0, 5)
    r = 16
    psi = I.gaussian_psi(prob.n, r, seed=3)
    with U_.usbs_create(prob, psi=psi, r=r, precision=precision, rho=0.1) as ctx:
        for _ in range(40):
            U_.usbs_step(ctx)
        lam, Ug, vals, best, z = U_.usbs_nystrom_round(ctx)
        P, Psi, _ = U_.usbs_get_sketch(ctx)
    Uo, lo = nystrom_reconstruct(P, Psi)
    assert np.all(np.abs(lam - lo) <= 1e-9 * lo[0]), (lam[:6], lo[:6])
    top = lo > 1e-4 * lo[0]
    cosines = np.abs(np.sum(Uo[:, top] * Ug[:, top], axis=0))
    gaps = np.abs(np.diff(lo))
    sep = np.array([min(gaps[k - 1] if k else np.inf, gaps[k] if k < len(gaps) else np.inf)
                    for k in range(len(lo))])[top] > 1e-3 * lo[0]
    assert np.all(cosines[sep] >= 1.0 - 1e-8), cosines
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(r), atol=1e-8)
    ref_vals = rounding_values(_C(prob), Ug)
    np.testing.assert_allclose(vals, ref_vals, rtol=1e-12, atol=1e-9)
    assert best == int(np.argmax(vals))
    np.testing.assert_array_equal(z, np.where(Ug[:, best] >= 0.0, 1, -1))


def test_bipartite_torus_rounds_to_the_maximum_cut(mods):
    """A bipartite graph's MaxCut SDP optimum is z z^T for its 2-colouring z, and the
    maximum cut is every edge: the rounded cut of a converged solve is |E| = 2 n."""
    torch, U_ = mods
    prob = I.maxcut_torus(8, signed=False)
    psi = I.gaussian_psi(prob.n, 4, seed=4)
    with U_.usbs_create(prob, psi=psi, r=4, rho=0.1, lanczos_basis=32, max_iters=3000) as ctx:
        res = U_.usbs_solve(ctx, tol=1e-4)
        lam, _, vals, best, z = U_.usbs_nystrom_round(ctx, want_u=False)
    assert res["converged"]
    assert abs(vals[best] - 2.0 * prob.n) <= 1e-9 * prob.n
    assert lam[0] >= 0.99 * prob.n and np.all(lam[1:] <= 1e-2 * prob.n)


def test_requires_a_sketch(mods):
    torch, U_ = mods
    prob = I.maxcut_er(100, 6.0, 1)
    with U_.usbs_create(prob) as ctx:
        with pytest.raises(U_.USBSError):
            U_.usbs_nystrom_round(ctx)
