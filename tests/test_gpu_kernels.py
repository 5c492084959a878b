"""Parity of the hot-path rows, each through the C ABI, against the FP64 oracle.

Sizes span several CTA tiles and a ragged tail; both precisions.  Tolerances: FP64
bulk 1e-12 relative; mixed (FP32 bulk) 2e-5 relative, from about 2^-24 per rounding
times the length of the longest accumulation chain seen here.
"""
import numpy as np
import pytest

from oracle import usbs as OU
from oracle.eig import top_eigenpairs
from paper_2312_11801_gb300 import instances as I
from tests.gpu_util import bulk_dtype, gpu_modules, rel_err

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-5}


def _cases():
    return {
        "er800": I.maxcut_er(800, 6.0, 0),
        "clust_ragged": I.clustering_sdp(1237, 5000, 2),
        "torus45": I.maxcut_torus(45, seed=1),
    }


@pytest.fixture(scope="module")
def mods():
    return gpu_modules()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["er800", "clust_ragged", "torus45"])
def test_matmul_operator(mods, case, precision):
    """a1 + a2: Y = (C - A*(y)) X with the A*(y) scatter and diagonal shift fused."""
    torch, U = mods
    prob = _cases()[case]
    rng = np.random.default_rng(5)
    sp_ = OU.scale_problem(prob)
    y = rng.standard_normal(prob.m) * 0.3
    X = rng.standard_normal((prob.n, 8))
    ref = OU.slack_matrix(sp_, y) @ X
    dt = bulk_dtype(torch, precision)
    with U.usbs_create(prob, precision=precision) as ctx:
        yd = torch.tensor(y, dtype=torch.float64, device="cuda")
        Xd = torch.tensor(X, dtype=dt, device="cuda")
        Yd = torch.empty_like(Xd)
        U.usbs_op_matmul(ctx, yd, Xd, Yd)
        torch.cuda.synchronize()
        got = Yd.double().cpu().numpy()
    assert rel_err(got, ref) <= TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["er800", "clust_ragged"])
def test_constraint_eval(mods, case, precision):
    """a9: z = A(V S V^T) from the factors."""
    torch, U = mods
    prob = _cases()[case]
    sp_ = OU.scale_problem(prob)
    rng = np.random.default_rng(6)
    V, _ = np.linalg.qr(rng.standard_normal((prob.n, 8)))
    S = rng.standard_normal((8, 8)); S = S + S.T
    dt = bulk_dtype(torch, precision)
    Vr = torch.tensor(V, dtype=dt).double().numpy()      # the rounded V the kernel sees
    ref = OU.A_lowrank(sp_, Vr, S)
    with U.usbs_create(prob, precision=precision) as ctx:
        z = torch.zeros(prob.m, dtype=torch.float64, device="cuda")
        U.usbs_op_constraint_eval(ctx, torch.tensor(V, dtype=dt, device="cuda"),
                                  torch.tensor(S, dtype=torch.float64, device="cuda"), z)
        torch.cuda.synchronize()
        got = z.cpu().numpy()
    assert rel_err(got, ref) <= TOL[precision] * 10


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("r", [16, 32])
def test_sketch_update(mods, precision, r):
    """a10: P <- eta P + V (S (V^T Psi))."""
    torch, U = mods
    prob = I.maxcut_er(2053, 6.0, 4)
    rng = np.random.default_rng(7)
    psi = I.gaussian_psi(prob.n, r, seed=3)
    V, _ = np.linalg.qr(rng.standard_normal((prob.n, 8)))
    S = rng.standard_normal((8, 8)); S = S @ S.T
    P0 = rng.standard_normal((prob.n, r)).astype(np.float32)
    eta = 0.37
    dt = bulk_dtype(torch, precision)
    Vr = torch.tensor(V, dtype=dt).double().numpy()
    ref = eta * P0.astype(np.float64) + Vr @ (S @ (Vr.T @ psi.astype(np.float64)))
    with U.usbs_create(prob, psi=psi, r=r, precision=precision) as ctx:
        Pd = torch.tensor(P0, device="cuda")
        U.usbs_op_sketch_update(ctx, torch.tensor(V, dtype=dt, device="cuda"),
                                torch.tensor(S, dtype=torch.float64, device="cuda"),
                                torch.tensor(psi, device="cuda"), Pd, eta)
        torch.cuda.synchronize()
        got = Pd.double().cpu().numpy()
    assert rel_err(got, ref) <= 2e-5       # P is FP32 in both modes


def _eig_gate(got, ref, normM, tol):
    return np.abs(np.asarray(got) - np.asarray(ref)) <= tol * np.maximum(np.abs(ref), normM)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case,ywhich", [("er800", "zero"), ("er800", "rand"),
                                         ("clust_ragged", "rand"), ("torus45", "rand")])
def test_extreme_eigs(mods, case, ywhich, precision):
    """a2-a4: block Lanczos top-k eigenvalues within 1e-5 (mixed) / 1e-9 (FP64) of the
    oracle, relative to max(|lambda|, ||M||_2); eigenvector residuals checked in FP64."""
    torch, U = mods
    prob = _cases()[case]
    sp_ = OU.scale_problem(prob)
    rng = np.random.default_rng(11)
    y_s = np.zeros(prob.m) if ywhich == "zero" else np.abs(rng.standard_normal(prob.m)) * 0.05 / np.sqrt(prob.n)
    M = OU.slack_matrix(sp_, y_s)
    w_ref, _ = top_eigenpairs(M, 8)
    normM = np.abs(np.linalg.eigvalsh(M.toarray())).max()
    tol = 1e-9 if precision == 0 else 1e-5
    ltol = 1e-11 if precision == 0 else 1e-6
    with U.usbs_create(prob, precision=precision, lanczos_restarts=300, lanczos_tol=ltol) as ctx:
        evals, evecs, info = U.usbs_extreme_eigs(ctx, y=y_s * sp_.c_scale)
    assert np.all(_eig_gate(evals, w_ref, normM, tol)), (evals - w_ref, info)
    res = np.linalg.norm(M @ evecs - evecs * evals, axis=0)
    assert res.max() <= (1e-8 if precision == 0 else 3e-5) * normM
    np.testing.assert_allclose(evecs.T @ evecs, np.eye(8), atol=1e-9 if precision == 0 else 2e-5)


def test_tf32_rounding_matches_the_ptx_conversion(mods):
    """The FP32 tiles split every operand into TF32 high and low parts; their rounding (two
    integer operations on the bit pattern) must give the bits of cvt.rna.tf32.f32 (nearest,
    ties away from zero) for finite normal inputs and zeros: random bit patterns over the
    normal exponent range, values with exact ties (dropped bits 0x1000), ties one bit off
    either way, values whose rounding carries into the exponent, and +-0."""
    torch, U = mods
    rng = np.random.default_rng(3)
    sign = rng.integers(0, 2, 200_000, dtype=np.uint32) << 31
    expo = rng.integers(1, 254, 200_000, dtype=np.uint32) << 23
    mant = rng.integers(0, 1 << 23, 200_000, dtype=np.uint32)
    bits = sign | expo | mant
    ties = (bits & ~np.uint32(0x1FFF)) | np.uint32(0x1000)
    near = np.concatenate([ties - np.uint32(1), ties + np.uint32(1)])
    carry = (sign[:1000] | expo[:1000] | np.uint32(0x7FF000))
    allb = np.concatenate([bits, ties, near, carry, np.array([0, 0x80000000], np.uint32)])
    x = allb.view(np.float32)
    ours, ref = U.usbs_selftest_tf32_round(x)
    bad = np.nonzero(ours != ref)[0]
    assert bad.size == 0, [(hex(allb[i]), hex(ours[i]), hex(ref[i])) for i in bad[:5]]
    # the high part keeps 10 mantissa bits and is within half a TF32 unit of x
    hi = ours.view(np.float32).astype(np.float64)
    assert np.all((ours & np.uint32(0x1FFF)) == 0)
    assert np.all(np.abs(hi - x) <= np.abs(x) * 2.0 ** -11 * (1 + 1e-12))
