"""usbs_sketch_update_static, the sketch update for callers that cannot allocate.

Some callers cannot call cudaMalloc (a serving process whose memory pool owns all of
HBM, or code that must not take the synchronisation an allocation may cause), so the
library offers one entry point whose scratch is a static device array.  This test
checks it against usbs_op_sketch_update, the context-based entry point that allocates
its scratch at usbs_create, on two calls in a row with different sketch ranks, so a
larger call's leftover scratch must not leak into the next one.  The file is named to
be collected last.
"""
import numpy as np
import pytest

from paper_2312_11801_gb300 import instances as I
from tests.gpu_util import gpu_modules, rel_err

pytestmark = pytest.mark.gpu


def test_static_sketch_update_matches_context_entry_point():
    torch, U = gpu_modules()
    prob = I.maxcut_er(2053, 6.0, 4)
    rng = np.random.default_rng(21)
    n = prob.n
    V, _ = np.linalg.qr(rng.standard_normal((n, 8)))
    Vd = torch.tensor(V, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    for call, (r, eta) in enumerate([(32, 0.37), (16, 1.25)]):
        psi = I.gaussian_psi(n, r, seed=3 + call)
        S = rng.standard_normal((8, 8)); S = S @ S.T
        P0 = rng.standard_normal((n, r)).astype(np.float32)
        Sd = torch.tensor(S, dtype=torch.float64, device="cuda")
        Psid = torch.tensor(psi, device="cuda")
        with U.usbs_create(prob, psi=psi, r=r, precision=U.PRECISION_MIXED) as ctx:
            P_ctx = torch.tensor(P0, device="cuda")
            U.usbs_op_sketch_update(ctx, Vd, Sd, Psid, P_ctx, eta)
            torch.cuda.synchronize()
        P_static = torch.tensor(P0, device="cuda")
        torch.cuda.synchronize()
        U.usbs_sketch_update_static(n, r, Vd, Sd, Psid, P_static, eta, stream=stream)
        stream.synchronize()
        got, ref = P_static.double().cpu().numpy(), P_ctx.double().cpu().numpy()
        assert rel_err(got, ref) <= 2e-5, (call, rel_err(got, ref))
        # and the update itself, from its definition with the FP32-rounded V
        Vr = Vd.double().cpu().numpy()
        dense = eta * P0.astype(np.float64) + Vr @ (S @ (Vr.T @ psi.astype(np.float64)))
        assert rel_err(got, dense) <= 2e-5, (call, rel_err(got, dense))


def test_static_sketch_update_rejects_oversized_rank():
    torch, U = gpu_modules()
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    s = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(U.USBSError) as ei:
        U.usbs_sketch_update_static(8, 33, x, s, x, x, 1.0)
    assert ei.value.code == U.USBS_EINVAL
