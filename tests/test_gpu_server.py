"""Batched and served solves on the GPU, and the warm start of a grown instance (Sec. 5.1).

The kernels reduce in a fixed order and every context owns its buffers, so a solve that
runs beside others on its own stream must reproduce the solve of the same instance run
alone, iteration for iteration.
"""
import time

import numpy as np
import pytest

from paper_2312_11801_gb300 import instances as I
from tests.gpu_util import gpu_modules

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module")
def mods():
    return gpu_modules()


CAP = 600
# random geometric graphs of a few hundred vertices need thousands of iterations at the
# paper's rho = 0.01 to reach 1e-3, and about 200 at rho = 0.1
RHO_RGG = 0.1


def _probs():
    return [I.maxcut_torus(side, seed=side, signed=True) for side in (12, 14, 16, 18)]


def _solo(U, prob, **kw):
    with U.usbs_create(prob, max_iters=CAP, **kw) as ctx:
        return U.usbs_solve(ctx, tol=TOL)


def test_batch_pool_matches_solo(mods):
    """Contexts the persistent kernel does not take (here a J = 16 basis) are solved by a
    pool of per-step solves on their own streams: identical to solving each alone."""
    torch, U = mods
    probs = _probs()
    solo = [_solo(U, p, lanczos_basis=16) for p in probs]
    ctxs = [U.usbs_create(p, max_iters=CAP, lanczos_basis=16) for p in probs]
    try:
        res, st = U.usbs_batch_solve(ctxs, tol=TOL, max_concurrency=4)
    finally:
        for c in ctxs:
            c.close()
    for a, b, s in zip(solo, res, st):
        assert s in (U.USBS_OK, U.USBS_ENOTCONV)
        assert b["iters"] == a["iters"] and b["converged"] == a["converged"]
        assert b["last"]["objective"] == a["last"]["objective"]
        assert b["last"]["dual_bound"] == a["last"]["dual_bound"]


def test_server_matches_solo(mods):
    torch, U = mods
    probs = _probs()
    solo = [_solo(U, p) for p in probs]
    with U.usbs_server_create(max_slots=3, cache_entries=2, solver={"r": 0, "max_iters": CAP}) as srv:
        for i, p in enumerate(probs):
            U.usbs_server_submit(srv, i, p, tol=TOL)
        done, t0 = [], time.time()
        while len(done) < len(probs) and time.time() - t0 < 120:
            done += U.usbs_server_poll(srv, 16, wait_ms=100)
        st = U.usbs_server_get_stats(srv)
    assert len(done) == len(probs)
    for c in done:
        a = solo[c["request_id"]]
        assert c["status"] in (U.USBS_OK, U.USBS_ENOTCONV) and c["warm"] == 0
        assert c["iters"] == a["iters"]
        assert c["objective"] == a["last"]["objective"]
    assert st["peak_running"] >= 2 and st["cached"] == 2


def _state_from_oracle(o, kc=8):
    """The oracle's iterate as usbs_set_state's vector (problem units)."""
    st, sp_ = o.state, o.sp
    c, tau = sp_.c_scale, sp_.tau
    V = np.zeros((sp_.n, kc))
    V[:, :st.V.shape[1]] = st.V
    return np.concatenate([st.y * c, st.ax * tau, [st.cx * c * tau, st.tr * tau, st.f_y * c * tau],
                           V.ravel()])


def test_grow_matches_oracle_warm_start(mods):
    """usbs_grow against the oracle's warm start (Sec. 5.1, reading R10): the GPU parent
    is loaded with the oracle's solved iterate, both grow the instance by 1 % new points,
    and the warm-started FP64 iterations agree step by step."""
    torch, U = mods
    from oracle.usbs import USBSOracle, warm_start
    parent = I.maxcut_rgg(400, 10.0, seed=5)
    child = I.grow_rgg(parent, frac=0.01, seed=6)
    o = USBSOracle(parent, k=8, rho=RHO_RGG)
    o.solve(tol=1e-3, max_iters=400)
    ow = warm_start(o, child)
    with U.usbs_create(parent, precision=0, rho=RHO_RGG, lanczos_restarts=300,
                       lanczos_tol=1e-12) as pc:
        U.usbs_set_state(pc, _state_from_oracle(o))
        y0 = U.usbs_get_dual(pc)
        cc = U.usbs_grow(pc, child)
    with cc:
        y1 = U.usbs_get_dual(cc)
        # old constraints keep their dual values; new ones start at zero
        assert np.allclose(y1[: parent.m], y0, rtol=1e-12, atol=1e-14 * np.abs(y0).max())
        assert np.all(y1[parent.m:] == 0.0)
        st = U.usbs_get_state(cc)
        c, tau = ow.sp.c_scale, ow.sp.tau
        m = child.m
        assert abs(st[2 * m] - ow.state.cx * c * tau) <= 1e-9 * (1 + abs(st[2 * m]))
        assert abs(st[2 * m + 1] - ow.state.tr * tau) <= 1e-9 * (1 + abs(st[2 * m + 1]))
        assert abs(st[2 * m + 2] - ow.state.f_y * c * tau) <= 1e-8 * (1 + abs(st[2 * m + 2]))
        # three steps: later ones drift apart at the 1e-5 level as rounding differences in
        # the eigen solves grow (the pre-growth state and these steps agree to 1e-6)
        for t in range(3):
            g = U.usbs_step(cc)
            r = ow.step()
            assert g["descent"] == int(r["descent"]), t
            for kg, ko in [("f_y", "f_y"), ("cx", "cx"), ("trx", "trX"), ("relinf", "relinf")]:
                assert abs(g[kg] - r[ko]) <= 1e-6 * (1 + abs(r[ko])), (t, kg, g[kg], r[ko])


def test_server_warm_start_from_parent(mods):
    """A request naming a finished request as its parent is grown from the resident
    instance: the same result, bit for bit, as usbs_grow and a warm usbs_solve on a
    parent solved the same way outside the server."""
    torch, U = mods
    parent = I.maxcut_rgg(400, 10.0, seed=5)
    child = I.grow_rgg(parent, frac=0.01, seed=6)
    with U.usbs_server_create(max_slots=2, cache_entries=4,
                              solver={"r": 0, "max_iters": CAP, "rho": RHO_RGG}) as srv:
        U.usbs_server_submit(srv, 1, parent, tol=TOL)
        first = U.usbs_server_poll(srv, 4, wait_ms=60000)
        U.usbs_server_submit(srv, 2, child, parent_id=1, tol=TOL)
        second = U.usbs_server_poll(srv, 4, wait_ms=60000)
    assert len(first) == 1 and len(second) == 1
    c = second[0]
    assert c["request_id"] == 2 and c["warm"] == 1
    assert c["status"] in (U.USBS_OK, U.USBS_ENOTCONV)
    with U.usbs_create(parent, max_iters=CAP, rho=RHO_RGG) as pc:
        U.usbs_solve(pc, tol=TOL)
        cc = U.usbs_grow(pc, child)
    with cc:
        w = U.usbs_solve(cc, warm_start=True, tol=TOL)
    assert c["iters"] == w["iters"]
    assert c["objective"] == w["last"]["objective"]
    assert c["dual_bound"] == w["last"]["dual_bound"]
