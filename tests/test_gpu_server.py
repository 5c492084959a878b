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


def test_grow_keeps_dual_and_warm_solve_agrees(mods):
    torch, U = mods
    parent = I.maxcut_rgg(400, 10.0, seed=5)
    child = I.grow_rgg(parent, frac=0.01, seed=6)
    with U.usbs_create(parent, max_iters=CAP, rho=RHO_RGG) as pc:
        pres = U.usbs_solve(pc, tol=TOL)
        assert pres["converged"]
        y0 = U.usbs_get_dual(pc)
        cc = U.usbs_grow(pc, child)
    with cc:
        y1 = U.usbs_get_dual(cc)
        # old constraints keep their dual values; new ones start at zero
        assert np.allclose(y1[: parent.m], y0, rtol=1e-12, atol=1e-14 * np.abs(y0).max())
        assert np.all(y1[parent.m:] == 0.0)
        warm = U.usbs_solve(cc, warm_start=True, tol=TOL)
    cold = _solo(U, child, rho=RHO_RGG)
    assert warm["converged"] and cold["converged"]
    ow, oc = warm["last"]["objective"], cold["last"]["objective"]
    assert abs(ow - oc) <= 4 * TOL * (1 + abs(oc))


def test_server_warm_start_from_parent(mods):
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
    assert c["request_id"] == 2 and c["warm"] == 1 and c["status"] == U.USBS_OK
    cold = _solo(U, child, rho=RHO_RGG)
    assert abs(c["objective"] - cold["last"]["objective"]) <= 4 * TOL * (1 + abs(cold["last"]["objective"]))
