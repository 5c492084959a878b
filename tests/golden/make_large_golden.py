"""Write tests/golden/oracle_large.json: FP64 oracle results for the full-size parity cases.

Calls only oracle/ and the input generators (paper_2312_11801_gb300.instances).  Cases:
  torus400_eig   top-8 eigenvalues of C - A*(y) on the 400 x 400 +-1 torus (n = 160,000)
                 at a seeded dual point (block Lanczos, App. E, to a 1e-11 residual);
  clust100k_eig  the same on a clustering SDP with n = 100,000 and 400,000 edge
                 inequalities (the off-diagonal A*(y) scatter);
  torus400_traj  cold start and six iterations of Algorithm 1 on the 400 x 400 torus
                 (k = 8, rho = 0.01, no sketch): per-step f(y), <C,X>, tr X, lambda_max,
                 relative infeasibility, model value and descent flag;
  er6000_solve   a solve of MaxCut on an Erdos-Renyi graph, n = 6000, average degree 6,
                 to both gates <= 1e-3 (rho = 0.03, at most 800 iterations).
Usage: python tests/golden/make_large_golden.py [case ...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import usbs as OU  # noqa: E402
from oracle.eig import block_lanczos_top  # noqa: E402
from paper_2312_11801_gb300 import instances as I  # noqa: E402

PATH = os.path.join(HERE, "oracle_large.json")

PROBLEMS = {
    "torus400": lambda: I.maxcut_torus(400, seed=7, signed=True),
    "clust100k": lambda: I.clustering_sdp(100_000, 400_000, seed=3),
    "er6000": lambda: I.maxcut_er(6000, 6.0, 2),
}


def eig_case(pname):
    prob = PROBLEMS[pname]()
    sp_ = OU.scale_problem(prob)
    y = I.dual_sample(prob, seed=11)
    M = OU.slack_matrix(sp_, y)
    t0 = time.time()
    w, _, info = block_lanczos_top(lambda X: M @ X, prob.n, 8, tol=1e-11)
    # ||M||_2 from the bottom of the spectrum too (the top is w[0])
    wb, _, _ = block_lanczos_top(lambda X: -(M @ X), prob.n, 1, tol=1e-8)
    return {"problem": pname, "n": prob.n, "m": prob.m, "dual_seed": 11, "evals": w.tolist(),
            "norm2": float(max(abs(w[0]), abs(wb[0]))), "residual_max": float(info["residuals"].max()),
            "restarts": int(info["restarts"]), "seconds": time.time() - t0}


def traj_case(pname, steps=6):
    prob = PROBLEMS[pname]()
    o = OU.USBSOracle(prob, k=8, rho=0.01)
    t0 = time.time()
    o.cold_start()
    rows = []
    for _ in range(steps):
        d = o.step()
        rows.append({"t": d["t"], "descent": int(d["descent"]), "f_y": d["f_y"], "cx": d["cx"],
                     "trx": d["trX"], "lambda_max": d["lambda_max"], "f_hat": d["f_hat"],
                     "relinf": d["relinf"], "relgap": d["relgap"]})
        print(pname, rows[-1], flush=True)
    return {"problem": pname, "n": prob.n, "k": 8, "rho": 0.01, "steps": rows,
            "seconds": time.time() - t0}


def solve_case(pname, tol=1e-3, max_iters=800, rho=0.03):
    prob = PROBLEMS[pname]()
    o = OU.USBSOracle(prob, k=8, rho=rho)
    t0 = time.time()

    def progress(d):
        if d["t"] % 25 == 0:
            print(pname, d["t"], d["relgap"], d["relinf"], round(time.time() - t0, 1), flush=True)

    hist = o.solve(tol=tol, max_iters=max_iters, callback=progress)
    last = hist[-1]
    return {"problem": pname, "n": prob.n, "rho": rho, "tol": tol, "iters": len(hist),
            "converged": bool(last["relgap"] <= tol and last["relinf"] <= tol),
            "objective": o.objective(), "dual_bound": o.dual_bound(),
            "cx_scaled": o.state.cx, "f_scaled": o.state.f_y, "relgap": last["relgap"],
            "relinf": last["relinf"], "seconds": time.time() - t0}


CASES = {
    "torus400_eig": lambda: eig_case("torus400"),
    "clust100k_eig": lambda: eig_case("clust100k"),
    "torus400_traj": lambda: traj_case("torus400"),
    "er6000_solve": lambda: solve_case("er6000"),
}

if __name__ == "__main__":
    out = os.environ.get("USBS_GOLDEN_OUT") or PATH
    data = json.load(open(out)) if os.path.exists(out) else {}
    for name in (sys.argv[1:] or list(CASES)):
        data[name] = CASES[name]()
        print(name, json.dumps(data[name])[:400], flush=True)
        json.dump(data, open(out, "w"), indent=1, sort_keys=True)
