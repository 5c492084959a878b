#!/usr/bin/env python
"""USBS solves/sec on GB300: MaxCut SDP on the 1000 x 1000 toroidal grid.

Workload (one "step"): a cold-start USBS solve of MaxCut on the 1000 x 1000 torus
(n = 1,000,000 vertices, 2,000,000 edges, weights +-1 with probability 1/2, seed 0)
with a rank-16 Nystrom sketch (Gaussian Psi, seed 1), k_c = 8, mixed precision (FP32
bulk, FP64 k-sized work), thick-restart block Lanczos with a 32-column basis and at most
10 restarts (the paper's eigen solver budget, App. E), until both the relative gap and
the relative infeasibility are <= 1e-3 (scaled units, the paper's gates).  The line also
reports f(y) at the final y from a longer eigen solve and the gap relative to the
objective, since at n = 1e6 the paper's 1 + |<C,X>| denominator makes its gate loose.  Inputs are synthetic; the problem data
(~100 MB) and the Lanczos basis (~290 MB) exceed the 126 MB L2, so no flush is needed.

`value` times usbs_solve with the problem already resident in HBM; `e2e` times, per
step, usbs_create from pinned host arrays (H2D inside), the solve, and the read-back of
y and the sketch.  Several GPUs run independent replicas (no collective).

--impl reference times the FP64 CPU oracle on a bounded sample (see cpu_baseline).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "solves/sec at gap<=1e-3: served vs plain (same GPU); Lanczos HBM GB/s; p99"
UNIT = "solves/sec"
TOL = 1e-3
SIDE, R_SKETCH = 1000, 16
WORKLOAD = "maxcut_torus_1000x1000_pm1_r16_mixed"
# DRAM bytes of one k_tupdate launch against its algorithmic bytes, from the ncu capture
# summarised in profiles/k_tupdate_c2_torus1000.md (nb = 4, n = 1e6); the bench scales the
# ratio to the average algorithmic bytes per launch of its own run
TUPDATE_TRAFFIC = {"dram_bytes": 174.96e6, "algorithmic_bytes": 192.0e6}
KERNEL_OF_KIND = {"spmm": "k_spmm", "reorth": "k_tproj", "reorth_update": "k_tupdate",
                  "reorth_final": "k_tfinalize", "restart": "k_trestart", "reduce": "k_reduce",
                  "constraint": "k_gstats+k_xupdate+k_alt", "sketch": "k_vt_psi+k_sketch_update"}


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_problem(side=SIDE):
    from paper_2312_11801_gb300 import instances as I
    prob = I.maxcut_torus(side, seed=0, signed=True)
    psi = I.gaussian_psi(prob.n, R_SKETCH, seed=1)
    return prob, psi


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 7
                          for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x):
    """The largest x over the ranks (the timing rule: max over ranks).  NCCL reduces a
    device tensor, gloo (the CPU tests of this path) a host one."""
    if pg is None:
        return x
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------------------
SAMPLE_SIDE = 200        # a 200 x 200 torus of the same family (n = 40,000, block Lanczos path)
SAMPLE_ITERS = 2


def oracle_sample(gpu_iters_per_solve, budget_s=40.0):
    """Oracle seconds per USBS iteration on the sample, scaled to the full workload.

    The sample runs the oracle (as it stands: block Lanczos to a 1e-6 residual for
    n > 4096, FP64 throughout) on a 200 x 200 torus with the same weights law and sketch
    rank, for up to SAMPLE_ITERS iterations after its cold start (10-30 s of CPU work).
    Every step of an iteration is linear in n for these graphs, so seconds per iteration
    are scaled by 1e6 / 40,000; solves/sec divides by the iterations the GPU solve needed.
    """
    from paper_2312_11801_gb300 import instances as I
    from oracle.usbs import USBSOracle
    prob = I.maxcut_torus(SAMPLE_SIDE, seed=0, signed=True)
    psi = I.gaussian_psi(prob.n, R_SKETCH, seed=1)
    o = USBSOracle(prob, k=8, psi=psi, eig_tol=1e-6)
    t0 = time.perf_counter()
    o.cold_start()
    t1 = time.perf_counter()
    done = 0
    while done < SAMPLE_ITERS and time.perf_counter() - t1 < budget_s:
        o.step()
        done += 1
    t2 = time.perf_counter()
    per_iter = (t2 - t1) / max(done, 1)
    scale = (SIDE * SIDE) / prob.n
    per_solve = scale * (per_iter * max(gpu_iters_per_solve, 1) + (t1 - t0))
    try:
        import threadpoolctl
        cores = max(info.get("num_threads", 1) for info in threadpoolctl.threadpool_info()) or 1
    except Exception:
        cores = os.cpu_count()
    return {"value": 1.0 / per_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"FP64 oracle: cold start + {done} USBS iterations on the "
                       f"{SAMPLE_SIDE}x{SAMPLE_SIDE} +-1 torus (n={prob.n}, r=16), "
                       f"{per_iter:.3f} s/iteration, scaled x{scale:.0f} in n and by "
                       f"{gpu_iters_per_solve} iterations per solve"),
            "seconds": t2 - t0}


# ---------------------------------------------------------------------------------------
def run_ours(args, world, rank, local, pg):
    import torch
    from paper_2312_11801_gb300 import build as B
    B.build()
    from paper_2312_11801_gb300 import usbs as U

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    prob, psi = make_problem(args.side)
    stream = torch.cuda.Stream(device=dev)
    params = dict(r=R_SKETCH, precision=U.PRECISION_MIXED, stream=stream, max_iters=args.max_iters,
                  lanczos_basis=args.lanczos_basis, lanczos_tol=args.lanczos_tol,
                  certify_restarts=args.certify_restarts)
    ctx = U.usbs_create(prob, psi=psi, **params)

    # warm-up solves (also give the iteration count of one solve)
    warm = []
    for _ in range(args.warmup):
        warm.append(U.usbs_solve(ctx, warm_start=False, tol=TOL))

    # timed region: per-launch event timing off (it adds host work to every launch)
    clocks = ClockSampler(local)
    clocks.start()
    U.usbs_profile(ctx, False)
    launches0 = U.usbs_launch_count(ctx)
    results = []
    barrier(pg)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        results.append(U.usbs_solve(ctx, warm_start=False, tol=TOL))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    elapsed = e0.elapsed_time(e1) / 1e3
    launches = U.usbs_launch_count(ctx) - launches0
    clk = clocks.stop()
    elapsed_max = max_over_ranks(pg, elapsed)

    # kernel timing pass: the same solves with every launch bracketed by CUDA events on
    # the solve's stream; per-kind device time, launches and algorithmic bytes
    U.usbs_profile(ctx, True)
    for _ in range(max(args.profile_steps, 1)):
        U.usbs_solve(ctx, warm_start=False, tol=TOL)
    stats = U.usbs_kernel_stats(ctx)
    U.usbs_profile(ctx, False)

    # end to end through the C ABI from pinned host arrays
    arrays = U._problem_arrays(prob)
    pinned = []
    for a in list(arrays) + [np.ascontiguousarray(psi, np.float32)]:
        t = torch.from_numpy(a).pin_memory()
        pinned.append(t.numpy())
    h2d = sum(a.nbytes for a in pinned)
    d2h = 8 * prob.m + 4 * prob.n * R_SKETCH + 16
    from paper_2312_11801_gb300.instances import Problem
    pprob = Problem(prob.n, pinned[0], pinned[1], pinned[2], pinned[3], pinned[4], pinned[5],
                    pinned[6], pinned[7], pinned[8], prob.trace, prob.name)
    barrier(pg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_iters = []
    for _ in range(args.e2e_steps):
        c2 = U.usbs_create(pprob, psi=pinned[9], **params)
        res = U.usbs_solve(c2, warm_start=False, tol=TOL)
        U.usbs_get_dual(c2)
        U.usbs_get_sketch(c2)
        c2.close()
        e2e_iters.append(res["iters"])
    torch.cuda.synchronize()
    e2e_elapsed = max_over_ranks(pg, time.perf_counter() - t0)

    iters = [r["iters"] for r in results]
    conv = all(r["converged"] for r in results)
    # the paper's gate divides by 1 + |<C,X>| in scaled units; the gap relative to the
    # objective itself is reported beside it.  f(y) bounds the optimum only through the
    # exact lambda_max: the solve certifies f(y) by a longer eigen solve before it accepts
    # the gates (certify_restarts), and f is recomputed once more at the final y by a
    # still longer one (check_restarts).  A Ritz value never exceeds lambda_max, so both
    # are floors under the true f(y); the larger is reported.
    last = results[-1]["last"]
    cert = {"restarts": args.certify_restarts, "certifications": results[-1]["certifications"],
            "residual": results[-1]["cert_residual"]}
    # rank-r reconstruction of the final primal from its sketch and the best rounded cut
    # (App. C, App. E), timed on its own outside the solve's timed region
    torch.cuda.synchronize()
    tn = time.perf_counter()
    try:
        lam_ny, _, cut_vals, cut_best, _ = U.usbs_nystrom_round(ctx, want_u=False, want_signs=False)
        nystrom = {"ms": 1e3 * (time.perf_counter() - tn), "r": R_SKETCH, "lam_top": float(lam_ny[0]),
                   "rounded_cut": float(cut_vals[cut_best]),
                   "rounded_over_objective": float(cut_vals[cut_best]) / last["objective"]}
    except U.USBSError as exc:
        nystrom = {"error": str(exc)}
    y_fin = U.usbs_get_dual(ctx)
    c_scale, tau = U.usbs_scaling(ctx)
    with U.usbs_create(prob, lanczos_basis=64, lanczos_restarts=args.check_restarts, lanczos_tol=1e-8,
                       stream=stream) as chk:
        ev, _, einfo = U.usbs_extreme_eigs(chk, y=y_fin, kc=8, want_vecs=False)
    alpha_tau = 2.0 * tau                       # alpha = 2 tr X* after scaling (App. E)
    f_check = alpha_tau * max(ev[0] * c_scale, 0.0) + float(np.dot(prob.b, y_fin))
    f_best = max(f_check, last["dual_bound"])
    obj_gap = (f_best - last["objective"]) / abs(last["objective"])
    # time to an objective-relative gap: a certified solve that must also reach
    # |f(y) - <C,X>| / |<C,X>| <= obj_gap (beside both gates <= 1e-3), on the same stream
    obj_rel = None
    if args.obj_gap > 0:
        with U.usbs_create(prob, psi=psi, **dict(params, obj_gap_tol=args.obj_gap,
                                                  max_iters=args.obj_max_iters)) as c3:
            torch.cuda.synchronize()
            o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            o0.record(stream)
            r3 = U.usbs_solve(c3, tol=TOL)
            o1.record(stream)
            torch.cuda.synchronize()
            secs = o0.elapsed_time(o1) / 1e3
        obj_rel = {"obj_gap_tol": args.obj_gap, "converged": bool(r3["converged"]), "iters": r3["iters"],
                   "seconds": secs, "solves_per_s": (1.0 / secs) if r3["converged"] else 0.0,
                   "obj_gap": r3["obj_gap"], "certifications": r3["certifications"],
                   "objective": r3["last"]["objective"], "dual_bound": r3["last"]["dual_bound"],
                   "relinf": r3["last"]["relinf"], "max_iters": args.obj_max_iters}
    # C5 serving (bounded): served (continuous batching, warm starts) against plain FP64
    serve = None
    if args.serve_requests > 0:
        from paper_2312_11801_gb300 import instances as I
        serve = serve_measure(U, I, args.serve_requests, args.n_lo, args.n_hi, args.rho, 32,
                              args.serve_max_iters, args.slots, args.load, seed=rank, k_c=args.k_c, k_p=args.k_p)
    hbm, peak_src = peaks()
    # roofline of the dominant bulk kernel (largest device time among the kinds with
    # algorithmic bytes; the k-sized one-CTA kernels are latency-bound, not HBM-bound)
    bulk = {k: v for k, v in stats.items() if v[2] > 0}
    dom = max(bulk, key=lambda k: bulk[k][0])
    ms, nl, by = bulk[dom]
    achieved = (by / nl) / ((ms / 1e3) / nl) / 1e9 if ms > 0 else 0.0
    spmm_ms, spmm_n, spmm_b = stats["spmm"]
    spmm_gbs = spmm_b / (spmm_ms / 1e3) / 1e9 if spmm_ms > 0 else 0.0
    total_ms = sum(v[0] for v in stats.values())
    line = {
        "metric": METRIC, "value": world * args.steps / elapsed_max, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": prob.n, "edges": 2 * SIDE * SIDE, "weights": "+-1",
                   "r": R_SKETCH, "k_c": 8, "rho": 0.01, "beta": 0.25, "tol": TOL,
                   "precision": "mixed: FP32 bulk, FP64 k-sized", "parallelism": f"replicas{world}",
                   "lanczos_basis": args.lanczos_basis, "lanczos_tol": args.lanczos_tol or "default",
                   "l2": "inputs and basis larger than L2 (no flush)",
                   "iters_per_solve": iters, "converged": conv,
                   "gates": {"relgap": last["relgap"], "relinf": last["relinf"],
                             "objective": last["objective"], "dual_bound_solver": last["dual_bound"],
                             "dual_bound_check": f_check, "check_residual": einfo["max_residual"],
                             "check_restarts": args.check_restarts, "certification": cert,
                             "objective_relative_gap": obj_gap},
                   "timing": "profiling off in the timed region; kernel figures from "
                             f"{max(args.profile_steps, 1)} further solves with per-launch CUDA events"},
        "objective_relative": obj_rel,
        "serve": serve,
        "e2e": {"value": world * args.e2e_steps / e2e_elapsed, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": KERNEL_OF_KIND.get(dom, dom), "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": (TUPDATE_TRAFFIC["dram_bytes"] / TUPDATE_TRAFFIC["algorithmic_bytes"] * by / nl)
                     if dom == "reorth_update" and nl else None,
                     "algorithmic_bytes_per_launch": by / nl if nl else None,
                     "peak_source": peak_src},
        "nystrom": nystrom,
        "lanczos_spmm": {"achieved_gbs": spmm_gbs, "frac": spmm_gbs / hbm, "launches": spmm_n,
                         "avg_us": 1e3 * spmm_ms / max(spmm_n, 1),
                         "bytes_per_launch": spmm_b / max(spmm_n, 1)},
        "kernel_share": {k: round(v[0] / total_ms, 4) for k, v in stats.items() if total_ms > 0},
        "clocks": clk,
    }
    if rank == 0:
        if not args.no_cpu:
            line["cpu_baseline"] = oracle_sample(int(statistics.median(iters)))
        print(json.dumps(line), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------------------
# Batched and served workloads (their own JSON lines, selected with --workload)
# ---------------------------------------------------------------------------------------
def _pct(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def plain_fp64_sample(U, probs, rho, tol, max_iters, budget_s, basis=32, k_c=8, k_p=0):
    """The plain path: one instance at a time, FP64 throughout, per-step kernels, cold
    start; solves in order until the time budget is spent.  Returns per-solve records."""
    out = []
    t_all = time.perf_counter()
    for p in probs:
        if out and time.perf_counter() - t_all > budget_s:
            break
        t0 = time.perf_counter()
        with U.usbs_create(p, precision=U.PRECISION_FP64, rho=rho, max_iters=max_iters,
                           lanczos_basis=basis, k_c=k_c, k_p=k_p) as c:
            r = U.usbs_solve(c, tol=tol)
        out.append({"secs": time.perf_counter() - t0, "iters": r["iters"], "converged": r["converged"],
                    "n": p.n})
    return out


def run_batched(args, world, rank, local, pg):
    """C4: independent MaxCut SDPs on Erdos-Renyi graphs, n ~ U{100..4000}, average
    degree 8, weights U[0, 1], solved by one persistent launch per (precision, basis)
    bucket.  A step is one cold-start solve of every instance."""
    import torch
    from paper_2312_11801_gb300 import build as B
    B.build()
    from paper_2312_11801_gb300 import usbs as U
    from paper_2312_11801_gb300 import instances as I
    torch.cuda.set_device(local)
    probs = I.batched_er(args.batch_count, seed0=1000 * rank)
    kw = dict(precision=U.PRECISION_MIXED, lanczos_basis=args.lanczos_basis, rho=args.rho,
              max_iters=args.max_iters, k_c=args.k_c, k_p=args.k_p)
    ctxs = [U.usbs_create(p, **kw) for p in probs]
    for _ in range(args.warmup):
        U.usbs_batch_solve(ctxs, tol=TOL)
    barrier(pg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    conv, iters = 0, []
    for _ in range(args.steps):
        res, st = U.usbs_batch_solve(ctxs, tol=TOL)
        conv += sum(r["converged"] for r in res)
        iters += [r["iters"] for r in res]
    torch.cuda.synchronize()
    elapsed = max_over_ranks(pg, time.perf_counter() - t0)
    for c in ctxs:
        c.close()
    # end to end: create from host arrays, solve, read every dual back
    barrier(pg)
    t0 = time.perf_counter()
    ctxs = [U.usbs_create(p, **kw) for p in probs]
    res, st = U.usbs_batch_solve(ctxs, tol=TOL)
    h2d = sum(p.C_rowptr.nbytes + p.C_col.nbytes + p.C_val.nbytes + p.A_con.nbytes + p.A_i.nbytes +
              p.A_j.nbytes + p.A_val.nbytes + p.b.nbytes + p.is_ineq.nbytes for p in probs)
    d2h = 0
    for c in ctxs:
        d2h += U.usbs_get_dual(c).nbytes
        c.close()
    e2e_conv = sum(r["converged"] for r in res)
    e2e_elapsed = max_over_ranks(pg, time.perf_counter() - t0)
    plain = plain_fp64_sample(U, probs, args.rho, TOL, args.max_iters, args.plain_budget,
                              args.lanczos_basis, args.k_c, args.k_p) \
        if rank == 0 and not args.no_plain else []
    pconv = sum(r["converged"] for r in plain)
    line = {
        "metric": METRIC, "value": world * conv / elapsed, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"batched_er_{args.batch_count}_n100-4000_d8_u01_mixed_J{args.lanczos_basis}",
                   "instances": len(probs), "rho": args.rho, "tol": TOL, "k_c": args.k_c, "k_p": args.k_p,
                   "precision": "mixed: FP32 bulk, FP64 k-sized", "launch": "persistent, one CTA per instance",
                   "parallelism": f"replicas{world}", "converged_per_step": conv / args.steps,
                   "iters_median": float(np.median(iters)), "iters_max": int(max(iters))},
        "e2e": {"value": world * e2e_conv / e2e_elapsed, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "plain_fp64": {"solves": len(plain), "converged": pconv,
                       "value": (pconv / sum(r["secs"] for r in plain)) if plain else None,
                       "unit": UNIT, "note": "one instance at a time, FP64, per-step kernels, a prefix of "
                                             "the same instances within the time budget"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_requests(I, count, n_lo, n_hi, seed=0):
    """C5 request stream: n log-uniform on [n_lo, n_hi], random geometric graphs of mean
    degree 10; every second request (after the first) is a prior request's instance grown
    by 1 % new points, naming that request as its parent."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for i in range(count):
        if i > 0 and rng.random() < 0.5:
            j = int(rng.integers(0, i))
            prob = I.grow_rgg(reqs[j]["prob"], 0.01, seed=10_000 + i)
            reqs.append({"id": i, "parent": j, "prob": prob})
        else:
            n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
            reqs.append({"id": i, "parent": -1, "prob": I.maxcut_rgg(n, 10.0, seed=20_000 + i)})
    return reqs


def serve_measure(U, I, requests, n_lo, n_hi, rho, basis, max_iters, slots, load, seed=0, k_c=8, k_p=0):
    """C5 serving: a Poisson stream of MaxCut requests (random geometric graphs, n
    log-uniform on [n_lo, n_hi], every second request a 1 %-grown copy of an earlier one)
    served by continuous batching (mixed precision, grown requests warm-started from their
    resident parents) against the plain path (FP64, one request at a time, cold).  Both arms
    see the same arrival times, at `load` times the plain path's measured capacity; the plain
    arm's latencies follow from its measured service times by a FIFO single-server queue.
    Solves/sec count converged requests over the makespan; p50/p99 are given over the
    converged requests and over all of them."""
    reqs = serve_requests(I, requests, n_lo, n_hi, seed=seed)
    plain_s = []
    for q in reqs:
        t0 = time.perf_counter()
        with U.usbs_create(q["prob"], precision=U.PRECISION_FP64, rho=rho, max_iters=max_iters,
                           lanczos_basis=basis, k_c=k_c, k_p=k_p) as c:
            r = U.usbs_solve(c, tol=TOL)
        plain_s.append((time.perf_counter() - t0, bool(r["converged"])))
    plain_cap = len(reqs) / sum(t for t, _ in plain_s)
    rate = load * plain_cap
    rng = np.random.Generator(np.random.PCG64(99 + seed))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    free_at, plain_lat = 0.0, []
    for a_t, (sv, _) in zip(arrivals, plain_s):
        start = max(a_t, free_at)
        free_at = start + sv
        plain_lat.append(free_at - a_t)
    plain_makespan = free_at - arrivals[0]
    srv = U.usbs_server_create(max_slots=slots, cache_entries=requests,
                               solver={"rho": rho, "lanczos_basis": basis, "max_iters": max_iters,
                                       "k_c": k_c, "k_p": k_p})
    done = []
    t0 = time.perf_counter()
    for q, a_t in zip(reqs, arrivals):
        while time.perf_counter() - t0 < a_t:
            done += U.usbs_server_poll(srv, 64, wait_ms=1)
        U.usbs_server_submit(srv, q["id"], q["prob"], parent_id=q["parent"], tol=TOL)
    while len(done) < len(reqs):
        done += U.usbs_server_poll(srv, 64, wait_ms=20)
    st = U.usbs_server_get_stats(srv)
    srv.close()
    lat = [c["t_finish"] - c["t_arrival"] for c in done]
    lat_conv = [c["t_finish"] - c["t_arrival"] for c in done if c["status"] == U.USBS_OK]
    conv = len(lat_conv)
    served_makespan = max(c["t_finish"] for c in done) - min(c["t_arrival"] for c in done)
    plain_conv_lat = [l for l, (_, ok) in zip(plain_lat, plain_s) if ok]
    return {
        "workload": f"serve_rgg_poisson_{requests}req_n{n_lo}-{n_hi}_grown50",
        "requests": len(reqs), "grown_from_parent": sum(q["parent"] >= 0 for q in reqs),
        "n_range": [min(q["prob"].n for q in reqs), max(q["prob"].n for q in reqs)],
        "rho": rho, "tol": TOL, "lanczos_basis": basis, "max_iters": max_iters, "slots": slots,
        "k_c": k_c, "k_p": k_p,
        "load_vs_plain_capacity": load, "arrival_rate_per_s": rate,
        "served": {"solves_per_s": conv / served_makespan, "converged": conv,
                   "p50_s_converged": _pct(lat_conv, 50), "p99_s_converged": _pct(lat_conv, 99),
                   "p50_s_all": _pct(lat, 50), "p99_s_all": _pct(lat, 99),
                   "warm": sum(c["warm"] for c in done), "peak_running": st["peak_running"],
                   "peak_bytes": st["peak_bytes"], "makespan_s": served_makespan},
        "plain_fp64": {"solves_per_s": len(plain_conv_lat) / plain_makespan, "converged": len(plain_conv_lat),
                       "p50_s_converged": _pct(plain_conv_lat, 50), "p99_s_converged": _pct(plain_conv_lat, 99),
                       "p50_s_all": _pct(plain_lat, 50), "p99_s_all": _pct(plain_lat, 99),
                       "capacity_solves_per_s": plain_cap, "makespan_s": plain_makespan},
    }


def run_serve(args, world, rank, local, pg):
    """C5 as its own line (see serve_measure)."""
    import torch
    from paper_2312_11801_gb300 import build as B
    B.build()
    from paper_2312_11801_gb300 import usbs as U
    from paper_2312_11801_gb300 import instances as I
    torch.cuda.set_device(local)
    sv = serve_measure(U, I, args.requests, args.n_lo, args.n_hi, args.rho, args.lanczos_basis,
                       args.max_iters, args.slots, args.load, seed=rank, k_c=args.k_c, k_p=args.k_p)
    line = {
        "metric": METRIC, "value": sv["served"]["solves_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": 1, "warmup": 0, "ms_per_step": 1e3 * sv["served"]["makespan_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {k: v for k, v in sv.items() if k not in ("served", "plain_fp64")},
        "served": sv["served"], "plain_fp64": sv["plain_fp64"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_c1(args, world, rank, local, pg):
    """C1: plain FP64 USBS on MaxCut, Erdos-Renyi n = 800, average degree 6, unit
    weights, seed 0, k = 8, no sketch, one instance at a time (per-step kernels)."""
    import torch
    from paper_2312_11801_gb300 import build as B
    B.build()
    from paper_2312_11801_gb300 import usbs as U
    from paper_2312_11801_gb300 import instances as I
    torch.cuda.set_device(local)
    prob = I.maxcut_er(800, 6.0, 0)
    stream = torch.cuda.Stream()
    kw = dict(precision=U.PRECISION_FP64, rho=args.c1_rho, max_iters=args.max_iters, stream=stream)
    ctx = U.usbs_create(prob, **kw)
    for _ in range(args.warmup):
        U.usbs_solve(ctx, tol=TOL)
    U.usbs_profile(ctx, True)
    n0 = U.usbs_launch_count(ctx)
    barrier(pg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = [U.usbs_solve(ctx, tol=TOL) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    elapsed = max_over_ranks(pg, e0.elapsed_time(e1) / 1e3)
    launches = U.usbs_launch_count(ctx) - n0
    stats = U.usbs_kernel_stats(ctx)
    U.usbs_profile(ctx, False)
    ctx.close()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        with U.usbs_create(prob, **kw) as c2:
            U.usbs_solve(c2, tol=TOL)
            U.usbs_get_dual(c2)
    e2e = max_over_ranks(pg, time.perf_counter() - t0)
    total_ms = sum(v[0] for v in stats.values()) or 1.0
    last = res[-1]["last"]
    line = {
        "metric": METRIC, "value": world * args.steps / elapsed, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "maxcut_er800_d6_s0_fp64_plain", "rho": args.c1_rho, "tol": TOL, "k_c": 8,
                   "iters_per_solve": [r["iters"] for r in res],
                   "converged": all(r["converged"] for r in res),
                   "objective": last["objective"], "dual_bound": last["dual_bound"]},
        "e2e": {"value": world * args.e2e_steps / e2e if args.e2e_steps else None, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(a.nbytes for a in U._problem_arrays(prob))),
                "d2h_bytes_per_step": 8 * prob.m},
        "gpu_launches": int(launches),
        "kernel_share": {k: round(v[0] / total_ms, 4) for k, v in stats.items()},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_c3(args, world, rank, local, pg):
    """C3: clustering SDP, n = 65,536 points, 655,360 signed similarity edges (weights
    N(0, 1)), X_ii = 1 and X_ij >= 0 on every edge (~2.1e9 implicit variables), sketch
    rank 32, mixed precision.  A step is a cold-start solve, capped at --max-iters."""
    import torch
    from paper_2312_11801_gb300 import build as B
    B.build()
    from paper_2312_11801_gb300 import usbs as U
    from paper_2312_11801_gb300 import instances as I
    torch.cuda.set_device(local)
    prob = I.clustering_sdp(args.c3_n, args.c3_n * 10, seed=0)
    psi = I.gaussian_psi(prob.n, 32, seed=1)
    stream = torch.cuda.Stream()
    kw = dict(precision=U.PRECISION_MIXED, r=32, rho=args.c3_rho, max_iters=args.max_iters,
              lanczos_basis=args.lanczos_basis, stream=stream)
    ctx = U.usbs_create(prob, psi=psi, **kw)
    for _ in range(args.warmup):
        U.usbs_solve(ctx, tol=TOL)
    U.usbs_profile(ctx, True)
    n0 = U.usbs_launch_count(ctx)
    barrier(pg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = [U.usbs_solve(ctx, tol=TOL) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    elapsed = max_over_ranks(pg, e0.elapsed_time(e1) / 1e3)
    launches = U.usbs_launch_count(ctx) - n0
    stats = U.usbs_kernel_stats(ctx)
    U.usbs_profile(ctx, False)
    ctx.close()
    total_ms = sum(v[0] for v in stats.values()) or 1.0
    last = res[-1]["last"]
    iters = sum(r["iters"] for r in res)
    line = {
        "metric": METRIC, "value": world * sum(r["converged"] for r in res) / elapsed, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"clustering_n{prob.n}_e{args.c3_n * 10}_r32_mixed", "m": prob.m,
                   "rho": args.c3_rho, "tol": TOL, "lanczos_basis": args.lanczos_basis,
                   "iters_per_solve": [r["iters"] for r in res],
                   "converged": [r["converged"] for r in res],
                   "ms_per_iteration": 1e3 * elapsed / max(iters, 1),
                   "gates": {"relgap": last["relgap"], "relinf": last["relinf"],
                             "objective": last["objective"], "dual_bound": last["dual_bound"]}},
        "gpu_launches": int(launches),
        "kernel_share": {k: round(v[0] / total_ms, 4) for k, v in stats.items()},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sweep(args, world, rank, local, pg):
    """k_c / k_p grid (the paper's App. F parameter sweeps, on synthetic graphs): cold-start
    solves to both gates <= 1e-3 in mixed precision, one per (graph, k_c, k_p) at --rho, for
    one setting the model value by the App. B.1 IPM against its closed form, and (k_c, k_p) =
    (8, 0) and (7, 1) at each rho of --sweep-rhos.  Reports iterations, seconds and the
    objective of each."""
    import torch
    from paper_2312_11801_gb300 import build as B
    B.build()
    from paper_2312_11801_gb300 import usbs as U
    from paper_2312_11801_gb300 import instances as I
    torch.cuda.set_device(local)
    graphs = {"er2000_d6": I.maxcut_er(2000, 6.0, 7), "rgg1000_d10": I.maxcut_rgg(1000, 10.0, seed=7)}
    grid = [(8, 0), (7, 1), (6, 2), (5, 3), (4, 0), (4, 2), (2, 1)]
    rhos = [float(x) for x in args.sweep_rhos.split(",") if x.strip()]
    runs = [(kc, kp, args.rho, mv) for (kc, kp) in grid for mv in ((0, 1) if (kc, kp) == (6, 2) else (0,))]
    runs += [(kc, kp, rho, 0) for rho in rhos if rho != args.rho for (kc, kp) in ((8, 0), (7, 1))]
    rows = []
    t_all = time.perf_counter()
    for gname, prob in graphs.items():
        for (kc, kp, rho, mv) in runs:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with U.usbs_create(prob, precision=U.PRECISION_MIXED, k_c=kc, k_p=kp, rho=rho,
                               max_iters=min(args.max_iters, 1500), model_value_ipm=mv) as c:
                r = U.usbs_solve(c, tol=TOL)
            torch.cuda.synchronize()
            rows.append({"graph": gname, "k_c": kc, "k_p": kp, "rho": rho, "model_value": "ipm" if mv else "closed",
                         "iters": r["iters"], "converged": bool(r["converged"]),
                         "seconds": time.perf_counter() - t0, "objective": r["last"]["objective"],
                         "relgap": r["last"]["relgap"], "relinf": r["last"]["relinf"]})
    elapsed = max_over_ranks(pg, time.perf_counter() - t_all)
    conv = sum(r["converged"] for r in rows)
    line = {
        "metric": METRIC, "value": conv / elapsed, "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": 1e3 * elapsed, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "kc_kp_sweep_er2000_rgg1000_mixed", "max_iters": min(args.max_iters, 1500), "rho": args.rho, "tol": TOL,
                   "grid": grid, "solves": rows},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args, world, rank):
    """The oracle arm: each step is the bounded oracle sample of run_ours's workload."""
    if rank != 0:
        return
    gpu_iters = args.ref_iters
    vals = []
    for _ in range(args.warmup):
        oracle_sample(gpu_iters, budget_s=20.0)
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = oracle_sample(gpu_iters, budget_s=20.0)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": WORKLOAD, "n": SIDE * SIDE, "r": R_SKETCH, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                         "sample": last["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=SIDE)
    ap.add_argument("--max-iters", type=int, default=2000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--lanczos-basis", type=int, default=32, choices=[16, 32, 64],
                    help="Lanczos basis of the C2 solve (the paper's 32 inner iterations)")
    ap.add_argument("--lanczos-tol", type=float, default=0.0, help="0 = the library default")
    ap.add_argument("--certify-restarts", type=int, default=50,
                    help="cycles of the eigen solve that certifies f(y) before the gates are accepted")
    ap.add_argument("--check-restarts", type=int, default=200,
                    help="cycles of the check eigen solve at the final y (outside the timed region)")
    ap.add_argument("--profile-steps", type=int, default=2,
                    help="solves timed launch by launch after the timed region (kernel shares, roofline)")
    ap.add_argument("--obj-gap", type=float, default=1e-2,
                    help="objective-relative gap of the extra time-to-solution figure; 0 = skip it")
    ap.add_argument("--obj-max-iters", type=int, default=1500)
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c3", "batched", "serve", "sweep"])
    ap.add_argument("--c3-n", type=int, default=65536)
    ap.add_argument("--c3-rho", type=float, default=0.01)
    ap.add_argument("--c1-rho", type=float, default=0.1)
    ap.add_argument("--rho", type=float, default=0.03, help="rho of the batched, served and sweep workloads")
    ap.add_argument("--sweep-rhos", default="0.1,0.01", help="further rho values of the sweep, for (8, 0) and (7, 1)")
    ap.add_argument("--k-c", type=int, default=8, help="k_c of the batched and served workloads")
    ap.add_argument("--k-p", type=int, default=0, help="k_p of the batched and served workloads")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--plain-budget", type=float, default=60.0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--serve-requests", type=int, default=16,
                    help="requests of the C5 serving figure added to the default line; 0 = skip it")
    ap.add_argument("--serve-max-iters", type=int, default=400)
    ap.add_argument("--n-lo", type=int, default=1000)
    ap.add_argument("--n-hi", type=int, default=200000)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--load", type=float, default=0.7)
    ap.add_argument("--ref-iters", type=int, default=35,
                    help="iterations per solve used to scale the reference arm's sample "
                         "(the GPU solve of this workload takes 34-37)")
    args = ap.parse_args()
    world, rank, local, pg = dist_setup() if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0, None)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "c3":
        run_c3(args, world, rank, local, pg)
    elif args.workload == "c1":
        run_c1(args, world, rank, local, pg)
    elif args.workload == "batched":
        run_batched(args, world, rank, local, pg)
    elif args.workload == "serve":
        run_serve(args, world, rank, local, pg)
    elif args.workload == "sweep":
        run_sweep(args, world, rank, local, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
