"""Seeded synthetic SDP instances in the form (C, A, b, I) of the primal (P), Sec. 2.1.

This module only builds problem data: graphs, the MaxCut cost ``C = L/4`` (Sec. 5.1,
eq. maxcut_sdp), the clustering cost ``C = W`` with ``X_ii = 1`` and ``X_ij >= 0``
(App. E.3 constraint structure), and the Gaussian sketch test matrix ``Psi`` (Sec. 4).
It holds none of the solver's arithmetic, so both the CPU oracle and the CUDA path
read the very same arrays from here.

Encoding (shared by every consumer):

* ``C`` is a full symmetric CSR matrix (both triangles, diagonal entries included
  where nonzero): ``C_rowptr`` int64 (n+1), ``C_col`` int32, ``C_val`` float64.
* ``A`` is a COO list of entries ``(con, i, j, val)``; an entry adds ``val * X_ij``
  to ``<A_con, X>``.  For ``i != j`` it stands for the symmetric matrix
  ``(val/2)(e_i e_j^T + e_j e_i^T)``.
* ``b`` float64 (m) and ``is_ineq`` uint8 (m): row ``c`` reads ``<A_c, X> <= b_c``
  when ``is_ineq[c]`` else ``<A_c, X> = b_c``.
* ``trace`` is ``tr(X*)``, which the constraints fix for every family built here
  (``diag(X) = 1`` gives ``tr X* = n``); the solvers use it for problem scaling.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem", "laplacian_maxcut", "maxcut_er", "maxcut_torus", "maxcut_rgg",
    "grow_rgg", "clustering_sdp", "maxcut_from_edges", "complete_graph_edges",
    "cycle_edges", "batched_er", "qap_sdp", "dual_sample", "gaussian_psi", "save_npz", "load_npz",
]


@dataclasses.dataclass
class Problem:
    n: int
    C_rowptr: np.ndarray
    C_col: np.ndarray
    C_val: np.ndarray
    A_con: np.ndarray
    A_i: np.ndarray
    A_j: np.ndarray
    A_val: np.ndarray
    b: np.ndarray
    is_ineq: np.ndarray
    trace: float
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.b.shape[0])

    @property
    def nnz_c(self) -> int:
        return int(self.C_col.shape[0])

    @property
    def nnz_a(self) -> int:
        return int(self.A_con.shape[0])


def _csr_from_sym_entries(n, rows, cols, vals):
    """Full symmetric CSR from upper-triangle (i<j) entries plus diagonal entries.

    ``rows/cols/vals`` list each off-diagonal pair once (either order) and each
    diagonal entry once; duplicates are summed.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    off = rows != cols
    r = np.concatenate([rows, cols[off]])
    c = np.concatenate([cols, rows[off]])
    v = np.concatenate([vals, vals[off]])
    key = r * n + c
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    uniq, start = np.unique(key, return_index=True)
    v = np.add.reduceat(v, start) if len(v) else v
    r = uniq // n
    c = uniq % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, c.astype(np.int32), v.astype(np.float64)


def laplacian_maxcut(n, ei, ej, w):
    """CSR of ``C = L/4`` with ``L = Diag(W 1) - W`` for an undirected weighted graph.

    Each edge is listed once.  ``<C, X> = (1/4) tr(L X)`` is the MaxCut SDP objective
    of Sec. 5.1 (eq. maxcut_sdp).
    """
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    deg = np.zeros(n, dtype=np.float64)
    np.add.at(deg, ei, w)
    np.add.at(deg, ej, w)
    rows = np.concatenate([ei, np.arange(n)])
    cols = np.concatenate([ej, np.arange(n)])
    vals = np.concatenate([-w / 4.0, deg / 4.0])
    keep = vals != 0.0
    return _csr_from_sym_entries(n, rows[keep], cols[keep], vals[keep])


def _diag_constraints(n):
    """``diag(X) = 1``: one equality row per vertex, entry (c=i, i, i, 1)."""
    idx = np.arange(n, dtype=np.int32)
    return (idx.copy(), idx.copy(), idx.copy(), np.ones(n, dtype=np.float64),
            np.ones(n, dtype=np.float64), np.zeros(n, dtype=np.uint8))


def maxcut_from_edges(n, ei, ej, w, name="maxcut", meta=None) -> Problem:
    rowptr, col, val = laplacian_maxcut(n, ei, ej, w)
    con, ai, aj, av, b, ineq = _diag_constraints(n)
    md = {"n_edges": int(len(ei)), "weight_sum": float(np.sum(w))}
    if meta:
        md.update(meta)
    return Problem(n, rowptr, col, val, con, ai, aj, av, b, ineq, float(n), name, md)


def complete_graph_edges(n):
    i, j = np.triu_indices(n, 1)
    return i, j, np.ones(len(i))


def cycle_edges(n):
    i = np.arange(n)
    return i, (i + 1) % n, np.ones(n)


def _er_edges(n, avg_deg, rng):
    p = avg_deg / (n - 1)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    return iu[keep], ju[keep]


def maxcut_er(n=800, avg_deg=6.0, seed=0, weights="unit") -> Problem:
    """MaxCut on G(n, p = avg_deg/(n-1)); unit weights or weights ~ U[0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ei, ej = _er_edges(n, avg_deg, rng)
    if weights == "unit":
        w = np.ones(len(ei))
    elif weights == "uniform":
        w = rng.random(len(ei))
    else:
        raise ValueError(weights)
    return maxcut_from_edges(n, ei, ej, w, name=f"maxcut_er_n{n}_d{avg_deg:g}_s{seed}",
                             meta={"avg_deg": avg_deg, "seed": seed, "weights": weights})


def maxcut_torus(side=1000, seed=0, signed=True) -> Problem:
    """MaxCut on the side x side toroidal grid; node (i, j) -> side*i + j.

    Edges join (i, j) to (i+1 mod side, j) and to (i, j+1 mod side), 2*side^2 in total.
    Weights are +-1 with probability 1/2 each (``signed``) or all +1.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    node = np.arange(side * side, dtype=np.int64).reshape(side, side)
    down = np.roll(node, -1, axis=0)
    right = np.roll(node, -1, axis=1)
    ei = np.concatenate([node.ravel(), node.ravel()])
    ej = np.concatenate([down.ravel(), right.ravel()])
    if signed:
        w = np.where(rng.random(len(ei)) < 0.5, -1.0, 1.0)
    else:
        w = np.ones(len(ei))
    return maxcut_from_edges(side * side, ei, ej, w,
                             name=f"maxcut_torus_{side}x{side}_{'pm1' if signed else 'unit'}_s{seed}",
                             meta={"side": side, "seed": seed, "signed": signed})


def _rgg_edges(points, radius):
    from scipy.spatial import cKDTree
    pairs = cKDTree(points).query_pairs(radius, output_type="ndarray")
    if len(pairs) == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)


def maxcut_rgg(n, avg_deg=10.0, seed=0, points=None, radius=None) -> Problem:
    """MaxCut on a random geometric graph in the unit square, unit weights.

    The radius ``sqrt(avg_deg / (pi n))`` gives expected degree ``avg_deg`` away from
    the boundary; the realised mean degree is recorded in ``meta``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if points is None:
        points = rng.random((n, 2))
    if radius is None:
        radius = math.sqrt(avg_deg / (math.pi * n))
    ei, ej = _rgg_edges(points, radius)
    prob = maxcut_from_edges(len(points), ei, ej, np.ones(len(ei)),
                             name=f"maxcut_rgg_n{len(points)}_s{seed}",
                             meta={"radius": radius, "seed": seed,
                                   "realised_deg": 2.0 * len(ei) / max(len(points), 1)})
    prob.meta["points"] = points
    return prob


def grow_rgg(parent: Problem, frac=0.01, seed=1) -> Problem:
    """Append ``ceil(frac n)`` uniform points to an RGG instance, same radius.

    Old vertices keep their indices and edges, so the parent is the leading
    principal subproblem of the grown instance (the warm-start setting of Sec. 5.1).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = parent.meta["points"]
    add = max(1, int(math.ceil(frac * len(pts))))
    new_pts = np.concatenate([pts, rng.random((add, 2))])
    child = maxcut_rgg(len(new_pts), points=new_pts, radius=parent.meta["radius"])
    child.name = parent.name + f"_grow{add}"
    child.meta["parent_n"] = len(pts)
    return child


def clustering_sdp(n=65536, n_edges=655360, seed=0) -> Problem:
    """Signed-similarity clustering SDP: maximise <W, X>, X_ii = 1, X_ij >= 0 on edges.

    W is symmetric with ``n_edges`` distinct uniformly random off-diagonal pairs,
    weights ~ N(0, 1).  Rows 0..n-1 are the equalities ``X_ii = 1``; row n+e is the
    inequality ``-X_ij <= 0`` of edge e (entry value -1, b = 0).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    need = n_edges
    got_i = np.zeros(0, np.int64)
    got_j = np.zeros(0, np.int64)
    while need > 0:
        draw = int(need * 1.2) + 16
        a = rng.integers(0, n, size=draw)
        c = rng.integers(0, n, size=draw)
        ok = a != c
        lo = np.minimum(a, c)[ok]
        hi = np.maximum(a, c)[ok]
        key = np.concatenate([got_i * n + got_j, lo * n + hi])
        _, first = np.unique(key, return_index=True)
        first.sort()
        key = key[first][:n_edges]
        got_i, got_j = key // n, key % n
        need = n_edges - len(got_i)
    w = rng.standard_normal(n_edges)
    rowptr, col, val = _csr_from_sym_entries(n, got_i, got_j, w)
    con_d = np.arange(n, dtype=np.int32)
    con_e = (n + np.arange(n_edges)).astype(np.int32)
    A_con = np.concatenate([con_d, con_e])
    A_i = np.concatenate([np.arange(n), got_i]).astype(np.int32)
    A_j = np.concatenate([np.arange(n), got_j]).astype(np.int32)
    A_val = np.concatenate([np.ones(n), -np.ones(n_edges)])
    b = np.concatenate([np.ones(n), np.zeros(n_edges)])
    ineq = np.concatenate([np.zeros(n, np.uint8), np.ones(n_edges, np.uint8)])
    return Problem(n, rowptr, col, val, A_con, A_i, A_j, A_val, b, ineq, float(n),
                   name=f"clustering_n{n}_e{n_edges}_s{seed}",
                   meta={"n_edges": n_edges, "seed": seed})


def qap_sdp(nq=6, seed=0) -> Problem:
    """Synthetic QAP relaxation in the form of App. E (QAP, eq. qap_sdp), for minimising
    tr(W Pi D Pi^T) over permutations Pi of nq items.

    W (flows) is a ring over the nq facilities plus nq/2 random chords, integer weights
    1..4; D (distances) is the Manhattan distance between nq random points of a
    nq x nq grid.  X = [[1, vec(B)^T], [vec(B), Y]] has n = nq^2 + 1 rows; index
    1 + i + nq j holds B_ij (vec stacks columns), so Y's Kronecker order matches D (x) W.
    The objective is maximised as <C, X> with C = -(D (x) W) on the Y block.  Rows:
      0                      X_00 = 1
      tr_1(Y) = I            sum_j Y[(i1, j), (i2, j)] = delta_i1i2, i1 <= i2
      tr_2(Y) = I            sum_i Y[(i, j1), (i, j2)] = delta_j1j2, j1 <= j2
      vec(B) = diag(Y)       X_{0, p} - X_{p, p} = 0 for every p
      B 1 = 1, 1^T B = 1^T   row and column sums of B
      tr(Y) = nq
      G(Y) >= 0              -Y_pq <= 0 on the support of D (x) W (inequalities)
      B >= 0                 -X_{0, p} <= 0 (inequalities)
    tr X* = 1 + nq (X_00 = 1 and tr Y = nq).
    """
    rng = np.random.Generator(np.random.PCG64(20_000 + seed))
    W = np.zeros((nq, nq))
    for a in range(nq):
        b_ = (a + 1) % nq
        W[a, b_] = W[b_, a] = rng.integers(1, 5)
    for _ in range(nq // 2):
        a, b_ = rng.choice(nq, size=2, replace=False)
        W[a, b_] = W[b_, a] = rng.integers(1, 5)
    pts = rng.choice(nq * nq, size=nq, replace=False)
    px, py = pts % nq, pts // nq
    D = (np.abs(px[:, None] - px[None, :]) + np.abs(py[:, None] - py[None, :])).astype(np.float64)
    n = nq * nq + 1
    K = np.kron(D, W)                     # K[j1 nq + i1, j2 nq + i2] = D[j1, j2] W[i1, i2]
    rr, cc = np.nonzero(np.triu(K, 1))
    rows = np.concatenate([rr + 1, cc + 1])
    cols = np.concatenate([cc + 1, rr + 1])
    vals = np.concatenate([-K[rr, cc], -K[rr, cc]])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    con, ai, aj, av, bb, iq = [], [], [], [], [], []

    def row(entries, rhs, ineq=0):
        c = len(bb)
        for (i, j, v) in entries:
            con.append(c)
            ai.append(min(i, j))
            aj.append(max(i, j))
            av.append(v)
        bb.append(rhs)
        iq.append(ineq)

    def y(i, j):                          # index of B_ij / of Y's row (i, j)
        return 1 + i + nq * j

    row([(0, 0, 1.0)], 1.0)
    for i1 in range(nq):
        for i2 in range(i1, nq):
            row([(y(i1, j), y(i2, j), 1.0) for j in range(nq)], 1.0 if i1 == i2 else 0.0)
    for j1 in range(nq):
        for j2 in range(j1, nq):
            row([(y(i, j1), y(i, j2), 1.0) for i in range(nq)], 1.0 if j1 == j2 else 0.0)
    for p in range(1, n):
        row([(0, p, 1.0), (p, p, -1.0)], 0.0)
    for i in range(nq):
        row([(0, y(i, j), 1.0) for j in range(nq)], 1.0)
    for j in range(nq):
        row([(0, y(i, j), 1.0) for i in range(nq)], 1.0)
    row([(p, p, 1.0) for p in range(1, n)], float(nq))
    for a, b_ in zip(rr, cc):
        row([(a + 1, b_ + 1, -1.0)], 0.0, 1)
    for p in range(1, n):
        row([(0, p, -1.0)], 0.0, 1)
    return Problem(n, rowptr, cols.astype(np.int32), vals, np.asarray(con, np.int32),
                   np.asarray(ai, np.int32), np.asarray(aj, np.int32), np.asarray(av, np.float64),
                   np.asarray(bb, np.float64), np.asarray(iq, np.uint8), float(1 + nq),
                   name=f"qap_n{nq}_s{seed}", meta={"nq": nq, "W": W, "D": D})


def batched_er(count=512, n_lo=100, n_hi=4000, avg_deg=8.0, seed0=0):
    """The batched workload: ``count`` MaxCut instances, n ~ U{n_lo..n_hi}, weights U[0,1]."""
    rng = np.random.Generator(np.random.PCG64(10_000 + seed0))
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    return [maxcut_er(int(nn), avg_deg, seed=seed0 + s, weights="uniform")
            for s, nn in enumerate(ns)]


def dual_sample(prob: Problem, seed=11, scale=0.05):
    """A seeded dual point for eigen-solve tests, in the scaled units of App. E: i.i.d.
    |N(0, 1)| * scale / sqrt(n) per constraint (non-negative, so every inequality row
    is admissible)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.abs(rng.standard_normal(prob.m)) * scale / math.sqrt(prob.n)


def gaussian_psi(n, r, seed=1, dtype=np.float32):
    """Sketch test matrix Psi (n x r, row-major) with i.i.d. N(0, 1) entries (Sec. 4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, r)).astype(dtype)


def extend_psi(psi, n_new, seed=2):
    """Rows for vertices added by growth; the old rows are kept unchanged."""
    rng = np.random.Generator(np.random.PCG64(seed))
    add = n_new - psi.shape[0]
    return np.concatenate([psi, rng.standard_normal((add, psi.shape[1])).astype(psi.dtype)])


def save_npz(path, prob: Problem):
    np.savez_compressed(
        path, n=prob.n, C_rowptr=prob.C_rowptr, C_col=prob.C_col, C_val=prob.C_val,
        A_con=prob.A_con, A_i=prob.A_i, A_j=prob.A_j, A_val=prob.A_val, b=prob.b,
        is_ineq=prob.is_ineq, trace=prob.trace, name=prob.name)


def load_npz(path) -> Problem:
    z = np.load(path)
    return Problem(int(z["n"]), z["C_rowptr"], z["C_col"], z["C_val"], z["A_con"],
                   z["A_i"], z["A_j"], z["A_val"], z["b"], z["is_ineq"],
                   float(z["trace"]), str(z["name"]))
