"""Small named graphs for the MaxCut pins (input construction only)."""
import numpy as np

from paper_2312_11801_gb300 import instances as I


def named_graph(name):
    if name.startswith("K") and "," in name:
        a, b = (int(x) for x in name[1:].split(","))
        i = [x for x in range(a) for _ in range(b)]
        j = [a + y for _ in range(a) for y in range(b)]
        return a + b, np.array(i), np.array(j), np.ones(len(i))
    if name.startswith("K"):
        n = int(name[1:])
        i, j, w = I.complete_graph_edges(n)
        return n, i, j, w
    if name.startswith("C"):
        n = int(name[1:])
        i, j, w = I.cycle_edges(n)
        return n, i, j, w
    if name == "petersen":
        e = ([(x, (x + 1) % 5) for x in range(5)] + [(5 + x, 5 + (x + 2) % 5) for x in range(5)]
             + [(x, 5 + x) for x in range(5)])
        return 10, np.array([a for a, _ in e]), np.array([b for _, b in e]), np.ones(15)
    if name == "Q3":
        e = [(u, u ^ (1 << d)) for u in range(8) for d in range(3) if u < u ^ (1 << d)]
        return 8, np.array([a for a, _ in e]), np.array([b for _, b in e]), np.ones(len(e))
    raise KeyError(name)


def named_problem(name):
    n, i, j, w = named_graph(name)
    return I.maxcut_from_edges(n, i, j, w, name=name)


def load_sdp_values(path):
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, n, val = line.split()
        out[name] = (int(n), float(val))
    return out


def brute_force_maxcut(n, i, j, w):
    """max over x in {+-1}^n of sum_edges w (1 - x_i x_j)/2, by enumeration (n <= 20)."""
    best = -np.inf
    i, j, w = np.asarray(i), np.asarray(j), np.asarray(w, float)
    for start in range(0, 1 << (n - 1), 1 << 12):
        codes = np.arange(start, min(start + (1 << 12), 1 << (n - 1)))
        bits = ((codes[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int8)
        cut = (bits[:, i] != bits[:, j]).astype(float) @ w
        best = max(best, cut.max())
    return best
