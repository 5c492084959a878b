"""Summarise an ncu launch list (``--metrics gpu__time_duration.sum --csv``) per kernel.

Usage: python -m paper_2312_11801_gb300.ncu_summary launches.csv [--top 20]

Prints, per kernel name (template arguments kept), the number of launches, the total
and mean device time and the share of the total, largest first, as a Markdown table.
ncu serialises launches and runs them with cold caches, so the shares, not the absolute
times, are what compares with timings taken without the profiler.
"""
import argparse
import collections
import csv
import io
import sys


def read_launches(path):
    """(kernel name, nanoseconds) for every captured launch in an ncu CSV log."""
    text = open(path, encoding="utf-8", errors="replace").read()
    start = text.find('"ID"')
    if start < 0:
        raise ValueError(f"{path}: no ncu CSV header found")
    rows = csv.DictReader(io.StringIO(text[start:]))
    out = []
    for r in rows:
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        v = float(r["Metric Value"].replace(",", ""))
        unit = r.get("Metric Unit", "nsecond")
        scale = {"nsecond": 1.0, "usecond": 1e3, "msecond": 1e6, "second": 1e9}.get(unit, 1.0)
        out.append((r["Kernel Name"], v * scale))
    return out


def summarise(launches):
    agg = collections.defaultdict(lambda: [0, 0.0])
    for name, ns in launches:
        agg[name][0] += 1
        agg[name][1] += ns
    total = sum(v[1] for v in agg.values()) or 1.0
    rows = sorted(((k, n, t) for k, (n, t) in agg.items()), key=lambda x: -x[2])
    return rows, total


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--top", type=int, default=25)
    a = ap.parse_args(argv)
    rows, total = summarise(read_launches(a.csv))
    n_all = sum(r[1] for r in rows)
    print(f"{n_all} launches, {total / 1e6:.3f} ms total device time\n")
    print("| kernel | launches | total ms | mean us | share |")
    print("|---|---:|---:|---:|---:|")
    for name, n, t in rows[: a.top]:
        short = name if len(name) <= 60 else name[:57] + "..."
        print(f"| `{short}` | {n} | {t / 1e6:.3f} | {t / n / 1e3:.2f} | {100 * t / total:.1f}% |")
    rest = rows[a.top:]
    if rest:
        n_r, t_r = sum(r[1] for r in rest), sum(r[2] for r in rest)
        print(f"| (other {len(rest)} kernels) | {n_r} | {t_r / 1e6:.3f} | | {100 * t_r / total:.1f}% |")
    return 0


if __name__ == "__main__":
    sys.exit(main())
