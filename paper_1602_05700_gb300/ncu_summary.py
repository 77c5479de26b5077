"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) into per-kernel launches, time and share.

usage: python -m paper_1602_05700_gb300.ncu_summary launches.csv
"""
import collections
import csv
import sys

SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3, "second": 1e3}


def short(name: str) -> str:
    base = name.split("(")[0]
    return base.replace("void ", "").strip()


def main(path):
    rows = list(csv.reader(open(path)))
    h = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[h]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[h + 1:]:
        if len(r) <= vi or not r[vi]:
            continue
        agg[short(r[ki])][0] += 1
        agg[short(r[ki])][1] += float(r[vi].replace(",", "")) * SCALE[r[ui]]
    tot = sum(a[1] for a in agg.values())
    print(f"{'kernel':70s} {'launches':>8s} {'total ms':>10s} {'share':>7s}")
    for k, (n, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"{k[:70]:70s} {n:8d} {t:10.3f} {100 * t / tot:6.2f}%")
    print(f"{'total':70s} {sum(a[0] for a in agg.values()):8d} {tot:10.3f}")


if __name__ == "__main__":
    main(sys.argv[1])
