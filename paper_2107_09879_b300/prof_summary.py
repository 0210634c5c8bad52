"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) by kernel:
launches, total device time and share. Usage: python -m paper_2107_09879_b300.prof_summary launches.csv"""
import collections
import csv
import sys

SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3, "second": 1e3}


def main(path):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, mi, vi, ui = (hdr.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        ms = float(r[vi].replace(",", "")) * SCALE[r[ui]]
        name = r[ki].split("(")[0].replace("void ", "")
        agg[name][0] += 1
        agg[name][1] += ms
    tot = sum(v[1] for v in agg.values())
    print(f"{sum(v[0] for v in agg.values())} launches, {tot:.1f} ms device time (serialised, cold cache)")
    print(f"{'kernel':72s} {'launches':>8s} {'total ms':>10s} {'share':>7s}")
    for k, (c, ms) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"{k[:72]:72s} {c:8d} {ms:10.2f} {100 * ms / tot:6.2f}%")


if __name__ == "__main__":
    main(sys.argv[1])
