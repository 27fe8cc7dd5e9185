"""Summarise an ncu launch list (``--metrics gpu__time_duration.sum --csv``):
per kernel, launches, total device time and share.  Usage:
    python -m paper_1506_04694_gb300.ncu_summary launches.csv [--skip N] [--from TEXT]
--skip N leaves out the first N launches (e.g. the set-up of a benchmark:
embedding tables and the launch-plan autotuner); --from TEXT leaves out every
launch before the first kernel whose name contains TEXT (bench.py's L2 flush,
a PyTorch fill kernel, marks the start of its timed steps)."""
import collections
import csv
import sys

UNITS = {"ns": 1.0, "nsecond": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6,
         "s": 1e9, "second": 1e9}


def summarise(path, skip=0, start_at=None):
    rows = list(csv.reader(open(path)))
    start = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[start]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    idi = hdr.index("ID") if "ID" in hdr else None
    agg = collections.OrderedDict()
    seen = start_at is None
    for n, r in enumerate(rows[start + 1:]):
        if len(r) <= vi or not r[vi]:
            continue
        if (int(r[idi]) if idi is not None else n) < skip:
            continue
        if not seen:
            if start_at not in r[ki]:
                continue
            seen = True
        name = r[ki].split("(")[0].strip()
        ns = float(r[vi].replace(",", "")) * UNITS[r[ui].strip()]
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += ns
    tot = sum(a[1] for a in agg.values())
    out = ["%-48s %8s %12s %7s" % ("kernel", "launches", "total ms", "share")]
    for k, (n, ns) in sorted(agg.items(), key=lambda x: -x[1][1]):
        out.append("%-48s %8d %12.3f %6.2f%%" % (k[:48], n, ns / 1e6, 100 * ns / tot))
    out.append("%-48s %8d %12.3f" % ("total", sum(a[0] for a in agg.values()), tot / 1e6))
    return "\n".join(out)


if __name__ == "__main__":
    skip = int(sys.argv[sys.argv.index("--skip") + 1]) if "--skip" in sys.argv else 0
    start_at = sys.argv[sys.argv.index("--from") + 1] if "--from" in sys.argv else None
    print(summarise(sys.argv[1], skip, start_at))
