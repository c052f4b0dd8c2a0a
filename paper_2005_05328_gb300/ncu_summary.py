"""Summarise an ncu CSV launch list (``--metrics gpu__time_duration.sum --csv``)
per kernel: launches, total device time and share, as a Markdown table.

usage: python -m paper_2005_05328_gb300.ncu_summary launches.csv [--skip-ids N]
"""
import collections
import csv
import re
import sys


def summarise(path, skip_ids=0):
    rows = list(csv.reader(open(path)))
    hdr_i = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hdr_i]
    ki, vi, ii = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("ID")
    mi = hdr.index("Metric Name")
    tot = collections.OrderedDict()
    for r in rows[hdr_i + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum" or int(r[ii]) < skip_ids:
            continue
        name = re.sub(r"\(.*$", "", r[ki]).replace("(anonymous namespace)::", "").replace("unnamed>::", "")
        m = re.search(r"<(float|double)>", r[ki])
        if m:
            name += "<%s>" % m.group(1)
        c, t = tot.get(name, (0, 0.0))
        tot[name] = (c + 1, t + float(r[vi]))
    total = sum(t for _, t in tot.values())
    out = ["| kernel | launches | total ms | share |", "|---|---:|---:|---:|"]
    for name, (c, t) in sorted(tot.items(), key=lambda kv: -kv[1][1]):
        out.append("| %s | %d | %.3f | %.1f%% |" % (name, c, t / 1e6, 100 * t / total))
    out.append("| **all** | %d | %.3f | 100%% |" % (sum(c for c, _ in tot.values()), total / 1e6))
    return "\n".join(out)


if __name__ == "__main__":
    skip = 0
    if "--skip-ids" in sys.argv:
        skip = int(sys.argv[sys.argv.index("--skip-ids") + 1])
    print(summarise(sys.argv[1], skip))
