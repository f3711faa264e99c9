"""Summaries of ncu output for the profiles/ notes.

  python -m paper_1806_06204_gb300.ncu_summary launches <launches.csv>
      per kernel: launches, summed gpu__time_duration, share (ncu --csv of
      `--metrics gpu__time_duration.sum`)
  python -m paper_1806_06204_gb300.ncu_summary raw <raw.csv>
      selected counters per captured launch (ncu -i rep --page raw --csv)
"""
from __future__ import annotations

import collections
import csv
import re
import sys

UNIT_MS = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0,
           "s": 1e3, "second": 1e3}

RAW = ["gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
       "sm__throughput.avg.pct_of_peak_sustained_elapsed",
       "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active",
       "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active",
       "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed",
       "sm__warps_active.avg.pct_of_peak_sustained_active",
       "launch__registers_per_thread", "launch__grid_size", "launch__block_size"]


def short(name: str) -> str:
    name = re.sub(r"\(.*", "", name)                 # drop the parameter list
    name = name.replace("void ", "").replace("zolo::", "").replace("<unnamed>::", "")
    return name.strip()


def launches(path: str) -> str:
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    k, m, u, v = (h.index(x) for x in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value"))
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hi + 1:]:
        if len(r) <= v or r[m] != "gpu__time_duration.sum":
            continue
        ms = float(r[v].replace(",", "")) * UNIT_MS.get(r[u], 1.0)
        a = agg[short(r[k])]
        a[0] += 1
        a[1] += ms
    tot = sum(x[1] for x in agg.values())
    out = [f"{'kernel':58s} {'launches':>8s} {'total ms':>10s} {'share':>7s}"]
    for name, (c, ms) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append(f"{name[:58]:58s} {c:8d} {ms:10.3f} {100 * ms / tot:6.2f}%")
    out.append(f"{'total':58s} {sum(x[0] for x in agg.values()):8d} {tot:10.3f}")
    return "\n".join(out)


def raw(path: str) -> str:
    rows = list(csv.reader(open(path)))
    h, units = rows[0], rows[1]
    out = []
    for r in rows[2:]:
        out.append(short(r[h.index("Kernel Name")]))
        for name in RAW:
            if name in h:
                i = h.index(name)
                out.append(f"    {name:62s} {r[i]:>14s} {units[i]}")
    return "\n".join(out)


if __name__ == "__main__":
    print(launches(sys.argv[2]) if sys.argv[1] == "launches" else raw(sys.argv[2]))
