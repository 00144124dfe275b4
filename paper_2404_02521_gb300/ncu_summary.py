"""Summaries of Nsight Compute output for the library's kernels (host-side tooling).

    python -m paper_2404_02521_gb300.ncu_summary launches <launch-list.csv>
        per kernel: launches, summed gpu__time_duration, share of the listed time
    python -m paper_2404_02521_gb300.ncu_summary report <capture.ncu-rep>
        the headline counters of each captured launch (time, DRAM bytes and throughput,
        pipe utilisation, occupancy, the largest warp-stall reasons)
    python -m paper_2404_02521_gb300.ncu_summary traffic <capture.ncu-rep> <kernel> <json> [--states S] <src>...
        record the DRAM bytes (read + write) per launch of <kernel> in <json> (and per state
        when the captured launches carried S states each), with the sha256 of the kernel's
        source files (a later source change invalidates the entry)

The launch list comes from `ncu --metrics gpu__time_duration.sum --csv --log-file`; a capture
from `ncu --set full -o`.  Reading a capture runs `ncu -i <file> --page raw --csv`.
"""
from __future__ import annotations

import collections
import csv
import hashlib
import io
import json
import os
import subprocess
import sys

_UNIT = {"ns": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3, "second": 1e3,
         "nsecond": 1e-6}
_BYTES = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}


def _short(name: str) -> str:
    name = name.split("(")[0]
    return name.replace("void ", "").replace("bsp::", "")


def launches(path: str) -> str:
    with open(path) as f:
        rows = [r for r in csv.reader(f)]
    head = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    hdr = rows[head]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    agg = collections.OrderedDict()
    for r in rows[head + 1:]:
        if len(r) < len(hdr):
            continue
        ms = float(r[vi].replace(",", "")) * _UNIT.get(r[ui], 1.0)
        k = _short(r[ki])
        n, t = agg.get(k, (0, 0.0))
        agg[k] = (n + 1, t + ms)
    total = sum(t for _, t in agg.values())
    out = ["| kernel | launches | total ms | share |", "|---|---:|---:|---:|"]
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append(f"| `{k}` | {n} | {t:.2f} | {100 * t / total:.1f}% |")
    out.append(f"| all | {sum(n for n, _ in agg.values())} | {total:.2f} | 100% |")
    return "\n".join(out)


def _raw(path: str):
    txt = subprocess.run(["ncu", "-i", path, "--page", "raw", "--csv"], check=True,
                         capture_output=True, text=True).stdout
    rows = list(csv.reader(io.StringIO(txt)))
    return rows[0], rows[1], rows[2:]


_REPORT = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("sm__throughput.avg.pct_of_peak_sustained_elapsed", "SM throughput % of peak"),
    ("sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "FMA pipe % active"),
    ("sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active", "tensor pipe % active"),
    ("sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active", "LSU pipe % active"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue slots busy %"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "achieved occupancy %"),
    ("launch__registers_per_thread", "registers / thread"),
    ("launch__grid_size", "grid (CTAs)"),
    ("launch__cluster_dim_x", "cluster size"),
]


def report(path: str) -> str:
    hdr, units, rows = _raw(path)
    out = []
    for r in rows:
        out.append(f"### `{_short(r[hdr.index('Kernel Name')])}`")
        out.append("| counter | value |")
        out.append("|---|---:|")
        for key, label in _REPORT:
            if key in hdr:
                i = hdr.index(key)
                out.append(f"| {label} (`{key}`) | {r[i]} {units[i]} |")
        stalls = []
        for i, h in enumerate(hdr):
            if h.startswith("smsp__average_warps_issue_stalled_") and h.endswith("_per_issue_active.ratio"):
                try:
                    stalls.append((float(r[i]), h[len("smsp__average_warps_issue_stalled_"):-len(
                        "_per_issue_active.ratio")]))
                except ValueError:
                    pass
        top = ", ".join(f"{n} {v:.2f}" for v, n in sorted(stalls, reverse=True)[:5])
        out.append(f"| largest stalls (warps per issue) | {top} |")
        out.append("")
    return "\n".join(out)


def sources_sha256(root: str, files) -> str:
    h = hashlib.sha256()
    for s in files:
        with open(os.path.join(root, s), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic(path: str, kernel: str, json_path: str, sources, states: int = 0) -> dict:
    hdr, units, rows = _raw(path)
    ki = hdr.index("Kernel Name")
    sel = [r for r in rows if kernel in r[ki]]
    if not sel:
        raise SystemExit(f"no launch of {kernel} in {path}")
    per = []
    for r in sel:
        b = 0.0
        for key in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            i = hdr.index(key)
            b += float(r[i].replace(",", "")) * _BYTES.get(units[i], 1.0)
        per.append(b)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    d = {}
    if os.path.exists(json_path):
        with open(json_path) as f:
            d = json.load(f)
    d[kernel] = {"dram_bytes_per_launch_full": sum(per) / len(per), "launches_captured": len(per),
                 "capture": os.path.basename(path), "sources": list(sources),
                 "source_sha256": sources_sha256(root, sources)}
    if states > 0:
        d[kernel]["states_per_launch_captured"] = states
        d[kernel]["dram_bytes_per_state_launch"] = sum(per) / len(per) / states
    with open(json_path, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
        f.write("\n")
    return d[kernel]


def main(argv):
    if len(argv) >= 2 and argv[0] == "launches":
        print(launches(argv[1]))
    elif len(argv) >= 2 and argv[0] == "report":
        print(report(argv[1]))
    elif len(argv) >= 5 and argv[0] == "traffic":
        rest, states = argv[4:], 0
        if rest[:1] == ["--states"]:
            states, rest = int(rest[1]), rest[2:]
        print(json.dumps(traffic(argv[1], argv[2], argv[3], rest, states)))
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
