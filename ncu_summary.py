"""Summaries of Nsight Compute CSV output as markdown tables.

    python ncu_summary.py launches LAUNCHES.csv
        per kernel: launches, total gpu__time_duration, share of the total
        (input: ncu --metrics gpu__time_duration.sum --csv --log-file ...)
    python ncu_summary.py raw RAW.csv
        per captured launch: the DRAM, throughput, tensor/FP pipe, occupancy
        and stall counters used for the roofline
        (input: ncu -i REPORT.ncu-rep --page raw --csv > RAW.csv)

Reads text only; nothing here touches a GPU.
"""
import collections
import csv
import sys

_UNIT_US = {"nsecond": 1e-3, "ns": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3,
            "second": 1e6, "s": 1e6}

RAW_METRICS = (
    "gpu__time_duration.sum",
    "dram__bytes_read.sum",
    "dram__bytes_write.sum",
    "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed",
    "dram__throughput.avg.pct_of_peak_sustained_elapsed",
    "sm__throughput.avg.pct_of_peak_sustained_elapsed",
    "lts__t_bytes.sum",
    "l1tex__t_sector_hit_rate.pct",
    "lts__t_sector_hit_rate.pct",
    "sm__warps_active.avg.pct_of_peak_sustained_active",
    "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active",
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active",
    "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active",
    "launch__registers_per_thread",
    "launch__grid_size",
    "launch__block_size",
    "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_lg_throttle_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_math_pipe_throttle_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio",
)


def _lines(path):
    with open(path, newline="") as f:
        return [l for l in f if not l.startswith("==")]


def _short(name):
    name = name.replace("void ", "")
    depth, out = 0, []
    for ch in name:  # drop the argument list, keep template arguments
        if ch == "(" and depth == 0:
            break
        depth += ch == "<"
        depth -= ch == ">"
        out.append(ch)
    return "".join(out).strip()


def launches(path):
    per = collections.OrderedDict()
    tot, n = 0.0, 0
    for row in csv.DictReader(_lines(path)):
        if row.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = _short(row.get("Kernel Name") or row.get("Function Name") or "?")
        v = float(row["Metric Value"].replace(",", "")) * _UNIT_US.get(row.get("Metric Unit", "ns"), 1e-3)
        c = per.setdefault(name, [0, 0.0])
        c[0] += 1
        c[1] += v
        tot += v
        n += 1
    out = ["launches %d, total %.1f us" % (n, tot), "",
           "| kernel | launches | total us | us/launch | share |", "|---|---|---|---|---|"]
    for k, (c, t) in sorted(per.items(), key=lambda kv: -kv[1][1]):
        out.append("| `%s` | %d | %.1f | %.2f | %.2f%% |" % (k, c, t, t / c, 100.0 * t / tot))
    return "\n".join(out)


def raw(path):
    rows = list(csv.reader(_lines(path)))
    head = rows[0]
    units = rows[1] if len(rows) > 1 and not rows[1][0].strip().isdigit() else None
    body = rows[2:] if units else rows[1:]
    col = {h: i for i, h in enumerate(head)}
    name_col = col.get("Kernel Name", None)
    out = []
    for r in body:
        out.append("### `%s`" % (_short(r[name_col]) if name_col is not None else "?"))
        out.append("")
        out.append("| metric | value | unit |")
        out.append("|---|---|---|")
        for m in RAW_METRICS:
            if m in col:
                out.append("| %s | %s | %s |" % (m, r[col[m]], units[col[m]] if units else ""))
        out.append("")
    return "\n".join(out)


def main(argv):
    if len(argv) != 3 or argv[1] not in ("launches", "raw"):
        print(__doc__)
        return 2
    print(launches(argv[2]) if argv[1] == "launches" else raw(argv[2]))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
