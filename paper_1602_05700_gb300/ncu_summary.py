"""Summaries of Nsight Compute output for the notes under profiles/.

  python -m paper_1602_05700_gb300.ncu_summary launches.csv
      per-kernel launches, total time and share of an ncu launch list (--metrics gpu__time_duration.sum --csv)
  python -m paper_1602_05700_gb300.ncu_summary --report capture.ncu-rep
      the headline counters of each captured launch (reads the report with `ncu -i ... --page raw --csv`)
"""
import collections
import csv
import io
import subprocess
import sys

SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3, "second": 1e3}

REPORT_METRICS = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("lts__t_sector_hit_rate.pct", "L2 hit rate %"),
    ("sm__throughput.avg.pct_of_peak_sustained_elapsed", "SM throughput %"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
    ("sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "FMA pipe %"),
    ("sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active", "ALU pipe %"),
    ("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active", "FP64 pipe %"),
    ("sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active", "tensor pipe %"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active %"),
    ("launch__registers_per_thread", "registers/thread"),
    ("launch__occupancy_limit_registers", "blocks/SM (register limit)"),
    ("launch__grid_size", "grid"),
    ("launch__block_size", "block"),
    ("sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active", "LSU issue %"),
    ("sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active", "XU issue %"),
    ("sm__inst_executed_pipe_adu.avg.pct_of_peak_sustained_active", "ADU issue %"),
    ("smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio", "stall long scoreboard"),
    ("smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio", "stall short scoreboard"),
    ("smsp__average_warps_issue_stalled_wait_per_issue_active.ratio", "stall wait"),
    ("smsp__average_warps_issue_stalled_lg_throttle_per_issue_active.ratio", "stall LG throttle"),
    ("smsp__average_warps_issue_stalled_mio_throttle_per_issue_active.ratio", "stall MIO throttle"),
    ("smsp__average_warps_issue_stalled_not_selected_per_issue_active.ratio", "stall not selected"),
    ("smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio", "stall barrier"),
    ("smsp__average_warps_issue_stalled_math_pipe_throttle_per_issue_active.ratio", "stall math pipe"),
    ("smsp__inst_executed.sum", "warp instructions"),
]


def short(name: str) -> str:
    for ns in ("(anonymous namespace)::", "<unnamed>::", "unnamed>::", "hg::"):
        name = name.replace(ns, "")
    return name.split("(")[0].replace("void ", "").strip()


def launches(path):
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
    print(f"| kernel | launches | total ms | share |\n|---|---|---|---|")
    for k, (n, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"| `{k}` | {n} | {t:.3f} | {100 * t / tot:.2f}% |")
    print(f"| total | {sum(a[0] for a in agg.values())} | {tot:.3f} | |")


def report(path):
    out = subprocess.run(["ncu", "-i", path, "--page", "raw", "--csv"], capture_output=True, text=True, check=True)
    rows = list(csv.reader(io.StringIO(out.stdout)))
    hdr, units = rows[0], rows[1]
    for launch in rows[2:]:
        name = short(launch[hdr.index("Kernel Name")]) if "Kernel Name" in hdr else "?"
        print(f"launch: `{name}`\n\n| counter | value |\n|---|---|")
        for metric, label in REPORT_METRICS:
            if metric in hdr:
                i = hdr.index(metric)
                print(f"| {label} (`{metric}`) | {launch[i]} {units[i]} |")
        print()


if __name__ == "__main__":
    if len(sys.argv) == 3 and sys.argv[1] == "--report":
        report(sys.argv[2])
    else:
        launches(sys.argv[1])
