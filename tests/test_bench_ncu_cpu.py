"""bench.py's ncu tooling (no GPU): kernel names map to the library's profile
groups, both ncu CSV layouts are read with their units, and the DRAM over
algorithmic-bytes ratio recorded from a capture scales the roofline traffic
only while the kernel sources are the ones it was taken on."""
import csv
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

NAMES = {
    "void cd::<unnamed>::k_hub_build_cl<cd::WUnit, 0>(cd::<unnamed>::ScanCtx)": "hub_build",
    "void unnamed>::k_hub_build<WI32, unsigned int>(unnamed>::ScanCtx)": "hub_build",
    "cd::<unnamed>::k_hub_prepare(cd::<unnamed>::ScanCtx)": "hub_prepare",
    "cd::<unnamed>::k_hub_route(cd::<unnamed>::ScanCtx, int *, int *, unsigned long long *)": "hub_prepare",
    "void unnamed>::k_hub_eval_small<1, 1>(unnamed>::ScanCtx)": "hub_eval",
    "void unnamed>::k_hub_eval<0, 0>(unnamed>::ScanCtx)": "hub_eval",
    "cd::<unnamed>::k_hub_apply_log(cd::<unnamed>::ScanCtx)": "hub_mark",
    "void unnamed>::k_scan_group<1, WI32, unsigned int, 128, 512, 2048, 5, 0, 1>(unnamed>::ScanCtx, const int *)":
        "scan_blk128",
    "void unnamed>::k_scan_group<0, WUnit, unsigned int, 512, 512, 8192, 6, 0, 0>(unnamed>::ScanCtx)": "scan_blk512",
    "void unnamed>::k_scan_tile<16, 1, WI32, 1>(unnamed>::ScanCtx, const int *)": "scan_tile16",
    "void unnamed>::k_scan_warp<1, WI32, unsigned int, 1>(unnamed>::ScanCtx, const int *)": "scan_warp",
    "void unnamed>::k_first_round<1, WUnit, 1, 32>(unnamed>::ScanCtx, const int *)": "first round (every bin)",
    "cd::<unnamed>::k_compact(cd::<unnamed>::ScanCtx, const int *)": "frontier",
    "void cd::<unnamed>::k_ag_cta<1>(const long *)": "aggregation and radix sort",
    "cd::<unnamed>::k_rs_scatter(const unsigned long *)": "aggregation and radix sort",
    "<unnamed>::rmat_keys_kernel(unsigned long, int)": "input generator and PyTorch",
    "void native::vectorized_elementwise_kernel<4>(int)": "input generator and PyTorch",
}


@pytest.mark.parametrize("name,group", list(NAMES.items()))
def test_kernel_group(name, group):
    assert bench.kernel_group(name) == group


def write_csv(path, rows):
    with open(path, "w", newline="") as f:
        csv.writer(f, quoting=csv.QUOTE_ALL).writerows(rows)


HDR = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
       "Grid Size", "Device", "CC"]


def long_rows():
    """ncu --csv --log-file layout: one row per metric per launch (after ncu's own log lines)."""
    rows = [HDR + ["Section Name", "Metric Name", "Metric Unit", "Metric Value"]]
    launches = [("k_hub_build_cl<cd::WUnit, 0>(x)", 2_000_000, 300.0, 500.0),
                ("k_hub_build_cl<cd::WUnit, 1>(x)", 1_000_000, 100.0, 100.0),
                ("k_hub_prepare(x)", 500_000, 1.0, 0.5),
                ("k_scan_warp<1, WI32, unsigned int, 1>(x)", 3_000_000, 900.0, 10.0)]
    for i, (name, ns, rd, wr) in enumerate(launches):
        base = [str(i), "1", "python3.12", "127.0.0.1", "void cd::<unnamed>::" + name, "1", "7", "(256, 1, 1)",
                "(608, 1, 1)", "0", "10.3", "Command line profiler metrics"]
        rows.append(base + ["gpu__time_duration.sum", "ns", f"{ns:,}"])
        rows.append(base + ["dram__bytes_read.sum", "Mbyte", f"{rd}"])
        rows.append(base + ["dram__bytes_write.sum", "Mbyte", f"{wr}"])
    return rows


def wide_rows():
    """ncu -i report --page raw --csv layout: one row per launch, a units row first."""
    rows = [HDR + ["dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum"],
            [""] * len(HDR) + ["Gbyte", "Gbyte", "ms"],
            ["0", "1", "python3.12", "h", "void unnamed>::k_scan_warp<1, WI32, unsigned int, 1>(unnamed>::ScanCtx)",
             "1", "7", "(256, 1, 1)", "(608, 1, 1)", "0", "10.3", "0.926", "0.007", "1.981"],
            ["1", "1", "python3.12", "h",
             "void unnamed>::k_scan_group<1, WI32, unsigned int, 128, 512, 2048, 5, 0, 1>(unnamed>::ScanCtx)",
             "1", "7", "(512, 1, 1)", "(304, 1, 1)", "0", "10.3", "0.433", "0.004", "0.821"]]
    return rows


def summary_table(capsys):
    out = capsys.readouterr().out
    table = {}
    for line in out.splitlines():
        cells = [c.strip() for c in line.strip("|").split("|")]
        if len(cells) == 5 and cells[1].isdigit():
            table[cells[0]] = (int(cells[1]), float(cells[2]), float(cells[4]))
    return table


def test_summary_long_layout(tmp_path, capsys):
    p = tmp_path / "launches.csv"
    with open(p, "w") as f:  # ncu prefixes its log lines
        f.write("==PROF== Connected to process 1\n")
    with open(p, "a", newline="") as f:
        csv.writer(f, quoting=csv.QUOTE_ALL).writerows(long_rows())
    bench.ncu_summary(str(p))
    t = summary_table(capsys)
    assert t["hub_build"] == (2, 3.0, 1000.0)  # ms summed, DRAM MB read + write summed
    assert t["hub_prepare"] == (1, 0.5, 1.5)
    assert t["scan_warp"] == (1, 3.0, 910.0)


def test_summary_wide_layout_and_traffic(tmp_path, capsys, monkeypatch):
    p = tmp_path / "raw.csv"
    write_csv(p, wide_rows())
    case = tmp_path / "case.json"
    case.write_text(json.dumps({"case": "level1", "scale": 23, "captured": "coarse-graph round 3",
                                "alg_bytes": {"scan_warp": 1.0e9, "scan_blk128": 0.5e9}}))
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2507_06471_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in ("scan.cu", "graph.cu", "common.cuh"):
        (csrc / name).write_text("// " + name + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    bench.ncu_summary(str(p), str(case))
    t = summary_table(capsys)
    assert t["scan_warp"][0] == 1 and abs(t["scan_warp"][1] - 1.981) < 0.05  # printed to 0.1 ms
    assert abs(t["scan_warp"][2] - 933.0) < 1e-6 and abs(t["scan_blk128"][2] - 437.0) < 1e-6
    traffic = json.loads((tmp_path / "profiles" / "traffic.json").read_text())
    assert abs(traffic["scan_warp"]["dram_bytes"] - 933.0e6) < 1.0
    # the bench scales the recorded ratio to a launch's algorithmic bytes
    t_b, src = bench.ncu_traffic("scan_warp", 2.0e9)
    assert abs(t_b - 2.0 * 933.0e6) < 10.0 and abs(src["dram_over_alg"] - 0.933) < 1e-9
    assert bench.ncu_traffic("hub_build", 1.0e9) == (None, None)  # no capture covers it
    (csrc / "scan.cu").write_text("// changed kernel source\n")
    assert bench.ncu_traffic("scan_warp", 2.0e9) == (None, None)  # stale once the sources change
