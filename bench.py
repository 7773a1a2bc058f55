#!/usr/bin/env python
"""Benchmark: Louvain + LPA on one GB300 per rank, through the C ABI.

One step = the whole hot path on one synthetic graph already resident in HBM:
ingest (validate, deg_w, vol, degree bins), Label Propagation to convergence
(Algorithm 1), Louvain to convergence (Algorithm 2 local moving + Algorithm 3
aggregation per level) and the modularity of the result.

value  = arcs scanned by all LPA and Louvain rounds of the step / step time
         (GTEPS, device time from CUDA events on the library's stream);
e2e    = the same through the C ABI with HOST buffers: the CSR is copied from
         pinned host memory inside the timed region and both label arrays are
         copied back;
roofline = the dominant kernel's algorithmic bytes per launch / its average
         CUDA-event launch time, against the measured HBM copy bandwidth.

Multi-GPU: the path does not shard a single graph here (replicas only): under
torchrun every rank solves its own copy of the workload; value sums all ranks'
arcs over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC_GTEPS = "GTEPS per iteration (arcs scanned by all LPA + Louvain rounds / step time)"
METRIC_BATCH = "batched graphs/s (Louvain to convergence, all graphs in one call)"
METRIC_SERVE = "requests/s (LPA or Louvain to convergence per request, continuous batching)"

WORKLOADS = {
    # name: (description, builder kwargs)
    "rmat26": "R-MAT scale 26, edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05), deduplicated, "
              "symmetrised, loops removed, unit weights, ids unpermuted, seed 3",
    "lfr1m": "LFR-style n = 1,000,000, degree power law 2.5 on [5,1000], community sizes 1.5 on "
             "[20,5000], mu = 0.3, weights U{1..8}, seed 2",
    "sbm10k": "planted-partition SBM n = 10,000, 100 blocks, p_in = 0.1, p_out = 0.001, seed 1",
    "batch4096": "4,096 planted-partition SBM graphs, n log-uniform in [50, 5000], k uniform in {2..50}, "
                 "p_in = 0.2, p_out = 0.002, weights U{1..4}, seeds 4+b, packed block-diagonally",
    "serve2048": "stream of 2,048 requests (1/3 LPA, 2/3 Louvain, seeded): 1,984 planted-partition SBM "
                 "graphs as in batch4096, 48 SBM graphs with n log-uniform in [10,000, 30,000] and "
                 "blocks of 100, 16 R-MAT graphs of scale 14-17 (edge factor 16); host buffers",
    "served": "the first --serve-requests of a 20,000-request stream, seed 5: n log-uniform in [100, 2e6], "
              "70% Louvain / 30% LPA, half R-MAT (edge factor 8 at scale ceil(log2 n), endpoints >= n "
              "rejected), half edge-sampled planted partition (k uniform in {2..50}, mean degree 16, "
              "p_out = p_in / 100); unit weights; host buffers",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="rmat26")
    ap.add_argument("--scale", type=int, default=None, help="override the R-MAT scale")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-arcs", type=float, default=2e8,
                    help="arcs per round of the oracle sample timed for cpu_baseline (about 20 s)")
    ap.add_argument("--ref-sample-arcs", type=float, default=2e7,
                    help="--impl reference: arcs per round of the oracle sample of each step (about 2 s)")
    ap.add_argument("--no-many", action="store_true",
                    help="R-MAT line only: skip the batched and served parts of the metric")
    ap.add_argument("--many-steps", type=int, default=3, help="timed steps of the batched and served parts")
    ap.add_argument("--served-in-line", type=int, default=256,
                    help="requests of the 20,000-request stream run in the R-MAT line's served part")
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--asynchronous", action="store_true",
                    help="the asynchronous variant (moves take effect at once; not reproducible)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-requests", type=int, default=512,
                    help="served: how many requests of the 20,000-request stream to run")
    ap.add_argument("--solo-sample", type=int, default=128,
                    help="batch workload: graphs timed one call per graph for the comparison")
    ap.add_argument("--case", choices=["level1", "first-rounds"], default=None,
                    help="profiling cases on R-MAT at --scale (default 23), run under ncu: 'level1' runs "
                         "level 0 to convergence, aggregates, then local moving on the coarse graph with "
                         "max_iter 3 and 4, the second inside cudaProfilerStart/Stop, and prints the "
                         "algorithmic bytes of round 3 per kernel; 'first-rounds' runs LPA and local moving "
                         "with max_iter 2 (round 1 builds every hub table) and prints the algorithmic "
                         "bytes of the LPA run per kernel")
    ap.add_argument("--ncu-summary", nargs="+", default=None, metavar="CSV",
                    help="summarise an ncu --csv launch list per kernel group (no GPU needed); with a "
                         "--case JSON as second argument, record the DRAM bytes of the captured launches "
                         "over their algorithmic bytes in profiles/traffic.json")
    return ap.parse_args()


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units: float, seconds: float, world: int) -> float:
    """Whole-job throughput of replicas: the units of all ranks over the slowest rank's time."""
    return allreduce_sum(float(units), world) / allreduce_max(float(seconds), world)


# the schedule parameters every timed run uses (cd_params_default)
RUN_PARAMS = {"max_iter": 100, "max_levels": 64, "threshold": 0}


def graph_config(args, scale, n, nnz, world):
    """The workload description both arms report."""
    return {"workload": f"{args.workload}" + (f"_scale{scale}" if scale else ""),
            "description": WORKLOADS[args.workload], "n": n, "arcs": nnz,
            "l2": "inputs larger than L2 (column array %.1f GB)" % (nnz * 4 / 1e9),
            "parallelism": f"replicas x{world}",
            "schedule": ("asynchronous rounds (moves applied at once), " if args.asynchronous else
                         "synchronous rounds, ") + "SplitMix64 deferral coin, strict-positive gain, "
                        "smallest-id ties, singleton rule",
            **RUN_PARAMS, "asynchronous": bool(args.asynchronous)}


def make_graph(name: str, scale_override, device: str):
    import synth
    if name == "rmat26":
        scale = scale_override or 26
        g = synth.rmat(scale, 16, seed=3, device=device)
        g.name = f"rmat{scale}_ef16"
        return g, scale
    if name == "lfr1m":
        return synth.lfr(1_000_000, seed=2).to(device), None
    return synth.sbm(10000, 100, "0.1", "0.001", seed=1).to(device), None


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ one step

def run_step(cd, g_dev, params, labels_lpa, labels_lv, host=False, g_host=None):
    """Upload + LPA + Louvain (+ modularity). Returns (arcs, info, profile)."""
    if host:
        h = cd.cd_csr_upload(g_host[0], g_host[1], g_host[2])
    else:
        h = cd.cd_csr_upload(g_dev.off, g_dev.cols, g_dev.w)
    rounds = cd.cd_lpa_run(h, params, labels_lpa)
    tr_lpa = cd.cd_trace_get(h)
    prof_lpa = cd.cd_profile_get(h) if params.timing else []
    levels, q = cd.cd_louvain_run(h, params, labels_lv)
    tr_lv = cd.cd_trace_get(h)
    prof_lv = cd.cd_profile_get(h) if params.timing else []
    cd.cd_graph_free(h)
    arcs = sum(t["arcs"] for t in tr_lpa) + sum(t["arcs"] for t in tr_lv)
    info = {"lpa_rounds": rounds, "louvain_levels": levels, "louvain_rounds": len(tr_lv), "q": q,
            "lpa_arcs": sum(t["arcs"] for t in tr_lpa), "louvain_arcs": sum(t["arcs"] for t in tr_lv),
            "lpa_scan_ms": sum(t["scan_ms"] for t in tr_lpa),
            "louvain_scan_ms": sum(t["scan_ms"] for t in tr_lv),
            "lpa_hit_max_iter": bool(rounds == params.max_iter and tr_lpa and
                                     tr_lpa[-1]["moved"] + tr_lpa[-1]["deferred"] > params.threshold),
            "louvain_levels_detail": level_summary(tr_lv, params.max_iter)}
    return arcs, info, prof_lpa + prof_lv, (tr_lpa, tr_lv)


def level_summary(tr_lv, max_iter):
    """Per Louvain level: rounds, arcs scanned, moves, and whether the level
    stopped at max_iter with vertices still wanting to move."""
    out = []
    for lv in sorted({t["level"] for t in tr_lv}):
        rows = [t for t in tr_lv if t["level"] == lv]
        out.append({"level": lv, "rounds": len(rows), "arcs": sum(t["arcs"] for t in rows),
                    "moved": sum(t["moved"] for t in rows),
                    "hit_max_iter": bool(len(rows) == max_iter and rows[-1]["moved"] + rows[-1]["deferred"] > 0)})
    return out


def round_bytes(t, louv: bool, wbytes: int, n: int) -> float:
    """Algorithmic bytes of one scan round of the method (independent of how
    the kernels organise the work): per examined vertex its offsets (8), label
    (4), label write (4) and flag (1); per scanned arc its column (4), the
    neighbour's label (4) and weight (wbytes); marking the neighbours of moved
    vertices (4 per arc of a moved vertex) and clearing n next-round flags.
    Louvain adds the Sigma_tot gather of every candidate pair (8), deg_w of
    every examined vertex (8) and the Sigma_tot/size updates of every move (24)."""
    b = t["arcs"] * (8 + wbytes) + t["active"] * 17 + 4 * t["moved_arcs"] + n
    if louv:
        b += 8 * t["cands"] + 8 * t["active"] + 24 * t["moved"]
    return float(b)


def round_figures(rows, louv, wbytes, n, peak):
    """Median over steps of one round's device time, with its GTEPS and
    algorithmic GB/s against the HBM peak."""
    ms = statistics.median(t["round_ms"] for t in rows)
    scan_ms = statistics.median(t["scan_ms"] for t in rows)
    t = rows[-1]
    b = round_bytes(t, louv, wbytes, n)
    return {"ms": ms, "scan_ms": scan_ms, "active": t["active"], "arcs": t["arcs"], "cands": t["cands"],
            "moved": t["moved"], "moved_arcs": t["moved_arcs"], "gteps": t["arcs"] / (ms / 1e3) / 1e9,
            "alg_bytes": b, "GBps": b / (ms / 1e3) / 1e9, "frac": b / (ms / 1e3) / 1e9 / peak}


def merge_profiles(acc: dict, prof: list):
    for p in prof:
        a = acc.setdefault(p["name"], {"launches": 0, "total_ms": 0.0, "alg_bytes": 0.0})
        a["launches"] += p["launches"]
        a["total_ms"] += p["total_ms"]
        a["alg_bytes"] += p["alg_bytes"]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# what the library counts as one launch's algorithmic bytes, per profile group
KERNEL_BYTES = {
    "hub_build": "hub-table builds: (column 4 + label 4 + weight) per arc of a rebuilt hub + 8 per table slot "
                 "written (the implementation's data structure, not a per-round figure of the method; the "
                 "method's per-round bytes are under 'rounds')",
    "hub_prepare": "8 per hub-table slot cleared, or read and written by a compaction, + 8 per hub (routing)",
    "hub_eval": "per live histogram entry 24 (+ 8 Sigma_tot for Louvain) + 12 per examined hub",
    "hub_mark": "5 per arc of a moved hub (column, flag) + 64 per logged hub-histogram update",
    "scan_warp": "per examined vertex 13 (+ 24 Louvain) + per scanned arc (column 4 + label 4 + weight) "
                 "+ 8 per candidate pair (Louvain)",
    "scan_blk128": "per examined vertex 13 (+ 24 Louvain) + per scanned arc (column 4 + label 4 + weight) "
                   "+ 8 per candidate pair (Louvain)",
}


def sources_digest() -> str:
    """Digest of the kernel sources a committed ncu figure was taken on."""
    h = hashlib.sha256()
    for name in ("scan.cu", "graph.cu", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2507_06471_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch of `kernel` (a kernel group of the library's
    profile), scaled from a small-case ncu capture: its measured DRAM bytes
    over its algorithmic bytes, times this run's algorithmic bytes per launch.
    None if no capture of the current kernel sources covers the group."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        e = json.load(f).get(kernel)
    if not e or e.get("sources") != sources_digest() or not e.get("alg_bytes"):
        return None, None
    ratio = e["dram_bytes"] / e["alg_bytes"]
    return ratio * alg_bytes_per_launch, {"dram_over_alg": ratio, "from": e["case"], "capture": e["capture"]}


def kernel_group(name: str) -> str:
    """The library's profile group of a kernel named as ncu prints it."""
    import re
    m = re.search(r"\b(k_[A-Za-z0-9_]+)", name)
    if not m:
        return "input generator and PyTorch"
    base = m.group(1)
    rest = name[m.end():]
    targs = rest[1:rest.find(">")].split(",") if rest.startswith("<") else []
    if base in ("k_hub_prepare", "k_hub_route"):
        return "hub_prepare"
    if base in ("k_hub_build_cl", "k_hub_build"):
        return "hub_build"
    if base in ("k_hub_eval_small", "k_hub_eval"):
        return "hub_eval"
    if base in ("k_hub_mark", "k_hub_apply_log"):
        return "hub_mark"
    if base == "k_scan_group" and len(targs) > 3:
        return "scan_blk" + targs[3].strip()
    if base == "k_scan_tile" and targs:
        return "scan_tile" + targs[0].strip()
    if base == "k_scan_warp":
        return "scan_warp"
    if base == "k_first_round":
        return "first round (every bin)"
    if base == "k_compact":
        return "frontier"
    if base in ("k_apply_state", "k_sigma32_moves"):
        return "apply_moves"
    if base.startswith("k_ag_") or base.startswith("k_rs_"):
        return "aggregation and radix sort"
    return "other library kernels"


def ncu_summary(csv_path: str, case_json: str = None):
    """Per kernel group of an ncu --csv log: launches, time, share, and DRAM
    bytes when the log has them. With a --case JSON, records each captured
    group's DRAM bytes over its algorithmic bytes in profiles/traffic.json."""
    import csv
    to_ms = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0}
    to_b = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    hdr, units, rows = None, None, {}
    for r in csv.reader(open(csv_path)):
        if r and r[0] == "ID":
            hdr, units = r, None
            continue
        if not hdr or len(r) != len(hdr):
            continue
        d = dict(zip(hdr, r))
        if "Metric Name" in d:  # one row per metric (ncu --csv --log-file)
            e = rows.setdefault(d["ID"], {"name": d["Kernel Name"]})
            v = float(d["Metric Value"].replace(",", ""))
            unit = d["Metric Unit"]
            if d["Metric Name"] == "gpu__time_duration.sum":
                e["ms"] = v * to_ms.get(unit, 1e-6)
            elif d["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                e["dram"] = e.get("dram", 0.0) + v * to_b.get(unit, 1)
            continue
        if not d["ID"]:  # the units row of a raw page (ncu -i report --page raw --csv)
            units = d
            continue
        e = rows.setdefault(d["ID"], {"name": d["Kernel Name"]})
        u = units or {}
        if d.get("gpu__time_duration.sum"):
            e["ms"] = float(d["gpu__time_duration.sum"].replace(",", "")) * to_ms.get(
                u.get("gpu__time_duration.sum", "nsecond"), 1e-6)
        for k in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            if d.get(k):
                e["dram"] = e.get("dram", 0.0) + float(d[k].replace(",", "")) * to_b.get(u.get(k, "byte"), 1)
    groups = {}
    for e in rows.values():
        g = groups.setdefault(kernel_group(e["name"]), {"launches": 0, "ms": 0.0, "dram": 0.0})
        g["launches"] += 1
        g["ms"] += e.get("ms", 0.0)
        g["dram"] += e.get("dram", 0.0)
    lib_ms = sum(g["ms"] for k, g in groups.items() if k != "input generator and PyTorch")
    print("| kernel group | launches | ms | share of library time | DRAM MB |")
    print("|---|---|---|---|---|")
    for k, g in sorted(groups.items(), key=lambda kv: -kv[1]["ms"]):
        share = f"{100 * g['ms'] / lib_ms:.1f}%" if k != "input generator and PyTorch" and lib_ms else "—"
        print(f"| {k} | {g['launches']} | {g['ms']:.1f} | {share} | {g['dram'] / 1e6:.1f} |")
    if not case_json:
        return
    case = json.load(open(case_json))
    path = os.path.join(ROOT, "profiles", "traffic.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for k, g in groups.items():
        alg = case["alg_bytes"].get(k)
        if not alg or not g["dram"]:
            continue
        out[k] = {"dram_bytes": g["dram"], "alg_bytes": alg, "launches": g["launches"],
                  "case": f"R-MAT {case['scale']}, {case['captured']} ({case['case']})",
                  "capture": os.path.basename(csv_path), "sources": sources_digest()}
        print(f"{k}: DRAM {g['dram'] / 1e6:.1f} MB / algorithmic {alg / 1e6:.1f} MB = {g['dram'] / alg:.2f}")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


# ------------------------------------------------------------------ CPU baseline (oracle)

def oracle_sample(off, cols, w, target_arcs: float, seed: int = 17):
    """The oracle's first LPA round and first Louvain local-move round on the
    same graph, with the initial active set a seeded uniform vertex sample
    holding about target_arcs arcs. Returns (arcs, seconds, description)."""
    import numpy as np
    import oracle
    n = len(off) - 1
    nnz = int(off[-1])
    frac = min(1.0, target_arcs / max(nnz, 1))
    act = (np.random.default_rng(seed).random(n) < frac).astype(np.uint8)
    t0 = time.perf_counter()
    _, tr1 = oracle.lpa(off, cols, w, max_iter=1, active_in=act)
    _, _, tr2 = oracle.local_move(off, cols, w, max_iter=1, active_in=act)
    dt = time.perf_counter() - t0
    arcs = int(tr1.arcs[0] + tr2.arcs[0])
    desc = (f"oracle (plain C, 1 thread): first LPA round + first Louvain local-move round of the "
            f"same graph, initial active set = seeded uniform {frac:.1%} vertex sample "
            f"({int(act.sum())} vertices, {int(tr1.arcs[0])} arcs per round)")
    return arcs, dt, desc


def host_graph(g):
    import numpy as np
    off = g.off.cpu().numpy().astype(np.int64)
    cols = g.cols.cpu().numpy().astype(np.int32)
    w = None if g.w is None else g.w.cpu().numpy().astype(np.int64)
    return off, cols, w


def run_reference(args, rank, world):
    """The oracle on the host cores, timed on bounded samples of the workload."""
    if rank != 0:
        return
    if args.workload in ("batch4096", "serve2048", "served"):
        run_reference_many(args)
        return
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    g, scale = make_graph(args.workload, args.scale, dev)
    off, cols, w = host_graph(g)
    del g
    samples = []
    for i in range(args.warmup + args.steps):
        arcs, dt, desc = oracle_sample(off, cols, w, args.ref_sample_arcs)
        if i >= args.warmup:
            samples.append((arcs, dt))
    arcs = sum(a for a, _ in samples)
    secs = sum(t for _, t in samples)
    value = arcs / secs / 1e9
    line = {"impl": "reference", "metric": METRIC_GTEPS,
            "value": value, "unit": "GTEPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, len(samples)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": graph_config(args, scale, len(off) - 1, int(off[-1]), world),
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_reference_many(args, budget_s: float = 20.0):
    """The oracle solving the graphs of a many-graph workload one after another
    (in their order, until a time budget per step is spent)."""
    import numpy as np
    import oracle
    if args.workload == "batch4096":
        import synth
        reqs = [(2, *host_graph(synth.sbm(n, k, "0.2", "0.002", seed=sd, wmax=4)))
                for n, k, sd in synth.batch_specs(4096, seed=4)[:64]]
    else:
        reqs = [(k, o, c, None if w is None else w.astype(np.int64))
                for k, o, c, w in serve_requests(args.workload, 11, min(args.serve_requests, 64))]
    per_step = max(1.0, budget_s / max(1, args.steps + args.warmup))
    done, secs, i = 0, 0.0, 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cnt = 0
        while time.perf_counter() - t0 < per_step:
            kind, off, cols, w = reqs[i % len(reqs)]
            i += 1
            if kind == 1:
                oracle.lpa(off, cols, w)
            else:
                oracle.louvain(off, cols, w)
            cnt += 1
        if step >= args.warmup:
            done += cnt
            secs += time.perf_counter() - t0
    unit = "graphs/s" if args.workload == "batch4096" else "requests/s"
    value = done / secs
    sample = f"oracle (plain C, 1 thread) solving the workload's graphs one by one, {done} graphs in {secs:.1f} s"
    line = {"impl": "reference", "metric": METRIC_BATCH if args.workload == "batch4096" else METRIC_SERVE,
            "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": args.workload, "description": WORKLOADS[args.workload]},
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ serving workload

def host_mem_available() -> int:
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


def _host_req(kind, g):
    import numpy as np
    off = g.off.cpu().numpy().astype(np.int64)
    cols = g.cols.cpu().numpy().astype(np.int32)
    w = None if g.w is None else g.w.cpu().numpy().astype(np.int32)
    return (kind, off, cols, w)


def serve_requests(workload: str, seed: int, count: int = 0):
    """A request stream as host arrays: [(kind, off int64, cols int32, w int32|None)], kind 1 = LPA,
    2 = Louvain. serve2048: mostly small graphs (packing); served: the heavy-tailed size mix."""
    import numpy as np
    import torch

    import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    if workload == "served":
        specs = synth.serve_specs(20_000, seed=5)[:count or 512]
        # host memory guard: the stream is held twice (here and in the server's queue)
        avail = host_mem_available()
        need = 0
        for i, sp in enumerate(specs):
            need += 2 * (sp[2] * 16 * 4 + sp[2] * 8)
            if avail and need > avail // 4:
                specs = specs[:i]
                break
        out = []
        for sp in specs:
            out.append(_host_req(2 if sp[0] == "louvain" else 1, synth.serve_graph(sp, dev)))
        return out
    rng = np.random.default_rng(seed)
    small = synth.batch_specs(1984, seed=seed)
    mid_n = np.exp(rng.uniform(np.log(10_000), np.log(30_000), 48)).astype(np.int64)
    mid = [(int(n), int(n) // 100, seed * 1000 + j) for j, n in enumerate(mid_n)]
    graphs = []
    for part in (small, mid):
        if dev == "cuda":
            g, vstart, _ = synth.sbm_batch_device(part)
            graphs += synth.unpack_batch(g.to("cpu"), vstart)
        else:
            graphs += [synth.sbm(n, k, "0.2", "0.002", seed=sd, wmax=4) for n, k, sd in part]
    for j in range(16):
        graphs.append(synth.rmat(14 + j % 4, 16, seed=seed * 100 + j, device=dev).to("cpu"))
    order = rng.permutation(len(graphs))
    kinds = rng.integers(0, 3, len(graphs))
    return [_host_req(1 if kinds[i] == 0 else 2, graphs[o]) for i, o in enumerate(order)]


def run_serve(args, rank, world, local, steps=None, warmup=None, workload=None, requests=None):
    """Requests through the serving engine (continuous batching over worker
    streams) vs the same requests one call at a time: throughput when all
    arrive at once, and latency under Poisson arrivals at 0.8x the measured
    one-at-a-time capacity, for both."""
    import threading

    import numpy as np
    import torch

    import paper_2507_06471_gb300 as cd

    cd.lib()
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    workload = workload or args.workload
    reqs = serve_requests(workload, 11 + 7919 * rank, requests or args.serve_requests)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    R = len(reqs)
    h2d = sum(o.nbytes + c.nbytes + (0 if w is None else w.nbytes) for _, o, c, w in reqs)
    d2h = sum(4 * (len(o) - 1) for _, o, _, _ in reqs)
    arcs = sum(len(c) for _, _, c, _ in reqs)

    def burst(srv):
        t0 = time.perf_counter()
        ids = [srv.submit(k, o, c, w) for k, o, c, w in reqs]
        out = [srv.result(i) for i in ids]
        return time.perf_counter() - t0, out

    def open_loop(srv, rate, seed=5):
        gaps = np.random.default_rng(seed).exponential(1.0 / rate, R)
        ids = []

        def feed():
            t = time.perf_counter()
            for i, (k, o, c, w) in enumerate(reqs):
                t += gaps[i]
                d = t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                ids.append(srv.submit(k, o, c, w))

        th = threading.Thread(target=feed)
        th.start()
        th.join()
        res = [srv.result(i)[1] for i in ids]
        lat = [r.latency_ms for r in res]
        return {"rate_per_s": rate, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(np.max(lat)),
                "queue_p50_ms": float(np.percentile([r.queue_ms for r in res], 50))}

    small_n, batch_arcs = 8192, 1 << 22
    srv = cd.Server(slots=args.serve_slots, small_n=small_n, batch_arcs=batch_arcs)
    seq = cd.Server(slots=1, small_n=0)
    for _ in range(max(1, warmup)):
        burst(srv)
    # one call at a time: capacity and labels
    seq_s, seq_out = burst(seq)
    seq_rps = R / seq_s

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = cd.cd_launch_count()
    secs, lat, packed = [], [], []
    last = None
    for _ in range(steps):
        dt, last = burst(srv)
        secs.append(dt)
        lat += [r.latency_ms for _, r in last]
        packed += [r.batched_with for _, r in last]
    torch.cuda.synchronize()
    barrier(world)
    launches = cd.cd_launch_count() - launches0
    clk = clocks.stop()
    wall = allreduce_max(sum(secs), world)
    value = allreduce_sum(float(R * steps), world) / wall
    stats = srv.stats()
    same = all(np.array_equal(a[0], b[0]) and a[1].iters == b[1].iters for a, b in zip(seq_out, last))

    rate = 0.8 * seq_rps
    ol_srv = open_loop(srv, rate)
    ol_seq = open_loop(seq, rate)
    srv.close()
    seq.close()

    line = {"metric": METRIC_SERVE,
            "value": value, "unit": "requests/s", "n_gpus": world, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * wall / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": workload, "description": WORKLOADS[workload], "requests": R,
                       "arcs": arcs, "slots": args.serve_slots, "small_n": small_n, "batch_arcs": batch_arcs,
                       "parallelism": f"replicas x{world}",
                       "timing": "host wall clock from the first submit to the last result; all requests "
                                 "submitted at once"},
            "latency_ms_all_at_once": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "open_loop": {"arrivals": "Poisson at 0.8x the measured one-at-a-time capacity",
                          "server": ol_srv, "one_at_a_time": ol_seq},
            "mean_batched_with": float(np.mean(packed)), "server_stats": stats,
            "one_at_a_time": {"requests_per_s": seq_rps, "same_labels_and_iters": bool(same),
                              "how": "the same server API with one worker and packing off"},
            "speedup_vs_one_at_a_time": value / seq_rps / world,
            "e2e": {"value": value, "unit": "requests/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "note": "the value itself is end to end: host buffers in, host labels out"},
            "gpu_launches": launches, "clocks": clk}
    return line


# ------------------------------------------------------------------ batched workload

def run_batch(args, rank, world, local, steps=None, warmup=None):
    """Louvain on 4,096 graphs at once (batched mode) vs one call per graph."""
    import numpy as np
    import torch

    import paper_2507_06471_gb300 as cd
    import synth

    cd.lib()
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    specs = synth.batch_specs(4096, seed=4 + 4096 * rank)
    g, vstart, _ = synth.sbm_batch_device(specs)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    B = len(specs)
    lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
    params = cd.cd_params_default()
    stream = torch.cuda.current_stream()

    # autotune the degree bins once on this workload (untimed)
    h = cd.cd_csr_upload(g.off, g.cols, g.w)
    tw, th = cd.cd_autotune(h, cd.cd_params_default(), 3)
    cd.cd_graph_free(h)

    def step(timing=False, device_loop=1):
        params.timing = 1 if timing else 0
        params.device_loop = device_loop
        h = cd.cd_csr_upload(g.off, g.cols, g.w)
        cd.cd_graph_set_bins(h, tw, th)
        cd.cd_graph_set_batches(h, vstart)
        levels, q = cd.cd_batch_louvain_run(h, params, lab, B)
        tr = cd.cd_trace_get(h)
        prof = cd.cd_profile_get(h) if timing else []
        cd.cd_graph_free(h)
        return sum(t["arcs"] for t in tr), len(tr), levels, q, prof

    for _ in range(warmup):
        step()
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = cd.cd_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    arcs = 0
    for _ in range(steps):  # the rounds after the first of each level run as one captured graph
        a, rounds, levels, q, _ = step()
        arcs += a
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = cd.cd_launch_count() - launches0
    clk = clocks.stop()
    ms = allreduce_max(ev0.elapsed_time(ev1), world)
    graphs_per_s = allreduce_sum(float(B * steps), world) / (ms / 1e3)
    # the same steps with one host read-back per round, for comparison
    step(device_loop=0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step(device_loop=0)
    e1.record(stream)
    torch.cuda.synchronize()
    host_loop_gps = B * steps / (e0.elapsed_time(e1) / 1e3)
    # per-kernel shares from one more step with per-kernel events (untimed)
    prof = {}
    merge_profiles(prof, step(timing=True)[4])

    # one call per graph (upload + cd_louvain_run) on an evenly spaced sample
    members = synth.unpack_batch(g, vstart)
    pick = np.linspace(0, B - 1, min(args.solo_sample, B)).astype(int)
    solo_lab = [torch.empty(members[b].n, dtype=torch.int32, device="cuda") for b in pick]
    same = True
    lab_h = lab.cpu().numpy()
    for i, b in enumerate(pick[:8]):  # warm-up of the solo path
        m = members[b]
        h = cd.cd_csr_upload(m.off, m.cols, m.w)
        cd.cd_louvain_run(h, cd.cd_params_default(), solo_lab[i])
        cd.cd_graph_free(h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, b in enumerate(pick):
        m = members[b]
        h = cd.cd_csr_upload(m.off, m.cols, m.w)
        cd.cd_louvain_run(h, cd.cd_params_default(), solo_lab[i])
        cd.cd_graph_free(h)
    torch.cuda.synchronize()
    solo_s = time.perf_counter() - t0
    for i, b in enumerate(pick):
        same = same and bool(np.array_equal(solo_lab[i].cpu().numpy(), lab_h[vstart[b]:vstart[b + 1]]))
    solo_gps = len(pick) / solo_s
    total_prof_ms = sum(v["total_ms"] for v in prof.values())
    kernels = {k: {"launches": v["launches"], "ms": round(v["total_ms"], 3),
                   "share": round(v["total_ms"] / total_prof_ms, 4) if total_prof_ms else 0}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["total_ms"]) if v["launches"]}
    line = {"metric": METRIC_BATCH,
            "value": graphs_per_s, "unit": "graphs/s", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "batch4096", "description": WORKLOADS["batch4096"], "graphs": B,
                       "n": g.n, "arcs": g.nnz, "parallelism": f"replicas x{world}",
                       "bins_autotuned": {"t_warp": tw, "t_hub": th}},
            "gteps": arcs / (ms / 1e3) / 1e9 * world, "louvain_rounds": rounds,
            "max_levels_reached": int(levels.max()), "mean_q": float(np.mean(q)),
            "solo": {"graphs_per_s": solo_gps, "sample": int(len(pick)), "same_labels_as_batched": same,
                     "how": "cd_csr_upload + cd_louvain_run per graph, one graph at a time"},
            "speedup_vs_solo": graphs_per_s / solo_gps,
            "host_loop": {"graphs_per_s": host_loop_gps,
                          "how": "the same calls with device_loop = 0 (one host read-back per round)"},
            "kernels": kernels, "gpu_launches": launches,
            "gpu_launches_note": "host launch calls; each level's rounds after the first are one graph "
                                 "launch whose body kernels run once per round",
            "clocks": clk}
    return line


# ------------------------------------------------------------------ main

def emit(line, args, rank):
    if rank == 0:
        print(json.dumps(line))
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(line, f, indent=1)


def compact_many(line):
    """The parts of a batched or served line carried inside the R-MAT line."""
    keep = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "config", "gteps",
            "louvain_rounds", "mean_q", "solo", "speedup_vs_solo", "latency_ms_all_at_once", "open_loop",
            "mean_batched_with", "one_at_a_time", "speedup_vs_one_at_a_time", "host_loop", "e2e", "gpu_launches",
            "clocks")
    return {k: line[k] for k in keep if k in line}


def run_case(args):
    """Small profiling cases (see --case); no timing line."""
    import torch

    import paper_2507_06471_gb300 as cd
    import synth
    g = synth.rmat(args.scale or 23, 16, seed=3, device="cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    G = cd.Graph(g.off, g.cols, None)
    if args.case == "first-rounds":
        G.lpa(max_iter=2, timing=1)
        alg = {x["name"]: x["alg_bytes"] for x in G.profile() if x["launches"]}
        G.local_move(max_iter=2)
        torch.cuda.synchronize()
        out = {"case": args.case, "scale": args.scale or 23, "n": G.n, "arcs": G.nnz,
               "captured": "LPA round 1", "alg_bytes": alg}
        print(json.dumps(out))
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(out, f)
        return
    lab, _, _ = G.local_move()
    C, _ = G.aggregate(lab)
    torch.cuda.synchronize()
    prof = {}
    for r in (3, 4):
        if r == 4:
            torch.cuda.profiler.start()
        C.local_move(max_iter=r, timing=1)
        torch.cuda.synchronize()
        if r == 4:
            torch.cuda.profiler.stop()
        prof[r] = {x["name"]: x["alg_bytes"] for x in C.profile() if x["launches"]}
    t = C.trace()[3]
    out = {"case": args.case, "scale": args.scale or 23, "n": C.n, "arcs": C.nnz,
           "captured": "coarse-graph round 3",
           "round3": {"active": t["active"], "arcs": t["arcs"], "moved": t["moved"]},
           "alg_bytes": {k: prof[4][k] - prof[3].get(k, 0.0) for k in prof[4]}}
    print(json.dumps(out))
    if args.json_out:
        with open(args.json_out, "w") as f:
            json.dump(out, f)


def main():
    args = parse()
    if args.ncu_summary:
        ncu_summary(*args.ncu_summary)
        return
    rank, world, local = dist_setup()
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch4096":
        emit(run_batch(args, rank, world, local), args, rank)
        return
    if args.workload in ("serve2048", "served"):
        emit(run_serve(args, rank, world, local), args, rank)
        return
    line = run_graph(args, rank, world, local)
    if args.workload == "rmat26" and args.scale is None and not args.no_many:
        # the batched and served parts of the metric, each timed on its own
        ms, wu = args.many_steps, min(args.warmup, 2)
        line["batch4096"] = compact_many(run_batch(args, rank, world, local, steps=ms, warmup=wu))
        line["serve2048"] = compact_many(run_serve(args, rank, world, local, steps=ms, warmup=wu,
                                                   workload="serve2048"))
        line["served"] = compact_many(run_serve(args, rank, world, local, steps=1, warmup=1, workload="served",
                                                requests=args.served_in_line))
    emit(line, args, rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_graph(args, rank, world, local):
    """One graph: upload + LPA + Louvain per step (the headline GTEPS line)."""
    import numpy as np
    import torch

    import paper_2507_06471_gb300 as cd

    assert torch.cuda.is_available(), "the benchmark needs a CUDA GPU"
    cd.lib()
    g, scale = make_graph(args.workload, args.scale, "cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # hand the generator's scratch back before the library allocates
    n, nnz = g.n, g.nnz
    wbytes = 0 if g.w is None else 4
    labels_lpa = torch.empty(n, dtype=torch.int32, device="cuda")
    labels_lv = torch.empty(n, dtype=torch.int32, device="cuda")
    params = cd.cd_params_default(asynchronous=int(args.asynchronous))
    assert {k: getattr(params, k) for k in RUN_PARAMS} == RUN_PARAMS
    stream = torch.cuda.current_stream()

    # warm-up (untimed)
    for _ in range(args.warmup):
        run_step(cd, g, params, labels_lpa, labels_lv)
    torch.cuda.synchronize()

    # timed region: device-resident inputs, per-round CUDA events (the degree
    # bins' scan kernels run concurrently on auxiliary streams)
    params.timing = 2
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = cd.cd_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    total_arcs = 0
    infos = []
    prof = {}
    traces = []
    for _ in range(args.steps):
        arcs, info, _, tr = run_step(cd, g, params, labels_lpa, labels_lv)
        total_arcs += arcs
        infos.append(info)
        traces.append(tr)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = cd.cd_launch_count() - launches0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = allreduce_max(ms, world)
    value = job_rate(total_arcs, ms / 1e3, world) / 1e9

    # end to end through the C ABI with host buffers (pinned)
    off_h = g.off.cpu().pin_memory()
    cols_h = g.cols.cpu().pin_memory()
    w_h = None if g.w is None else g.w.cpu().pin_memory()
    lab_h1 = torch.empty(n, dtype=torch.int32).pin_memory()
    lab_h2 = torch.empty(n, dtype=torch.int32).pin_memory()
    params_e2e = cd.cd_params_default(asynchronous=int(args.asynchronous))
    e2e_value, e2e_s = None, 0.0
    if args.e2e_steps > 0:
        run_step(cd, None, params_e2e, lab_h1, lab_h2, host=True, g_host=(off_h, cols_h, w_h))
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_arcs = 0
        for _ in range(args.e2e_steps):
            a, _, _, _ = run_step(cd, None, params_e2e, lab_h1, lab_h2, host=True, g_host=(off_h, cols_h, w_h))
            e2e_arcs += a
        torch.cuda.synchronize()
        e2e_s = allreduce_max(time.perf_counter() - t0, world)
        e2e_value = allreduce_sum(float(e2e_arcs), world) / e2e_s / 1e9
    h2d = off_h.numel() * 8 + cols_h.numel() * 4 + (0 if w_h is None else w_h.numel() * 4)
    d2h = 2 * n * 4

    # per-kernel events: one more step with timing = 1, where each kernel runs
    # alone (the bins' kernels one after another), so its events bracket it
    params.timing = 1
    _, _, p, _ = run_step(cd, g, params, labels_lpa, labels_lv)
    merge_profiles(prof, p)
    params.timing = 0

    # roofline of the dominant kernel (by device time in the profiled step)
    peak, peak_kind = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1]["total_ms"])
    dname, d = dom
    achieved = (d["alg_bytes"] / d["launches"]) / (d["total_ms"] / d["launches"] / 1e3) / 1e9
    traffic, traffic_src = ncu_traffic(dname, d["alg_bytes"] / d["launches"])
    total_prof_ms = sum(v["total_ms"] for v in prof.values())
    kernels = {k: {"launches": v["launches"], "ms": round(v["total_ms"], 3),
                   "share": round(v["total_ms"] / total_prof_ms, 4) if total_prof_ms else 0,
                   "GBps": round(v["alg_bytes"] / (v["total_ms"] / 1e3) / 1e9, 1) if v["total_ms"] else 0}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["total_ms"]) if v["launches"]}

    # the method's per-round figures: the first LPA round and the first
    # local-moving round of level 0 (every vertex examined), median over steps
    rounds = {"bytes": "per round: arcs x (column 4 + neighbour label 4 + weight) + examined vertices x 17 "
                       "(offsets, label, label write, flag) + 4 x arcs of moved vertices + n flag clears; "
                       "Louvain adds 8 per candidate pair, 8 per examined vertex, 24 per move",
              "time": "CUDA events on the library stream from the round's first to its last kernel "
                      "(scan_ms: up to the end of the scan kernels)",
              "round0": "every vertex starts alone, so round 0 decides from the rows (labels are the vertex "
                        "ids: no label gathers, no hub tables); round 1 is the first round that reads labels "
                        "and builds the hub tables",
              "peak": peak}
    for k in (0, 1):
        lpa_k = [tr[0][k] for tr in traces if len(tr[0]) > k]
        lv_k = [[t for t in tr[1] if t["level"] == 0][k] for tr in traces
                if sum(1 for t in tr[1] if t["level"] == 0) > k]
        if lpa_k:
            rounds[f"lpa_round{k}"] = round_figures(lpa_k, False, wbytes, n, peak)
        if lv_k:
            rounds[f"louvain_level0_round{k}"] = round_figures(lv_k, True, wbytes, n, peak)
    # every round of the last step: arcs scanned over round time, and bytes over round time
    last_lpa, last_lv = traces[-1]
    for name, rows, louv in (("lpa_all_rounds", last_lpa, False), ("louvain_all_rounds", last_lv, True)):
        ms_all = sum(t["round_ms"] for t in rows)
        if ms_all > 0:
            b_all = sum(round_bytes(t, louv, wbytes, n if louv is False or t["level"] == 0 else 0) for t in rows)
            rounds[name] = {"rounds": len(rows), "ms": ms_all, "arcs": sum(t["arcs"] for t in rows),
                            "gteps": sum(t["arcs"] for t in rows) / (ms_all / 1e3) / 1e9,
                            "GBps": b_all / (ms_all / 1e3) / 1e9, "frac": b_all / (ms_all / 1e3) / 1e9 / peak}

    line = {
        "metric": METRIC_GTEPS,
        "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": graph_config(args, scale, n, nnz, world),
        "time_to_converge_ms": {"lpa_plus_louvain_step": ms_max / args.steps},
        "step": infos[-1],
        "rounds": rounds,
        "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": args.e2e_steps, "ms_per_step": 1e3 * e2e_s / max(1, args.e2e_steps)},
        "roofline": {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_scaled_from": traffic_src,
                     "bytes": KERNEL_BYTES.get(dname, "library-counted algorithmic bytes of the kernel"),
                     "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
        "kernels": kernels,
        "kernels_how": "one step after the timed region with per-kernel CUDA events on each kernel's stream "
                       "(timing = 1: the degree bins' kernels run one after another there, concurrently in "
                       "the timed steps); ms over that step",
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        off, cols = off_h.numpy(), cols_h.numpy()
        w = None if w_h is None else w_h.numpy().astype(np.int64)
        arcs, dt, desc = oracle_sample(off, cols, w, args.cpu_sample_arcs)
        line["cpu_baseline"] = {"value": arcs / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                                "sample": desc, "seconds": dt}
    del g, off_h, cols_h, w_h, lab_h1, lab_h2, labels_lpa, labels_lv
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return line


if __name__ == "__main__":
    main()
