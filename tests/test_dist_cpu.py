"""The multi-process side of bench.py on CPU (gloo, world size 2): the path is
replicas only, so ranks exchange nothing but the timing reduction: the
whole-job value is the units of all ranks over the slowest rank's time; the
reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
rank, world, local = bench.dist_setup()
units = [3.0e9, 5.0e9][rank]
secs = [2.0, 4.0][rank]
out = {{"rank": rank, "world": world,
       "max": bench.allreduce_max(secs, world), "sum": bench.allreduce_sum(units, world),
       "rate": bench.job_rate(units, secs, world)}}
bench.barrier(world)

class A: pass
a = A(); a.workload = "sbm10k"; a.scale = None; a.steps = 1; a.warmup = 0; a.gpus = world
a.cpu_sample_arcs = 1e4; a.serve_requests = 4
if rank != 0:
    bench.run_reference(a, rank, world)   # returns at once on every rank but 0
print("RESULT " + json.dumps(out), flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_like_the_bench():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    results = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        line = [ln for ln in out.splitlines() if ln.startswith("RESULT ")]
        assert line, out + err
        results.append(json.loads(line[0][7:]))
    for r in results:
        assert r["world"] == 2
        assert r["max"] == 4.0
        assert r["sum"] == 8.0e9
        assert r["rate"] == 8.0e9 / 4.0   # all ranks' units over the slowest rank's time
    assert sorted(r["rank"] for r in results) == [0, 1]


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.allreduce_max(2.5, 1) == 2.5
    assert bench.allreduce_sum(7.0, 1) == 7.0
    assert bench.job_rate(10.0, 4.0, 1) == 2.5
