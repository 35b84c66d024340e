"""The multi-GPU form of the benchmark is independent replicas: every rank
fits its own seeded input and the job's throughput is all ranks' fits over
the slowest rank's time (a MAX all-reduce of the timings, no data-path
collective). This runs that host logic as two gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
from hamls_synth import workload
rank, world = dist.get_rank(), dist.get_world_size()
local_s = [2.0, 3.0][rank]
v = bench.aggregate_fits_per_s(10, local_s, world, dist, "cpu")
m = bench.max_over_ranks(float(rank + 1), dist, "cpu")
w = workload("s2_n16_k2_m5k", fit_index=rank)
print(json.dumps({"rank": rank, "value": v, "max": m, "probe": float(w.values[:16].sum())}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_rank():
    port = str(_free_port())
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=port, RANK=str(rank), WORLD_SIZE="2",
                   REPO_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    out = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e[-2000:]
        out.append(json.loads(o.strip().splitlines()[-1]))
    out.sort(key=lambda d: d["rank"])
    for d in out:
        assert abs(d["value"] - 2 * 10 / 3.0) < 1e-12      # 20 fits when the slower rank ends at 3 s
        assert d["max"] == 2.0
    assert out[0]["probe"] != out[1]["probe"]               # each replica fits its own seeded input


def test_one_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5, None, "cpu") == 1.5
    assert bench.aggregate_fits_per_s(10, 2.0, 1, None, "cpu") == 5.0
