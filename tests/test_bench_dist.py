"""The multi-GPU path of bench.py is replicas only: every rank runs the same
workload on its own GPU with no data-path collective, and rank 0 reports the
whole-job throughput at the slowest rank's time.  These CPU tests run the
aggregation with two gloo ranks."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


_WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="env://")
ms = [2.0, 3.5][rank]                 # rank 1 is the slow replica
bench.barrier(world)
slow = bench.max_over_ranks(ms, world)
value = bench.replica_throughput(1e9, slow, world)
print(json.dumps({{"rank": rank, "slow": slow, "value": value}}))
dist.destroy_process_group()
"""


def test_replicas_report_slowest_rank_time():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    import json
    res = [json.loads(o[0].strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["slow"] == 3.5
        assert abs(r["value"] - 2 * 1e9 / 3.5e-3) < 1e-3 * r["value"]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
