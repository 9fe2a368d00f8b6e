"""Host logic of the multi-rank benchmark path on CPU ranks (gloo, world size 2):
each rank times its own replica, the job takes the slowest rank, and the whole-job
value counts every rank's grid-point steps.  The reference arm runs on rank 0
only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, %(root)r)
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%(port)d", rank=rank, world_size=world)
local_ms = [120.0, 150.0][rank]
t = bench.max_over_ranks(local_ms, world)
v = bench.job_value(257 * 768, 10, world, t)
print(json.dumps({"rank": rank, "t": t, "v": v}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def test_max_over_ranks_and_job_value_on_two_gloo_ranks():
    pytest.importorskip("torch")
    port = _free_port()
    code = WORKER % {"root": ROOT, "port": port}
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["t"] == 150.0
        assert abs(o["v"] - 2 * 257 * 768 * 10 / 0.150 / 1e6) < 1e-9


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "int_n33_p96", "--steps", "2", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
    env0 = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r0 = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                         "int_n33_p96", "--steps", "2", "--warmup", "1"], env=env0, capture_output=True, text=True,
                        timeout=300)
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
