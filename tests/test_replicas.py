"""The benchmark's multi-GPU form is "replicas only": one independent copy of
the workload per rank, no data-path collective, a barrier around the timed
region and the job's time taken as the slowest rank's.  This tests that host
logic with two gloo ranks on the CPU: the max-over-ranks reduction, the
whole-job value, and the reference arm's rank > 0 exit without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
rank, world, _ = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one
mx = bench.max_over_ranks(ms, world, "cpu")
dist.barrier()
print(json.dumps({"rank": rank, "max": mx, "value": bench.replicas_value(1000.0, mx, world)}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(code, world, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_max_over_ranks_and_job_value_with_two_gloo_ranks():
    pytest.importorskip("torch")
    import json
    outs = _launch(WORKER, 2)
    rows = [json.loads([l for l in o.splitlines() if l.startswith("{")][-1]) for o in outs]
    for r in rows:
        assert r["max"] == 15.0
        # two replicas of 1000 units per step, 15 ms per step: 2000 / 0.015
        assert abs(r["value"] - 2000.0 / 0.015) < 1e-6


def test_reference_arm_other_ranks_exit_without_work():
    code = r"""
import os, sys
sys.path.insert(0, os.environ["ROOT"])
import bench
class A: steps = 1; warmup = 3
sys.exit(bench.run_reference(A()))
"""
    env = dict(os.environ, ROOT=ROOT, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_oracle_on_all_host_cores():
    """The CPU baseline's all-cores figure: one spawned replica of the sample
    per usable core, aggregate rate over the slowest replica, the CPU model
    named."""
    code = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import bench
print(json.dumps(bench.cpu_oracle_all_cores(steps=1, nel=3)))
"""
    env = dict(os.environ, ROOT=ROOT)
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    import json
    r = json.loads(p.stdout.strip().splitlines()[-1])
    assert r["cores"] == len(os.sched_getaffinity(0))
    assert r["value"] > 0 and r["kind"] == "oracle" and r["cpu_model"]
    assert f"{r['cores']} independent replicas" in r["sample"]
