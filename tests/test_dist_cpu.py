"""Multi-process paths of bench.py on the CPU (gloo, world size 2).

A single solve does not shard, so N GPUs run N independent replicas; the
only cross-rank step is the timing reduction (slowest rank's time, sum of
the ranks' units).  The reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
dist.init_process_group("gloo")
sec, units = bench.reduce_timing(1.0 + rank, 10 * (rank + 1), dist, "cpu")
dist.barrier()
if rank == 0:
    print(json.dumps({"sec": sec, "units": units}))
dist.destroy_process_group()
"""


def test_reduce_timing_two_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    got = json.loads(outs[0][0].strip().splitlines()[-1])
    assert got == {"sec": 2.0, "units": 30.0}  # max time, summed work
    assert outs[1][0].strip() == ""  # only rank 0 reports


def test_reduce_timing_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_timing(1.5, 7, None, "cpu") == (1.5, 7)


def test_reference_arm_other_ranks_exit_without_work():
    sys.path.insert(0, ROOT)
    import bench
    args = type("A", (), {"n": 64, "warmup": 0, "steps": 1, "gpus": 2})()
    assert bench.run_reference(args, rank=1) == 0
