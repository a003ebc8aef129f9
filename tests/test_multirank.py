"""The multi-process path of bench.py on CPU: two ranks over gloo (the GPU
run uses NCCL the same way). Each rank runs an independent replica; the
whole-job figures are the slowest rank's time and the sum of the ranks'
pairs. The reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
sys.path.insert(0, os.environ["REPO"])
import torch.distributed as dist
rank = int(sys.argv[1])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + os.environ["PORT"], rank=rank, world_size=2)
import bench
ms, pairs = bench.over_ranks(10.0 + 2.5 * rank, 100.0 * (rank + 1), dist, "cpu")
dist.barrier()
print(ms, pairs)
dist.destroy_process_group()
"""


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_over_ranks_takes_slowest_time_and_all_pairs():
    env = dict(os.environ, REPO=ROOT, PORT=str(_port()))
    procs = [subprocess.Popen([sys.executable, "-c", CHILD, str(r)], env=env, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out.split())
    for o in outs:
        assert float(o[0]) == 12.5 and float(o[1]) == 300.0


def test_over_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(3.0, 7.0, None, "cpu") == (3.0, 7.0)


def test_reference_arm_prints_only_on_rank_zero(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse([])
    bench.run_reference(args, 1)
    assert capsys.readouterr().out == ""
