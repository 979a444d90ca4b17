"""The benchmark's multi-rank plumbing on CPU: two gloo ranks (world size 2).

bench.py runs one replica per GPU under torchrun and reports the whole job:
the maximum of the ranks' timed seconds, and the bytes of all ranks over it.
Here two CPU processes exercise the same helpers (max over ranks, barrier,
aggregate) and the reference arm's rule that only rank 0 works and prints.
"""
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT

WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, _, world = bench.dist_env()
dist.init_process_group("gloo", init_method="env://")
assert dist.get_world_size() == world == 2
secs = [1.5, 2.5][rank]
bench.barrier()
m = bench.max_over_ranks(secs)
assert m == 2.5, m
value = bench.aggregate(8e9, m, world)
assert abs(value - 8e9 * 2 / 2.5 / 1e9) < 1e-9, value
bench.barrier()
print(json.dumps({"rank": rank, "max": m, "value": value}), flush=True)
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(script: str, extra_env: dict, args=()):
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), **extra_env)
        procs.append(subprocess.Popen([sys.executable, "-c", script, ROOT, *args], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        outs.append((p.returncode, out, err))
    return outs


def test_two_gloo_ranks_max_and_aggregate():
    outs = _launch(WORKER, {})
    for rc, out, err in outs:
        assert rc == 0, err
    lines = [o[1].strip() for o in outs]
    assert all('"max": 2.5' in line for line in lines), lines


REFERENCE = r"""
import sys
sys.path.insert(0, sys.argv[1])
import bench
sys.exit(bench.main(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]))
"""


def test_reference_arm_rank0_only():
    """Under two ranks the reference arm runs on rank 0 alone; rank 1 exits 0
    without output."""
    pytest.importorskip("numpy")
    outs = _launch(REFERENCE, {})
    (rc0, out0, err0), (rc1, out1, err1) = outs
    assert rc0 == 0, err0
    assert rc1 == 0, err1
    assert '"impl": "reference"' in out0
    assert out1.strip() == ""
