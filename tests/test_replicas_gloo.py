"""The multi-process path of bench.py on the CPU: two ranks over gloo, launched
the way torchrun launches them (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_* in the
environment).  The method's single-GPU path has no data-parallel split, so N
ranks are independent replicas: the host logic under test is the process-group
set-up, the slowest-rank timer and the whole-job rate, and the reference arm,
which only rank 0 runs."""
import json
import os
import socket
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import bench
rank, world, local, dist = bench.dist_setup(2)
assert dist is not None and dist.get_backend() == "gloo"
ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
dist.barrier()
print(json.dumps({"rank": rank, "world": world, "local": local, "ms": ms,
                  "rate": bench.whole_job_rate(20, world, ms)}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2 and o["local"] == o["rank"]
        assert o["ms"] == 15.0                         # the slower rank's 15 ms on both
        assert o["rate"] == pytest.approx(20 * 2 / 0.015)  # both ranks' units over that time


def test_single_process_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.whole_job_rate(20, 1, 250.0) == pytest.approx(80.0)


def test_reference_arm_runs_on_rank_zero_only():
    import bench

    args = types.SimpleNamespace(steps=1, warmup=3)
    assert bench.run_reference(args, rank=1, world=2) == 0  # returns at once, without the oracle
