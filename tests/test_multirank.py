"""The multi-rank (torchrun) path of bench.py on CPU: two ranks over gloo.

Under torchrun every rank reduces a matrix of its own (the path shards into
independent problems, so there is no data-path collective), the timed region
is bracketed by barriers and the job's time is the largest over the ranks.
These tests run the host side of that with world_size 2 on the gloo backend:
the environment parsing, the max-over-ranks reduction, the per-rank
workloads, and the reference arm's rank filter.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys
import torch.distributed as dist
sys.path.insert(0, sys.argv[1])
import bench
world, rank, local = bench.dist_env()
dist.init_process_group("gloo")
dist.barrier()
mx = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
spec = bench.rank_workload("fl_2000x3000", 1.0, rank)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"world": world, "rank": rank, "local": local, "max": mx, "seed": spec.seed,
                  "m": spec.m, "n": spec.n, "p": spec.p}))
"""


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_over_gloo():
    pytest.importorskip("torch.distributed")
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for pr in procs:
        out, err = pr.communicate(timeout=240)
        assert pr.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in outs] == [0, 1] and all(d["world"] == 2 for d in outs)
    assert [d["local"] for d in outs] == [0, 1]
    assert all(d["max"] == 15.0 for d in outs)                      # the slowest rank's time
    assert outs[0]["seed"] != outs[1]["seed"]                        # independent matrices
    assert (outs[0]["m"], outs[0]["n"], outs[0]["p"]) == (outs[1]["m"], outs[1]["n"], outs[1]["p"])


def test_max_over_ranks_without_a_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    a = bench.args_parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(a, 2, 1) is None
    assert capsys.readouterr().out == ""
