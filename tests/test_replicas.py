"""Host logic of the multi-GPU path, on the CPU: the LPT split of a batch of
independent equations, and the world-size-2 exchange of a replicated or split run
(the slowest rank's time by a MAX reduction, every rank's share of a split batch) as
a gloo process group of two processes."""
import json
import os
import socket
import subprocess
import sys
import textwrap

import pytest

from paper_1905_10574_gb300 import inputs, replicas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_lpt_split_covers_and_balances():
    shapes = inputs.batch_shapes(4096, 16, 512, seed=1234)
    costs = [m * n * (m + n) for m, n in shapes]
    for ws in (1, 2, 3, 8):
        shards = replicas.lpt_shards(costs, ws)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))  # every equation exactly once
        loads = [sum(costs[i] for i in s) for s in shards]
        # Graham's bound for longest-processing-time-first: within 4/3 of the optimum,
        # whose makespan is at least max(total / ws, largest unit)
        lower = max(sum(costs) / ws, max(costs))
        assert max(loads) <= 4.0 / 3.0 * lower
        assert shards == replicas.lpt_shards(costs, ws)  # every rank computes the same split


def test_lpt_split_small_cases():
    assert replicas.lpt_shards([], 2) == [[], []]
    assert replicas.lpt_shards([5.0], 3) == [[0], [], []]
    assert replicas.lpt_shards([3, 3, 2, 2, 2], 2) == [[0, 2, 4], [1, 3]]
    with pytest.raises(ValueError):
        replicas.lpt_shards([1.0], 0)


def test_whole_job_rate_is_weak_scaling():
    assert replicas.whole_job_rate(10.0, 4, 2.0) == 20.0
    assert replicas.max_over_ranks(3.25) == 3.25  # no process group: the rank's own value


WORKER = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, os.environ["REPO_ROOT"])
    import torch
    import torch.distributed as dist
    from paper_1905_10574_gb300 import inputs, replicas
    rank, ws = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        slowest = replicas.max_over_ranks(1.5 + rank)
        shapes = inputs.batch_shapes(64, 16, 512, seed=7)
        costs = [m * n * (m + n) for m, n in shapes]
        shard = replicas.lpt_shards(costs, ws)[rank]
        t = torch.tensor([float(sum(costs[i] for i in shard)), float(len(shard))], dtype=torch.float64)
        dist.all_reduce(t)
        print(json.dumps({"rank": rank, "slowest": slowest, "sum": t.tolist(), "shard": shard,
                          "total": float(sum(costs)), "count": len(costs)}))
    finally:
        dist.destroy_process_group()
""")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_gloo_exchange(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), REPO_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=180)
        finally:
            if p.poll() is None:
                p.kill()
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["slowest"] == 2.5  # the MAX over ranks reaches every rank
        assert o["sum"] == [o["total"], float(o["count"])]  # the shards add up to the whole batch
    assert not set(outs[0]["shard"]) & set(outs[1]["shard"])
