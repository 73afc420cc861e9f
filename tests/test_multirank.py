"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2).

The solver does not shard a grid: for one problem, N GPUs run N independent
replicas (weak scaling, no data-path collective); a batch of independent
problems is split over the ranks by size. What the N-rank run adds is host
logic: the job's time is the maximum over ranks, the value counts every
rank's solves, the problem split covers every problem once and balances the
bytes, and in the reference arm only rank 0 works and prints. These run here
as two processes on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world, _ = bench.dist_env()
ms = bench.job_ms(5.0 + 2.0 * rank, world)
print(json.dumps({"rank": rank, "ms": ms, "value": bench.job_value(world, ms)}))
dist.barrier()
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch(code, world, extra_env=None, args=()):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), BENCH_ROOT=ROOT)
        env.update(extra_env or {})
        cmd = [sys.executable, "-c", code, *args] if code else [sys.executable, os.path.join(ROOT, "bench.py"), *args]
        procs.append(subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      cwd=ROOT))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_job_time_is_the_max_over_ranks_and_value_counts_every_rank():
    pytest.importorskip("torch")
    outs = launch(CHILD, 2)
    recs = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in recs:
        assert r["ms"] == 7.0  # rank 1's 7 ms, the slower replica
        assert r["value"] == pytest.approx(2 * 1e3 / 7.0)


def test_reference_arm_works_on_rank_zero_only():
    # a rank other than 0 of the reference arm exits 0 without output or work
    outs = launch(None, 1, extra_env={"RANK": "1", "WORLD_SIZE": "2"}, args=("--impl", "reference"))
    assert outs[0].strip() == ""


def test_problem_partition_is_exact_and_balanced():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    ms_ = synth.batch_levels(4096, 0x5EED0004)
    w = [float(4 ** int(m)) for m in ms_]
    for world in (1, 2, 3, 8):
        parts = bench.partition(w, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(w)))  # every problem exactly once
        loads = [sum(w[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(w)  # greedy bound: within one problem
        assert parts == bench.partition(w, world)  # deterministic


CHILD_PARTS = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world, _ = bench.dist_env()
w = [float(4 ** (5 + (i * 7) % 6)) for i in range(100)]
mine = bench.partition(w, world)[rank]
# each rank "solves" its share in a time proportional to its bytes
ms = bench.job_ms(sum(w[i] for i in mine) / 1e3, world)
print(json.dumps({"rank": rank, "mine": mine, "ms": ms}))
dist.barrier()
dist.destroy_process_group()
"""


def test_two_ranks_split_problems_without_overlap():
    pytest.importorskip("torch")
    recs = [json.loads(o.strip().splitlines()[-1]) for o in launch(CHILD_PARTS, 2)]
    a, b = recs[0]["mine"], recs[1]["mine"]
    assert not set(a) & set(b) and sorted(a + b) == list(range(100))
    assert recs[0]["ms"] == recs[1]["ms"]  # both report the slower rank's time
