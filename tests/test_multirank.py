"""Multi-rank path of bench.py on CPU (gloo, world size 2): each rank maps its own replica
(distinct scene seed), the job time is the slowest rank's (all-reduce MAX), and the job
throughput sums all ranks' points over that time.  The data path has no collective."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.workload("loop64", rank)
    local_ms = 10.0 * (rank + 1)             # rank 1 is the slower one
    slowest = bench.rank_max(local_ms, dist, "cpu")
    value = bench.job_throughput(131072, 4, world, slowest)
    out[rank] = (w.seed, slowest, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    seeds = {res[r][0] for r in range(world)}
    assert len(seeds) == world                       # one replica (scene) per rank
    for r in range(world):
        assert res[r][1] == pytest.approx(20.0)      # every rank sees the slowest time
        assert res[r][2] == pytest.approx(world * 4 * 131072 / 20e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(100, 2, 1, 1.0) == pytest.approx(2e5)


def test_bench_spawns_its_own_ranks_when_asked_for_two_gpus():
    """`bench.py --gpus 2` with no launcher around it starts two local ranks itself (here in its
    CPU-only --dry form over gloo) and prints one line, from rank 0, with n_gpus = 2 and one
    replica seed per rank."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--dry", "--workload",
                        "line16"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = lines[0]
    assert line["n_gpus"] == 2 and line["dry"] is True and line["value"] is None
    assert len(set(line["config"]["replica_seeds"])) == 2
