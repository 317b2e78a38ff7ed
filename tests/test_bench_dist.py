"""Multi-rank host logic of bench.py on CPU: two gloo ranks on 127.0.0.1 agree on
the max-over-ranks time and pass the barriers (each rank runs its own replica, so
no collective touches the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench._barrier(world)
    got = bench._max_over_ranks(10.0 + rank * 5.0, world)
    bench._barrier(world)
    out[rank] = got
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_single_rank_is_identity():
    import bench
    assert bench._max_over_ranks(3.5, 1) == 3.5
    bench._barrier(1)


@pytest.mark.gpu
def test_bench_two_ranks_sharing_the_gpu():
    """bench.py launched as the driver launches it for N > 1 (torchrun, one process per
    rank), here two ranks on one GPU with the exchange staged through host memory
    (gloo): rank 0 prints one JSON line for both ranks, with the replicas' value, the
    tile-sharded system's and the cluster-sharded batch's."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SD_BENCH_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--gpus", "2", "--steps", "3", "--warmup",
           "3", "--quick"]
    r = subprocess.run(cmd, cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    lines = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["n_gpus"] == 2 and line["value"] > 0 and line["config"]["parallelism"] == "replicas"
    ts = line["tile_sharded"]
    assert ts["ranks"] == 2 and ts["value"] > 0 and ts["scaling"] == "strong"
    bs = line["batched_sharded"]
    assert bs["ranks"] == 2 and bs["steps_per_s"] > 0 and 0 < bs["clusters_this_rank_0"] < 16384
