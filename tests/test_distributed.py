"""Row sharding of one system over ranks (paper_1205_6333_gb300.distributed): the
partition and the all-gather logic on CPU with gloo ranks (a stand-in system whose
rows are computed by the FP64 oracle), and the shard calls of the library on one GPU
as logical shards, bit-identical to the unsharded result."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1205_6333_gb300 import inputs
from paper_1205_6333_gb300.distributed import shard_rows


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class _OracleRows:
    """Stand-in for a System on a CPU rank: the same row-shard interface, rows computed
    by the oracle (forces F_ext + gravity)."""

    def __init__(self, x, fext, g):
        self.n = x.shape[0]
        self.x = np.array(x, dtype=np.float64)
        self.F = fext + g

    def mobility_apply_rows(self, F, r0, r1):
        import torch
        rows = np.arange(r0, r1, dtype=np.int32)
        return torch.from_numpy(oracle.mobility_rows(self.x, F.numpy(), rows))

    def step_rows(self, dt, r0, r1):
        rows = np.arange(r0, r1, dtype=np.int32)
        v = oracle.mobility_rows(self.x, self.F, rows)
        self.x[r0:r1] = self.x[r0:r1] + dt * v

    def get_positions(self, out):
        out.copy_(__import__("torch").from_numpy(self.x))
        return out

    def set_positions(self, x):
        self.x = x.numpy().copy()


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_1205_6333_gb300.distributed import sharded_apply, sharded_steps
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 700
    x0, _ = inputs.cube_rsa(n, 0.05, 901)
    fe = inputs.normal_forces(n, 902)
    g = np.array([0.0, 0.0, -1.0])
    sysr = _OracleRows(x0, fe, g)
    V = sharded_apply(sysr, torch.from_numpy(fe), rank, world)
    xT = sharded_steps(sysr, 0.05, 4, rank, world, x=torch.empty((n, 3), dtype=torch.float64))
    out[rank] = (V.numpy().tobytes(), xT.numpy().tobytes())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_apply_and_steps_gloo(world):
    """Each rank computes only its rows; after the all-gathers every rank holds the
    whole result, equal bit for bit to the unsharded oracle computation."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    n = 700
    x0, _ = inputs.cube_rsa(n, 0.05, 901)
    fe = inputs.normal_forces(n, 902)
    g = np.array([0.0, 0.0, -1.0])
    Vref = oracle.mobility_apply(x0, fe)
    xref = oracle.euler(x0, 4, 0.05, fe, g)
    for r in range(world):
        V = np.frombuffer(out[r][0]).reshape(n, 3)
        xT = np.frombuffer(out[r][1]).reshape(n, 3)
        np.testing.assert_array_equal(V, Vref)
        np.testing.assert_array_equal(xT, xref)


def test_shard_rows_partition():
    for n in [1, 255, 256, 257, 5000, 65536]:
        for world in [1, 2, 3, 8]:
            ranges = [shard_rows(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a0, b0), (a1, b1) in zip(ranges, ranges[1:]):
                assert b0 == a1 and a0 <= b0
            assert all(a % 256 == 0 for a, _ in ranges)


# ---------------------------------------------------------------- logical shards on one GPU

@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_logical_shards_apply_bitwise(prec):
    import paper_1205_6333_gb300 as sd
    n = 5000
    x, _ = inputs.cube_rsa(n, 0.05, 910)
    F = inputs.normal_forces(n, 911)
    with sd.System(n, prec=prec, dense="directed") as s:
        s.set_positions(x)
        full = s.mobility_apply(F)
        for cuts in ([0, 2560, 5000], [0, 1234, 3001, 5000], [0, 256, 512, 768, 5000], [0, 4999, 5000]):
            parts = [s.mobility_apply_rows(F, a, b) for a, b in zip(cuts, cuts[1:])]
            np.testing.assert_array_equal(np.concatenate(parts), full)


@pytest.mark.gpu
def test_logical_shards_steps_bitwise():
    """Three logical ranks (three handles on one GPU) advancing their rows and exchanging
    positions each step, against the unsharded graph-replayed steps."""
    import paper_1205_6333_gb300 as sd
    n, world, steps, dt = 3000, 3, 5, 0.02
    x0, _ = inputs.cube_rsa(n, 0.10, 920)
    fe = inputs.normal_forces(n, 921)
    kw = dict(gravity=(0.0, 0.0, -1.0), rep_eps=1.0, rep_rc=2.5, dense="directed")
    with sd.System(n, **kw) as ref:
        ref.set_positions(x0)
        ref.set_forces(fe)
        ref.step(dt, steps)
        xref = ref.get_positions()
    ranks = [sd.System(n, **kw) for _ in range(world)]
    try:
        for s in ranks:
            s.set_positions(x0)
            s.set_forces(fe)
        x = x0.copy()
        for _ in range(steps):
            for r, s in enumerate(ranks):
                a, b = shard_rows(n, r, world)
                s.step_rows(dt, a, b)
                x[a:b] = s.get_positions()[a:b]
            for s in ranks:
                s.set_positions(x)
        np.testing.assert_array_equal(x, xref)
    finally:
        for s in ranks:
            s.close()


@pytest.mark.gpu
def test_row_shards_need_the_directed_kernel():
    import paper_1205_6333_gb300 as sd
    n = 8192
    x, _ = inputs.cube_rsa(n, 0.05, 930)
    with sd.System(n) as s:
        assert s.dense_kernel() == "symmetric"
        s.set_positions(x)
        with pytest.raises(sd.SDError) as ei:
            s.mobility_apply_rows(inputs.normal_forces(n, 931), 0, 100)
        assert ei.value.status_name == "SD_ERR_UNSUPPORTED"
        full = s.mobility_apply_rows(inputs.normal_forces(n, 931), 0, n)   # all rows: allowed
        assert full.shape == (n, 3)
    with sd.System(64, lubrication=True, dense="directed") as s:
        s.set_positions(x[:64])
        with pytest.raises(sd.SDError) as ei:
            s.step_rows(0.01, 0, 32)
        assert ei.value.status_name == "SD_ERR_UNSUPPORTED"
