"""One system split over ranks (paper_1205_6333_gb300.distributed).

Tile shards (the all-pairs sum divided by pairs, either kernel, every precision):
  * gloo ranks on CPU drive the partition / all-gather / combine logic with a
    stand-in system whose shares are computed from the oracle's mobility matrix;
  * on one GPU, logical shards through the library's part/combine calls against the
    FP64 oracle element by element, for the apply and for Euler steps;
  * two processes sharing one GPU run the real kernels and exchange their shares
    over gloo (host staging), as distributed.tile_sharded_steps does between GPUs.
Row shards (directed kernel): the same on CPU, and bit-identical logical shards.
Cluster shards (batched workloads): the work-balanced partition, gloo ranks that
gather their clusters' results, and logical shards on one GPU equal to the whole
batch bit for bit."""
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


class _OracleTiles:
    """Stand-in for a System on a CPU rank with the tile-shard interface: shard s of G
    owns the source columns [s n / G, (s + 1) n / G) of the oracle's assembled mobility
    matrix; its share is that block of columns times the forces."""

    def __init__(self, x, fext, g):
        self.n = x.shape[0]
        self.x = np.array(x, dtype=np.float64)
        self.F = fext + g
        self.staged = None

    def _share(self, F, shard, nshards):
        import torch
        M = oracle.assemble(self.x)
        j0, j1 = shard * self.n // nshards, (shard + 1) * self.n // nshards
        P = (M[:, 3 * j0:3 * j1] @ np.asarray(F, dtype=np.float64).reshape(-1)[3 * j0:3 * j1]).reshape(self.n, 3)
        return torch.from_numpy(P)

    def mobility_apply_part(self, F, shard, nshards):
        return self._share(F.numpy(), shard, nshards)

    def mobility_apply_combine(self, Pall):
        V = Pall[0].clone()
        for q in range(1, Pall.shape[0]):
            V += Pall[q]
        return V

    def step_part(self, shard, nshards, P=None):
        return self._share(self.F, shard, nshards)

    def step_combine(self, dt, Pall):
        self.x = self.x + dt * self.mobility_apply_combine(Pall).numpy()


def _tile_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_1205_6333_gb300.distributed import tile_sharded_apply, tile_sharded_steps
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 200
    x0, _ = inputs.cube_rsa(n, 0.05, 903)
    fe = inputs.normal_forces(n, 904)
    g = np.array([0.0, 0.0, -1.0])
    sysr = _OracleTiles(x0, fe, g)
    V = tile_sharded_apply(sysr, torch.from_numpy(fe), rank, world, via_host=True)
    tile_sharded_steps(sysr, 0.05, 3, rank, world, via_host=True)
    out[rank] = (V.numpy().tobytes(), sysr.x.tobytes())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_tile_sharded_apply_and_steps_gloo(world):
    """Every rank computes a share of the sum for every row; after the all-gather and
    the combine in rank order every rank holds the same result, the full product."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_tile_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    n = 200
    x0, _ = inputs.cube_rsa(n, 0.05, 903)
    fe = inputs.normal_forces(n, 904)
    g = np.array([0.0, 0.0, -1.0])
    Vref = oracle.mobility_apply(x0, fe)
    xref = oracle.euler(x0, 3, 0.05, fe, g)
    V0 = np.frombuffer(out[0][0]).reshape(n, 3)
    x0r = np.frombuffer(out[0][1]).reshape(n, 3)
    for r in range(world):   # identical on every rank, bit for bit
        np.testing.assert_array_equal(np.frombuffer(out[r][0]).reshape(n, 3), V0)
        np.testing.assert_array_equal(np.frombuffer(out[r][1]).reshape(n, 3), x0r)
    assert np.abs(V0 - Vref).max() <= 1e-13 * np.abs(Vref).max()
    assert np.abs(x0r - xref).max() <= 1e-13 * np.abs(xref - x0).max()


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


# ---------------------------------------------------------------- tile shards on one GPU

_TILE_CASES = [("fp32c", "symmetric", 1e-5), ("fp32c", "directed", 1e-5), ("fp64", "symmetric", 1e-12),
               ("fp64", "directed", 1e-12)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec,dense,tol", _TILE_CASES)
def test_tile_shards_apply_match_oracle(prec, dense, tol):
    """Logical tile shards (1, 2, 3 and 7 of them) of the apply, combined in shard order,
    against the oracle element by element; overlapping pairs included."""
    import torch
    import paper_1205_6333_gb300 as sd
    from helpers import rel_err, system_with_overlaps
    n = 5000
    x, _ = system_with_overlaps(n, 0.05, seed=940, overlaps=5)
    F = inputs.normal_forces(n, 941)
    ref = oracle.mobility_apply(x, F, "rpy", nthreads=8)
    Ft = torch.tensor(F, dtype=torch.float64, device="cuda")
    with sd.System(n, prec=prec, dense=dense) as s:
        assert s.dense_kernel() == dense
        s.set_positions(x)
        full = s.mobility_apply(F)
        for G in (1, 2, 3, 7):
            Pall = torch.stack([s.mobility_apply_part(Ft, r, G) for r in range(G)])
            V = s.mobility_apply_combine(Pall).cpu().numpy()
            assert rel_err(V, ref) <= tol, (G, rel_err(V, ref))
            assert rel_err(V, full) <= (1e-14 if prec == "fp64" else 2e-6), G
        # host forces in, host velocities out
        Pall = torch.stack([s.mobility_apply_part(F, r, 2) for r in range(2)])
        assert rel_err(s.mobility_apply_combine(Pall, like=F), ref) <= tol


@pytest.mark.gpu
@pytest.mark.parametrize("prec,dense,tol", [("fp32c", "symmetric", 1e-5), ("fp64", "symmetric", 1e-10),
                                            ("fp64", "directed", 1e-10)])
def test_tile_shards_steps_match_oracle(prec, dense, tol):
    """Three logical ranks (three handles on one GPU), each computing its tile shard of
    every step; the shares are exchanged (stacked in rank order) and every rank
    finishes the step.  The three states stay identical bit for bit and follow the
    oracle's trajectory (gravity + soft repulsion, 10 steps)."""
    import torch
    import paper_1205_6333_gb300 as sd
    n, world, steps, dt = 3000, 3, 10, 0.02
    x0, _ = inputs.cube_rsa(n, 0.10, 950)
    fe = inputs.normal_forces(n, 951)
    g = (0.0, 0.0, -1.0)
    kw = dict(prec=prec, dense=dense, gravity=g, rep_eps=1.0, rep_rc=2.5)
    ref = oracle.euler(x0, steps, dt, fe, g, rep_eps=1.0, rep_rc=2.5, nthreads=8)
    ranks = [sd.System(n, **kw) for _ in range(world)]
    try:
        for s in ranks:
            s.set_positions(x0)
            s.set_forces(fe)
        for _ in range(steps):
            Pall = torch.stack([s.step_part(r, world) for r, s in enumerate(ranks)])
            for s in ranks:
                s.step_combine(dt, Pall)
        xs = [s.get_positions() for s in ranks]
    finally:
        for s in ranks:
            s.close()
    for xr in xs[1:]:
        np.testing.assert_array_equal(xr, xs[0])
    disp = np.linalg.norm(ref - x0, axis=1).max()
    assert np.linalg.norm(xs[0] - ref, axis=1).max() <= tol * disp


@pytest.mark.gpu
def test_tile_shards_lubrication_and_call_order():
    """Lubrication works with tile shards (every rank finishes every row, so the lagged
    velocities are complete); a combine without its part is refused."""
    import torch
    import paper_1205_6333_gb300 as sd
    m, spacing = 8, 2.8
    g1 = np.arange(m) * spacing
    x0 = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    x0 = x0 + np.random.default_rng(960).uniform(-0.05, 0.05, x0.shape)
    n = x0.shape[0]
    fe = inputs.normal_forces(n, 961)
    ref = oracle.euler(x0, 6, 0.02, fe, lubrication=True, nthreads=8)
    with sd.System(n, prec="fp64", lubrication=True) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        with pytest.raises(sd.SDError) as ei:
            s.step_combine(0.02, torch.zeros((1, n, 3), dtype=torch.float64, device="cuda"))
        assert ei.value.status_name == "SD_ERR_STATE"
        for _ in range(6):
            Pall = torch.stack([s.step_part(r, 2).clone() for r in range(2)])
            s.step_combine(0.02, Pall)
        xT = s.get_positions()
    disp = np.linalg.norm(ref - x0, axis=1).max()
    assert np.linalg.norm(xT - ref, axis=1).max() <= 1e-10 * disp


def _gpu_tile_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300.distributed import tile_sharded_apply, tile_sharded_steps
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 4000
    x0, _ = inputs.cube_rsa(n, 0.05, 970)
    fe = inputs.normal_forces(n, 971)
    with sd.System(n, gravity=(0.0, 0.0, -1.0)) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        V = tile_sharded_apply(s, torch.tensor(fe, device="cuda"), rank, world, via_host=True)
        tile_sharded_steps(s, 0.05, 4, rank, world, via_host=True)
        out[rank] = (V.cpu().numpy().tobytes(), s.get_positions().tobytes(), s.dense_kernel())
    dist.destroy_process_group()


@pytest.mark.gpu
def test_tile_sharded_two_processes_one_gpu():
    """distributed.tile_sharded_apply / tile_sharded_steps in two processes that share
    the GPU: real kernels, shares exchanged over gloo through host memory (no kernel
    waits on another process)."""
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_tile_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    from helpers import rel_err
    n = 4000
    x0, _ = inputs.cube_rsa(n, 0.05, 970)
    fe = inputs.normal_forces(n, 971)
    assert out[0][2] == "symmetric"
    V0 = np.frombuffer(out[0][0]).reshape(n, 3)
    X0 = np.frombuffer(out[0][1]).reshape(n, 3)
    np.testing.assert_array_equal(np.frombuffer(out[1][0]).reshape(n, 3), V0)
    np.testing.assert_array_equal(np.frombuffer(out[1][1]).reshape(n, 3), X0)
    assert rel_err(V0, oracle.mobility_apply(x0, fe, nthreads=8)) <= 1e-5
    ref = oracle.euler(x0, 4, 0.05, fe, (0.0, 0.0, -1.0), nthreads=8)
    assert np.linalg.norm(X0 - ref, axis=1).max() <= 1e-5 * np.linalg.norm(ref - x0, axis=1).max()

# ---------------------------------------------------------------- cluster shards (batched)

def _cluster_case():
    sizes = np.array([0, 5, 256, 3, 130, 0, 77, 200, 1, 64, 33, 150], dtype=np.int64)
    x, off = inputs.ball_rsa_batch(sizes, 0.05, 931)
    F = inputs.normal_forces(x.shape[0], 932)
    return x, off, F


def test_shard_clusters_partition():
    from paper_1205_6333_gb300.distributed import shard_clusters
    x, off, F = _cluster_case()
    sizes = np.diff(off)
    for world in [1, 2, 3, 5, 12, 20]:
        ranges = [shard_clusters(off, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == len(sizes)
        for (a0, b0), (a1, b1) in zip(ranges, ranges[1:]):
            assert b0 == a1 and a0 <= b0
        work = [int((sizes[a:b] ** 2).sum()) for a, b in ranges]
        # every rank is within one cluster's work of an equal share
        assert max(work) <= (sizes ** 2).sum() / world + (sizes ** 2).max()
    sizes = inputs.cluster_sizes(16384, 4, 256, 933)
    off = np.concatenate([[0], np.cumsum(sizes)])
    work = [int((sizes[a:b] ** 2).sum()) for a, b in (shard_clusters(off, r, 8) for r in range(8))]
    assert max(work) / (sum(work) / 8) < 1.005


def _cluster_worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_1205_6333_gb300.distributed import gather_cluster_rows, shard_clusters
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, off, F = _cluster_case()
    c0, c1 = shard_clusters(off, rank, world)
    local = []
    for c in range(c0, c1):   # the oracle stands in for this rank's batch
        a, b = off[c], off[c + 1]
        local.append(oracle.euler(x[a:b], 3, 0.01, fext=F[a:b]) if b > a else np.empty((0, 3)))
    xl = np.concatenate(local) if local else np.empty((0, 3))
    out[rank] = gather_cluster_rows(xl, off, rank, world).tobytes()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_cluster_shards_gloo(world):
    """Each rank steps its clusters; one all-gather gives every rank the whole batch,
    equal bit for bit to stepping all clusters in one place."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_cluster_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    x, off, F = _cluster_case()
    ref = np.concatenate([oracle.euler(x[off[c]:off[c + 1]], 3, 0.01, fext=F[off[c]:off[c + 1]])
                          for c in range(len(off) - 1) if off[c + 1] > off[c]])
    for r in range(world):
        np.testing.assert_array_equal(np.frombuffer(out[r]).reshape(-1, 3), ref)


@pytest.mark.gpu
@pytest.mark.parametrize("shape", ["sym", "blocks"])
def test_cluster_shards_logical_gpu(shape):
    """Two cluster shards on one GPU, each its own Batch with the same kernel pinned,
    give the whole batch's positions and match the oracle.  With the symmetric kernel
    bit for bit (a cluster's result does not depend on which clusters share its
    launch); the block kernel aligns its four-source steps to where a cluster lands in
    a CTA's staging area, which its neighbours decide, so there the shards agree to
    FP32 rounding."""
    from paper_1205_6333_gb300.distributed import ShardedBatch
    import paper_1205_6333_gb300 as sd
    x, off, F = _cluster_case()
    r = 0 if shape == "sym" else 1

    def pin(b):
        b.set_shape(next(k for k, sh in enumerate(b.shapes()) if sh["targets_per_thread"] == r and sh["threads"] == 128))

    full = sd.Batch(off.astype(np.int32))
    pin(full)
    full.set_positions(x)
    full.set_forces(F)
    full.step(0.01, 5)
    xf = full.get_positions()
    full.close()
    xs = np.zeros_like(x)
    for rank in range(2):
        sb = ShardedBatch(off, rank, 2)
        pin(sb.batch)
        sb.set_positions(x)
        sb.set_forces(F)
        sb.step(0.01, 5)
        sb.get_positions(xs)
        sb.close()
    if shape == "sym":
        np.testing.assert_array_equal(xs, xf)
    else:
        assert np.abs(xs - xf).max() <= 1e-7 * np.abs(xf - x).max()
    for c in range(len(off) - 1):
        a, b = off[c], off[c + 1]
        if b > a:
            ref = oracle.euler(x[a:b], 5, 0.01, fext=F[a:b])
            assert np.abs(xs[a:b] - ref).max() <= 1e-5 * max(np.abs(ref - x[a:b]).max(), 1e-300)
