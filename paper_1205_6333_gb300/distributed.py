"""One system split over several devices (one process per GPU, torch.distributed).

Two splits of the all-pairs sum of Sec. 3.1 step 3 are offered; in both, every
rank holds the whole state (all n positions and forces) in its own ``System``.

Tile shards (either all-pairs kernel, every precision; the default):
  Rank r runs the CTAs [r G / world, (r + 1) G / world) of the all-pairs kernel's
  persistent launch of G CTAs (``sd_*_part``): its share of the pair sum for every
  row.  One all-gather of those FP64 shares (24 B per particle and rank) brings all
  of them to every rank, and ``sd_*_combine`` adds them in rank order with the self
  term and the FP64 near-pair corrections.  Each rank therefore finishes the step
  for every particle, identically, and no positions need to be exchanged.

Row shards (the directed kernel only):
  Rank r computes the velocities of its own rows (``sd_*_rows``) and an all-gather
  of those rows (24 B per particle) restores the replicated state.

Cluster shards (batched workloads): the clusters are independent, so rank r simply
steps a contiguous run of them (``shard_clusters``, ``ShardedBatch``), balanced by
pair work (the sum of N_c^2); no data moves between ranks.

This module only partitions the work and moves data (the collective and nothing
else); every step of the method runs in the library's kernels.  Collectives run on
the default process group unless ``group`` is given (NCCL between GPUs; gloo with
host staging, ``via_host=True``, for tests that share one GPU between processes).
"""
from __future__ import annotations

ROW_BLOCK = 256   # i-block of the directed all-pairs kernels: shards of whole blocks share no work


def shard_rows(n: int, rank: int, world: int, block: int = ROW_BLOCK):
    """Contiguous rows [r0, r1) of `rank`: whole `block`-row blocks, as even as possible."""
    nb = (n + block - 1) // block
    b0 = rank * nb // world
    b1 = (rank + 1) * nb // world
    return min(b0 * block, n), min(b1 * block, n)


def _all_gather_parts(P, world, group=None, via_host=False, out=None):
    """(world, n, 3) tensor of every rank's P, in rank order."""
    import torch
    import torch.distributed as dist
    if via_host:
        src = P.cpu()
        recv = [torch.empty_like(src) for _ in range(world)]
        dist.all_gather(recv, src, group=group)
        return torch.stack(recv).to(P.device)
    if out is None:
        out = torch.empty((world,) + tuple(P.shape), dtype=P.dtype, device=P.device)
    dist.all_gather_into_tensor(out, P, group=group)
    return out


def tile_sharded_apply(system, F, rank: int, world: int, group=None, via_host=False):
    """v = mu(x) F on `world` ranks by tile shards: F is the whole n x 3 force tensor on
    every rank; returns the whole n x 3 FP64 velocity tensor (CUDA) on every rank."""
    P = system.mobility_apply_part(F, rank, world)
    Pall = _all_gather_parts(P, world, group, via_host)
    return system.mobility_apply_combine(Pall)


def tile_sharded_steps(system, dt: float, nsteps: int, rank: int, world: int, group=None, via_host=False):
    """nsteps Euler steps of a replicated system by tile shards (one all-gather of the
    FP64 shares per step; the state stays identical on every rank)."""
    P = Pall = None
    for _ in range(int(nsteps)):
        P = system.step_part(rank, world, P)
        Pall = _all_gather_parts(P, world, group, via_host, out=Pall)
        system.step_combine(dt, Pall)


def _gather_rows(local_full, rank, world, group=None):
    """Replace, in the n x 3 tensor `local_full`, every other rank's rows by that rank's
    values (all-gather of equal-size padded row blocks)."""
    import torch
    import torch.distributed as dist
    n = local_full.shape[0]
    ranges = [shard_rows(n, r, world) for r in range(world)]
    chunk = max(b - a for a, b in ranges)
    r0, r1 = ranges[rank]
    send = torch.zeros((chunk, 3), dtype=local_full.dtype, device=local_full.device)
    send[: r1 - r0] = local_full[r0:r1]
    recv = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(recv, send, group=group)
    for r, (a, b) in enumerate(ranges):
        if r != rank:
            local_full[a:b] = recv[r][: b - a]
    return local_full


def sharded_apply(system, F, rank: int, world: int, group=None):
    """Row shards: v = mu(x) F on `world` ranks (directed kernel); F is the whole n x 3
    force tensor on every rank; returns the whole n x 3 velocity tensor on every rank."""
    import torch
    n = system.n
    r0, r1 = shard_rows(n, rank, world)
    V = torch.zeros((n, 3), dtype=F.dtype, device=F.device)
    if r1 > r0:
        V[r0:r1] = system.mobility_apply_rows(F, r0, r1)
    return _gather_rows(V, rank, world, group)


def sharded_steps(system, dt: float, nsteps: int, rank: int, world: int, x=None, group=None):
    """Row shards: nsteps Euler steps of a replicated system, each rank advancing its
    own rows.  `x` (n x 3 float64 tensor on the system's device, optional) is used as
    the exchange buffer and holds the positions after the last step."""
    import torch
    n = system.n
    r0, r1 = shard_rows(n, rank, world)
    if x is None:
        x = torch.empty((n, 3), dtype=torch.float64,
                        device="cuda" if torch.cuda.is_available() else "cpu")
    for _ in range(int(nsteps)):
        system.step_rows(dt, r0, r1)
        system.get_positions(x)
        _gather_rows(x, rank, world, group)
        system.set_positions(x)
    return x


def shard_clusters(offsets, rank: int, world: int):
    """Contiguous clusters [c0, c1) of `rank`, cut where the running pair work (the sum
    of N_c^2 over the clusters before the cut) first reaches rank / world of the total,
    so every rank gets about the same work (up to one cluster's)."""
    import numpy as np
    off = np.asarray(offsets, dtype=np.int64)
    nc = off.size - 1
    work = np.cumsum(np.diff(off) ** 2)
    total = int(work[-1]) if nc > 0 else 0

    def cut(r):
        if r <= 0 or nc == 0:
            return 0
        if r >= world:
            return nc
        return int(np.searchsorted(work, total * r / world, side="left")) + 1

    c0, c1 = cut(rank), cut(rank + 1)
    return min(c0, nc), min(max(c1, c0), nc)


class ShardedBatch:
    """This rank's share of a batch of independent clusters: the clusters
    [c0, c1) of ``shard_clusters`` as one ``Batch``.  Positions and forces are given and
    returned for the whole batch (n_total x 3); only this rank's rows are used or
    written."""

    def __init__(self, offsets, rank: int, world: int, **kw):
        import numpy as np
        from . import Batch
        off = np.asarray(offsets, dtype=np.int64)
        self.c0, self.c1 = shard_clusters(off, rank, world)
        self.p0, self.p1 = int(off[self.c0]), int(off[self.c1])
        # (more ranks than clusters: an empty share, no batch)
        self.batch = Batch((off[self.c0:self.c1 + 1] - self.p0).astype(np.int32), **kw) if self.c1 > self.c0 else None

    def set_positions(self, x):
        if self.batch:
            self.batch.set_positions(x[self.p0:self.p1])

    def set_forces(self, f):
        if self.batch:
            self.batch.set_forces(f[self.p0:self.p1])

    def step(self, dt, nsteps=1):
        if self.batch:
            self.batch.step(dt, nsteps)

    def get_positions(self, out):
        """Writes this rank's rows of `out` (the whole batch's n_total x 3 array)."""
        if self.batch:
            out[self.p0:self.p1] = self.batch.get_positions()
        return out

    def close(self):
        if self.batch:
            self.batch.close()


def gather_cluster_rows(x_local, offsets, rank: int, world: int, group=None):
    """The whole batch's n_total x 3 positions on every rank, from each rank's rows of
    its ``shard_clusters`` share (x_local, a CPU tensor or array): one all-gather of
    equal-size padded blocks."""
    import numpy as np
    import torch
    import torch.distributed as dist
    off = np.asarray(offsets, dtype=np.int64)
    ranges = [shard_clusters(off, r, world) for r in range(world)]
    rows = [(int(off[a]), int(off[b])) for a, b in ranges]
    chunk = max(max(b - a for a, b in rows), 1)
    send = torch.zeros((chunk, 3), dtype=torch.float64)
    p0, p1 = rows[rank]
    send[: p1 - p0] = torch.as_tensor(np.asarray(x_local), dtype=torch.float64)[: p1 - p0]
    recv = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(recv, send, group=group)
    out = np.empty((int(off[-1]), 3))
    for r, (a, b) in enumerate(rows):
        out[a:b] = recv[r][: b - a].numpy()
    return out
