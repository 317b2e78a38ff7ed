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
