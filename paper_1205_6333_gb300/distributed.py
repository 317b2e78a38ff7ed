"""One system split over several devices by target rows (one process per GPU,
torch.distributed; Sec. 3.1 step 3 with the rows of the sum divided between ranks).

Every rank holds the whole state (all n positions and forces) in its own
``System`` created with ``dense="directed"``.  Rank r owns the rows of
``shard_rows(n, r, world)``:

* ``sharded_apply``: the rank computes v for its rows with
  ``sd_mobility_apply_rows`` (the whole sum over j, in the library's kernels),
  and an all-gather assembles the n velocities;
* ``sharded_steps``: per step the rank advances its rows with ``sd_step_rows``,
  and an all-gather of positions (24 B per particle) restores the replicated
  state before the next step.

Each row is bit-identical to the unsharded result.  This module only partitions
rows and moves data (device-to-device copies and the collective); it does no
arithmetic of the method.  Collectives run on the default process group unless
``group`` is given (NCCL between GPUs, gloo for host tensors).
"""
from __future__ import annotations

ROW_BLOCK = 256   # i-block of the directed all-pairs kernels: shards of whole blocks share no work


def shard_rows(n: int, rank: int, world: int, block: int = ROW_BLOCK):
    """Contiguous rows [r0, r1) of `rank`: whole `block`-row blocks, as even as possible."""
    nb = (n + block - 1) // block
    b0 = rank * nb // world
    b1 = (rank + 1) * nb // world
    return min(b0 * block, n), min(b1 * block, n)


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
    """v = mu(x) F on `world` ranks: F is the whole n x 3 force tensor on every rank;
    returns the whole n x 3 velocity tensor on every rank."""
    import torch
    n = system.n
    r0, r1 = shard_rows(n, rank, world)
    V = torch.zeros((n, 3), dtype=F.dtype, device=F.device)
    if r1 > r0:
        V[r0:r1] = system.mobility_apply_rows(F, r0, r1)
    return _gather_rows(V, rank, world, group)


def sharded_steps(system, dt: float, nsteps: int, rank: int, world: int, x=None, group=None):
    """nsteps Euler steps of a replicated system, each rank advancing its own rows.
    `x` (n x 3 float64 tensor on the system's device, optional) is used as the
    exchange buffer and holds the positions after the last step."""
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
