"""Sharding of sine modes across ranks.

In the sine basis every mode of the two-state system evolves independently for
all N steps, so a problem splits over ranks by contiguous ranges of modes with no
exchange during the time loop; the only collective is the final gather of the
modal result (or, for gradients, a sum of two scalars).
"""
from __future__ import annotations


def mode_shards(nmodes: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [lo, hi) ranges, one per rank, sizes differing by at most one."""
    if world < 1:
        raise ValueError("world >= 1")
    base, extra = divmod(nmodes, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def gather_modal(local, nmodes: int, group=None):
    """All-gather the [2][hi-lo] modal shards of every rank into a [2][nmodes] tensor."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    shards = mode_shards(nmodes, world)
    width = max(hi - lo for lo, hi in shards)
    buf = torch.zeros((2, width), dtype=local.dtype, device=local.device)
    buf[:, : local.shape[1]] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:, : hi - lo] for p, (lo, hi) in zip(parts, shards)], dim=1)


def solve_sharded(fc, problem, g0_modal, group=None, stream=None):
    """This rank's contiguous shard of the sine modes solved with ``fp2s_solve_modes`` (no
    exchange during the time loop), then the modal G^N of every rank all-gathered.

    ``fc`` is the binding module, ``problem`` an ``fp2s_problem_t`` and ``g0_modal`` the
    [2][M^dim] sine coefficients of G^0 on this rank's device (every rank holds them; only
    its shard is read). Returns the [2][M^dim] modal G^N. A rank whose shard is empty (more
    ranks than modes) solves nothing and contributes an empty shard."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    nm = g0_modal.shape[1]
    lo, hi = mode_shards(nm, world)[rank]
    if hi > lo:
        g0 = g0_modal[:, lo:hi].contiguous()
        gN = torch.empty_like(g0)
        ws = fc.workspace(fc.fp2s_solve_modes(problem, lo, hi, g0, gN, None, stream=stream), g0.device)
        fc.fp2s_solve_modes(problem, lo, hi, g0, gN, ws, stream=stream)
    else:
        gN = torch.empty((2, 0), dtype=g0_modal.dtype, device=g0_modal.device)
    return gather_modal(gN, nm, group)
