"""Partitioned runs across processes: the host side of the multi-process layout.

The paper renumbers its grid once before time stepping, for every process
(Sec. III-B).  A partitioned run gives rank r the contiguous slab of the
renumbered element order that ``dg_partition_plan`` assigns (slab boundaries
on multiples of 96 elements, a common multiple of the kernels' tile sizes)
and a halo: the other
ranks' elements that its own elements' faces reach.  Per residual evaluation
a rank needs one halo exchange; the time step and the conserved totals are
reduced over the ranks.

This module holds the communication of that layout over a
``torch.distributed`` process group -- who needs which blocks from whom
(exchanged once), the block exchange itself (point-to-point send/recv into
a local halo buffer, so that every kernel reads local memory only), and the
min / sum reductions.  It does no arithmetic of the method.  The single-device
emulation of the same layout (k partitions on one GPU, the exchange a device
gather) is ``dg_partition_create`` / ``dg_partition_residual`` in the C ABI.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import dg


@dataclass
class Plan:
    """Partition r of k: own slab [first, first + count) of internal element
    ids, the halo's internal ids (ascending) and each halo element's owner."""
    rank: int
    k: int
    first: int
    count: int
    halo_ids: np.ndarray
    halo_part: np.ndarray


def make_plan(tet_vid, tet_xyz, bc_tag, renumber, k, rank) -> Plan:
    first, count, ids, part = dg.dg_partition_plan(tet_vid, tet_xyz, bc_tag, renumber, k, rank)
    return Plan(rank, k, first, count, ids, part)


class HaloExchange:
    """Point-to-point halo exchange of element blocks between the ranks of a
    process group.  Construction exchanges, once, which blocks every rank needs
    from every other (the request lists); ``exchange`` then sends each peer the
    blocks it asked for and receives the own halo, in halo order."""

    def __init__(self, plan: Plan, group=None):
        import torch.distributed as dist
        self.plan, self.group = plan, group
        world = dist.get_world_size(group)
        if world != plan.k:
            raise ValueError(f"process group has {world} ranks, the plan {plan.k} partitions")
        # what this rank needs from each peer: positions in its halo and the owners' local ids
        self.recv_from = {}
        for q in range(plan.k):
            sel = np.nonzero(plan.halo_part == q)[0]
            if len(sel):
                self.recv_from[q] = sel
        requests = [None] * world
        dist.all_gather_object(requests, {q: plan.halo_ids[sel].tolist() for q, sel in self.recv_from.items()},
                               group=group)
        # what each peer needs from this rank, as local ids of the own slab
        self.send_to = {}
        for q in range(world):
            ids = requests[q].get(plan.rank, []) if q != plan.rank else []
            if ids:
                self.send_to[q] = np.asarray(ids, dtype=np.int64) - plan.first

    def exchange(self, own, halo):
        """own: [count, ...] tensor of this rank's blocks; halo: [nhalo, ...]
        tensor, filled in halo order.  Non-blocking sends and receives,
        completed before return."""
        import torch
        import torch.distributed as dist
        reqs, bufs = [], []
        for q, lid in self.send_to.items():
            blk = own[torch.as_tensor(lid, device=own.device)].contiguous()
            bufs.append(blk)
            reqs.append(dist.isend(blk, q, group=self.group))
        recv = {}
        for q, pos in self.recv_from.items():
            buf = torch.empty((len(pos),) + tuple(halo.shape[1:]), dtype=halo.dtype, device=halo.device)
            recv[q] = buf
            reqs.append(dist.irecv(buf, q, group=self.group))
        for r in reqs:
            r.wait()
        for q, pos in self.recv_from.items():
            halo[torch.as_tensor(pos, device=halo.device)] = recv[q]
        return halo


def allreduce_min(x, group=None):
    """The time-step minimum over the ranks (exact: a minimum has no rounding)."""
    import torch.distributed as dist
    dist.all_reduce(x, op=dist.ReduceOp.MIN, group=group)
    return x


def allreduce_sum(x, group=None):
    """The conserved totals over the ranks (equal to one rank's sum of everything up to the
    summation order)."""
    import torch.distributed as dist
    dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
    return x
