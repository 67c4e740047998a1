"""Sharding a batch of simulations across ranks (one process per GPU).

A batch splits by instance.  Instances are the tasks of one design (Eq. 35,
arxiv 2503.22767) or independent design candidates.  Every instance runs
whole on one rank, so a substep needs no communication.  A single instance
does not shard; it runs as a replica on each rank.

Multi-task sharing (Eq. 35) adds each task's gradient to its shared design.
When a design's tasks land on different ranks, their gradients are summed
with one sum-allreduce per design iteration.  Designs held by one rank
exchange nothing.

Everything here is host logic.  The plan is a pure function of the particle
counts, and the reduction runs on whatever process group the caller set up
(NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from .workloads import MpmConfig, Workload


@dataclass
class ShardPlan:
    """Assignment of the global instances to ``world`` ranks."""

    world: int
    owner: List[int]  # rank of each global instance
    local: List[List[int]]  # global instance ids of each rank, ascending
    counts: List[int]  # particle count of each global instance
    designs: List[int]  # design of each global instance
    shared: List[int]  # designs whose instances sit on more than one rank

    def load(self, rank: int) -> int:
        """Particles held by ``rank``."""
        return sum(self.counts[i] for i in self.local[rank])

    def local_designs(self, rank: int) -> List[int]:
        """Global design ids used on ``rank``, ascending (the local design order)."""
        return sorted({self.designs[i] for i in self.local[rank]})


def plan(counts, designs: Optional[List[int]], world: int) -> ShardPlan:
    """Balance instances over ``world`` ranks by particle count.

    The rule is greedy longest-processing-time: instances go in order of
    decreasing count (ties by id) to the rank with the fewest particles (ties
    to the lowest rank).  Its load is within one instance of the optimum
    (at most 4/3 of it).  A rank may receive no instance when
    world > len(counts).
    """
    counts = [int(c) for c in counts]
    if world < 1:
        raise ValueError("world must be >= 1")
    n = len(counts)
    designs = list(range(n)) if designs is None else [int(d) for d in designs]
    if len(designs) != n:
        raise ValueError("designs must have one entry per instance")
    order = sorted(range(n), key=lambda i: (-counts[i], i))
    load = [0] * world
    owner = [0] * n
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += counts[i]
    local = [[i for i in range(n) if owner[i] == r] for r in range(world)]
    ranks_of = {}
    for i, d in enumerate(designs):
        ranks_of.setdefault(d, set()).add(owner[i])
    shared = sorted(d for d, rs in ranks_of.items() if len(rs) > 1)
    return ShardPlan(world, owner, local, counts, designs, shared)


def local_workload(w: Workload, p: ShardPlan, rank: int) -> Workload:
    """The instances of ``rank`` as a workload of their own.

    Design ids are renumbered 0.. in ascending global order.  phi / mag hold
    only the local designs.
    """
    cfg = w.cfg
    ioff = np.concatenate([[0], np.cumsum(cfg.counts)]).astype(np.int64)
    dcounts = cfg.design_counts()
    doff = np.concatenate([[0], np.cumsum(dcounts)]).astype(np.int64)
    inst = p.local[rank]
    gdes = p.local_designs(rank)
    remap = {g: k for k, g in enumerate(gdes)}

    def take_particles(a):
        if a is None:
            return None
        return np.ascontiguousarray(np.concatenate([a[:, ioff[i]:ioff[i + 1]] for i in inst], axis=1))

    def take_designs(a):
        return np.ascontiguousarray(np.concatenate([a[..., doff[g]:doff[g + 1]] for g in gdes], axis=-1))

    shared_design = cfg.design_of_instance is not None
    lcfg = MpmConfig(**{**cfg.as_dict(), "counts": [cfg.counts[i] for i in inst],
                        "design_of_instance": [remap[p.designs[i]] for i in inst] if shared_design else None})
    return Workload(f"{w.name}[rank {rank}/{p.world}]", lcfg, take_particles(w.x0), take_particles(w.v0),
                    take_designs(w.phi), take_designs(w.mag),
                    np.ascontiguousarray(w.field[inst]), take_particles(w.target), dict(w.meta))


def reduce_design_grads(p: ShardPlan, rank: int, dim: int, g_phi, g_mag, group=None) -> int:
    """Sum the gradients of designs shared across ranks, in place.

    g_phi [Nd_local] and g_mag [dim][Nd_local] are torch tensors in the local
    design order of ``rank``.  On return, every shared design holds the sum
    over all ranks of its tasks' gradients (Eq. 35).  The other designs are
    untouched.  Returns the number of collectives issued: 0 when no design is
    shared, else 1.  The call is collective over ``group``, and every rank
    must make it.
    """
    if not p.shared or p.world == 1:
        return 0
    import torch
    import torch.distributed as dist

    dcount = {}
    for i, d in enumerate(p.designs):
        dcount[d] = p.counts[i]
    # one packed buffer over the shared designs, in global design order:
    # [phi block | mag rows] per design
    sizes = [dcount[d] * (1 + dim) for d in p.shared]
    buf = torch.zeros(int(sum(sizes)), dtype=g_phi.dtype, device=g_phi.device)
    gdes = p.local_designs(rank)
    loff = {}
    o = 0
    for g in gdes:
        loff[g] = o
        o += dcount[g]
    off = 0
    for d, sz in zip(p.shared, sizes):
        n = dcount[d]
        if d in loff:
            a = loff[d]
            buf[off:off + n] = g_phi[a:a + n]
            buf[off + n:off + sz] = g_mag[:, a:a + n].reshape(-1)
        off += sz
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for d, sz in zip(p.shared, sizes):
        n = dcount[d]
        if d in loff:
            a = loff[d]
            g_phi[a:a + n] = buf[off:off + n]
            g_mag[:, a:a + n] = buf[off + n:off + sz].reshape(dim, n)
        off += sz
    return 1
