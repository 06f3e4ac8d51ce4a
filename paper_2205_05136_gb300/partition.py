"""Distributed-memory partition of a slab for the matrix-free operator.

Section 4.1: the mesh cells and degrees of freedom are partitioned among
processes; each process applies the operator on its own cells, and the
results at nodes shared between processes must be summed.  This module gives
the host logic of that partition for a structured slab cut into contiguous
layers of elements along z:

* rank r owns element layers [ez0, ez1) and the node planes K in
  [ez0 p, ez1 p] (the planes at a cut belong to both neighbours);
* after a local operator apply, the two interface planes are summed with the
  neighbours (one exchange per apply, with torch.distributed send / recv);
* inner products count each node once: a node plane at a cut is owned by the
  upper rank.

On this GB300 pool every process gets one GPU, so the benchmark runs
independent replicas; the partition is exercised by CPU ranks (gloo).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist


def split_layers(nz: int, world: int):
    """Balanced contiguous split of nz element layers over `world` ranks."""
    if world > nz:
        raise ValueError("more ranks than element layers")
    base, extra = divmod(nz, world)
    out, start = [], 0
    for r in range(world):
        cnt = base + (1 if r < extra else 0)
        out.append((start, start + cnt))
        start += cnt
    return out


@dataclass
class SlabPartition:
    nx: int
    ny: int
    nz: int
    p: int
    rank: int
    world: int

    def __post_init__(self):
        self.ez0, self.ez1 = split_layers(self.nz, self.world)[self.rank]
        self.NX = self.p * self.nx + 1
        self.NY = self.p * self.ny + 1
        self.plane = self.NX * self.NY
        self.K0 = self.ez0 * self.p
        self.K1 = self.ez1 * self.p
        self.nlocal = (self.K1 - self.K0 + 1) * self.plane
        self.offset = self.K0 * self.plane  # global index of local node 0

    def local_elements(self):
        """Global indices (x fastest) of this rank's elements."""
        per_layer = self.nx * self.ny
        return range(self.ez0 * per_layer, self.ez1 * per_layer)

    def local_range(self):
        """Global node range [start, stop) held by this rank (interface planes included)."""
        return self.offset, self.offset + self.nlocal

    def owned_mask(self) -> torch.Tensor:
        """1 for nodes this rank owns in inner products (cut planes: the upper rank)."""
        m = torch.ones(self.nlocal, dtype=torch.float64)
        if self.rank < self.world - 1:
            m[-self.plane:] = 0.0
        return m

    def exchange(self, y_local: torch.Tensor, group=None) -> torch.Tensor:
        """Sum the interface planes with the neighbouring ranks (in place)."""
        reqs = []
        bufs = {}
        if self.rank > 0:
            lo = y_local[:self.plane].contiguous()
            bufs["lo"] = torch.empty_like(lo)
            reqs.append(dist.isend(lo, self.rank - 1, group=group))
            reqs.append(dist.irecv(bufs["lo"], self.rank - 1, group=group))
        if self.rank < self.world - 1:
            hi = y_local[-self.plane:].contiguous()
            bufs["hi"] = torch.empty_like(hi)
            reqs.append(dist.isend(hi, self.rank + 1, group=group))
            reqs.append(dist.irecv(bufs["hi"], self.rank + 1, group=group))
        for r in reqs:
            r.wait()
        if "lo" in bufs:
            y_local[:self.plane] += bufs["lo"]
        if "hi" in bufs:
            y_local[-self.plane:] += bufs["hi"]
        return y_local

    def dot(self, a: torch.Tensor, b: torch.Tensor, group=None) -> float:
        """Global inner product of two local vectors (each node counted once)."""
        v = torch.sum(a * b * self.owned_mask().to(a.device)).reshape(1).to(torch.float64)
        dist.all_reduce(v, group=group)
        return float(v.item())
