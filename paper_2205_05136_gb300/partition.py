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
  upper rank;
* a neighbour that fails (its process exits, or it stops answering) makes the
  next exchange or inner product raise PeerLost on the other ranks within the
  given timeout instead of waiting forever.

Each rank's elements form a slab of their own (sub_slab_vertices), so a rank
can apply libsem's operator to its layers on its device and exchange the
interface planes through host memory.  On this GB300 pool every process gets
one GPU, so the benchmark runs independent replicas; the partition is
exercised by CPU ranks (gloo), with the oracle's or libsem's local apply.
"""
from __future__ import annotations

from dataclasses import dataclass
from datetime import timedelta

import numpy as np
import torch
import torch.distributed as dist


class PeerLost(RuntimeError):
    """A neighbouring rank did not take part in an exchange or reduction in time."""


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

    def exchange(self, y_local: torch.Tensor, group=None, timeout_s: float | None = None) -> torch.Tensor:
        """Sum the interface planes with the neighbouring ranks (in place).  With
        timeout_s, a neighbour that has exited or does not answer within that
        many seconds raises PeerLost."""
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
            try:
                if timeout_s is None:
                    r.wait()
                else:
                    r.wait(timeout=timedelta(seconds=timeout_s))
            except RuntimeError as exc:
                raise PeerLost(f"rank {self.rank}: interface exchange with a neighbour failed: {exc}") from exc
        if "lo" in bufs:
            y_local[:self.plane] += bufs["lo"]
        if "hi" in bufs:
            y_local[-self.plane:] += bufs["hi"]
        return y_local

    def dot(self, a: torch.Tensor, b: torch.Tensor, group=None, timeout_s: float | None = None) -> float:
        """Global inner product of two local vectors (each node counted once);
        PeerLost when a rank does not join the reduction within timeout_s."""
        v = torch.sum(a * b * self.owned_mask().to(a.device)).reshape(1).to(torch.float64)
        try:
            work = dist.all_reduce(v, group=group, async_op=True)
            if timeout_s is None:
                work.wait()
            else:
                work.wait(timeout=timedelta(seconds=timeout_s))
        except RuntimeError as exc:
            raise PeerLost(f"rank {self.rank}: inner product reduction failed: {exc}") from exc
        return float(v.item())

    def sub_slab_vertices(self, vertices) -> np.ndarray:
        """The vertex lattice of this rank's element layers, (nx+1)(ny+1)(ez1-ez0+1)
        points, x fastest, taken from the global lattice (same point order)."""
        v = np.asarray(vertices, dtype=np.float64).reshape(self.nz + 1, self.ny + 1, self.nx + 1, 3)
        return np.ascontiguousarray(v[self.ez0:self.ez1 + 1].reshape(-1, 3))
