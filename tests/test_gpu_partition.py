"""libsem's operator applied on a slab partition (Section 4.1's distributed cell
loop): two ranks (processes, gloo) each create a libsem context for their own
element layers, apply the FP64 operator on the GPU, sum the interface planes
through host memory, and together reproduce the global apply of an
unpartitioned context to 1e-13, and its inner product u . A u.  Both ranks use
the one GPU of the box; their kernels never wait on each other (the exchange is
between host processes)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, quad, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    from datetime import timedelta
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=120))
    try:
        import workloads as W
        import paper_2205_05136_gb300 as gb
        from paper_2205_05136_gb300.partition import SlabPartition
        nx, ny, nz, p = 6, 5, 7, 3
        s = W.slab(nx, ny, nz, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
        rng = np.random.default_rng(5)
        ne = s.n_elements
        sl, st = 0.12 * rng.uniform(0.8, 1.2, ne), 0.03 * rng.uniform(0.8, 1.2, ne)
        th = W.transmural_fiber_angles(s)
        part = SlabPartition(nx, ny, nz, p, rank, world)
        e0, e1 = part.local_elements().start, part.local_elements().stop
        # this rank's layers as a slab of their own
        loc = gb.Slab(part.sub_slab_vertices(s.flat_vertices()), nx, ny, part.ez1 - part.ez0, p, quad)
        loc.set_tissue(sl[e0:e1], st[e0:e1], th[e0:e1])
        assert loc.ndofs == part.nlocal
        u = W.uniform_vector((p * nx + 1) * (p * ny + 1) * (p * nz + 1), -1.0, 1.0, seed=2)
        lo, hi = part.local_range()
        y = loc.apply(torch.tensor(u[lo:hi], device="cuda"), 30.0, 1.0).cpu()
        part.exchange(y, timeout_s=60.0)
        d = part.dot(torch.tensor(u[lo:hi]), y, timeout_s=60.0)
        # the unpartitioned context on the same device
        g = gb.Slab(s.flat_vertices(), nx, ny, nz, p, quad)
        g.set_tissue(sl, st, th)
        yg = g.apply(torch.tensor(u, device="cuda"), 30.0, 1.0).cpu().numpy()
        err = float(np.abs(y.numpy() - yg[lo:hi]).max() / np.abs(yg).max())
        derr = abs(d - float(u @ yg)) / abs(float(u @ yg))
        out[rank] = (err, derr)
        loc.close()
        g.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_libsem_partitioned_apply_equals_global(quad):
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, quad, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(300)
        assert pr.exitcode == 0
    for r in range(world):
        err, derr = out[r]
        assert err < 1e-13, (r, err)
        assert derr < 1e-13, (r, derr)
