"""Partitioned operator apply on CPU ranks (gloo, world size 2 and 3): each
rank applies the oracle's element-by-element operator on its own element
layers, the interface planes are summed with the neighbours, and the result
equals the unpartitioned apply to 1e-14; partitioned inner products equal
the global ones."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, quad, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import workloads as W
        from oracle import mesh as Mh
        from paper_2205_05136_gb300.partition import SlabPartition
        s = W.slab(3, 2, 5, (3.0, 2.0, 5.0), perturb=0.1, seed=1)
        p = 2
        sp_ = Mh.SlabSpace(s.flat_vertices(), 3, 2, 5, p, quad)
        tissue = (np.full(s.n_elements, 0.12), np.full(s.n_elements, 0.03), W.transmural_fiber_angles(s))
        u = W.uniform_vector(sp_.ndofs, seed=2)
        part = SlabPartition(3, 2, 5, p, rank, world)
        y_global_local_elems = Mh.apply_element_by_element(sp_, tissue, u, 30.0, 1.0,
                                                           elements=part.local_elements())
        lo, hi = part.local_range()
        y_local = torch.tensor(y_global_local_elems[lo:hi])
        part.exchange(y_local)
        full = Mh.apply_element_by_element(sp_, tissue, u, 30.0, 1.0)
        err = float(np.abs(y_local.numpy() - full[lo:hi]).max() / np.abs(full).max())
        d = part.dot(torch.tensor(u[lo:hi]), y_local)
        derr = abs(d - float(u @ full)) / abs(float(u @ full))
        out[rank] = (err, derr)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_partitioned_apply_equals_global(world, quad):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, quad, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    for r in range(world):
        err, derr = out[r]
        assert err < 1e-14, (r, err)
        assert derr < 1e-13, (r, derr)


def test_split_layers_is_balanced_and_covering():
    from paper_2205_05136_gb300.partition import split_layers
    for nz in (2, 5, 13):
        for w in range(1, min(nz, 6) + 1):
            parts = split_layers(nz, w)
            assert parts[0][0] == 0 and parts[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
