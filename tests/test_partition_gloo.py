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


def _failing_worker(rank, world, port, mode, out):
    """Rank 1 stops after the first exchange (its process exits, or it goes
    silent); the other ranks' next exchange and inner product raise PeerLost
    within the timeout instead of waiting forever."""
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    from datetime import timedelta
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=20))
    from paper_2205_05136_gb300.partition import PeerLost, SlabPartition
    part = SlabPartition(3, 2, 6, 2, rank, world)
    y = torch.ones(part.nlocal, dtype=torch.float64)
    part.exchange(y, timeout_s=10.0)
    out[(rank, "first")] = float(y[0])
    if rank == 1:
        if mode == "exit":
            os._exit(0)  # the process ends between two applies
        time.sleep(25.0)  # alive but silent
        os._exit(0)
    t0 = time.perf_counter()
    try:
        part.exchange(torch.ones(part.nlocal, dtype=torch.float64), timeout_s=3.0)
        out[(rank, "second")] = "no error"
    except PeerLost as exc:
        out[(rank, "second")] = ("PeerLost", time.perf_counter() - t0, str(exc)[:200])
    try:
        part.dot(torch.ones(part.nlocal, dtype=torch.float64), torch.ones(part.nlocal, dtype=torch.float64),
                 timeout_s=3.0)
        out[(rank, "dot")] = "no error"
    except PeerLost:
        out[(rank, "dot")] = "PeerLost"
    os._exit(0)


@pytest.mark.parametrize("mode", ["exit", "silent"])
def test_lost_rank_is_detected_not_waited_for(mode):
    import time
    world = 3
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, world, port, mode, out)) for r in range(world)]
    t0 = time.perf_counter()
    for pr in procs:
        pr.start()
    for pr in (procs[0], procs[2]):
        pr.join(60)
        assert pr.exitcode == 0, pr.exitcode
    elapsed = time.perf_counter() - t0
    procs[1].join(40)
    for r in (0, 2):
        assert out[(r, "first")] == 2.0 or out[(r, "first")] == 1.0  # a cut plane was summed (or rank 0's own)
        res = out[(r, "second")]
        assert res[0] == "PeerLost", res
        assert res[1] < 15.0, res  # detected within the timeout, not after the group's 20 s
        assert out[(r, "dot")] == "PeerLost"
    assert elapsed < 60.0
