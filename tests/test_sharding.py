"""The operator pair shards with no exchange of partial results: H over transducers (each rank
writes its own rows of u) and H^T over z-slabs of the volume (each rank gathers, for its own
nodes, every transducer's samples).  Checked with two gloo ranks on the CPU, each computing its
share with the FP64 oracle; gathered, the shares equal the unsharded operators.  (The GPU build
runs replicas only: every box has one GPU.)"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _geom():
    from paper_1304_2017_gb300 import workloads as W
    return W.make_geometry((9, 8, 10), 0.35, 2, 3, 6.0, 48)


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    from paper_1304_2017_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    geom = _geom()
    alpha = W.spheres_phantom(geom, 2, seed=3) + 0.1 * W.random_volume(geom, seed=4)
    y = W.random_data(geom, seed=5).astype(np.float64)
    # H: transducers q = rank, rank + world, ...
    qs = list(range(rank, geom.n_transducers, world))
    u_part = oracle.H(geom.subset(qs), alpha)
    # H^T: z-slab [z0, z1) of the nodes, from D^T y of all transducers
    z0, z1 = geom.nz * rank // world, geom.nz * (rank + 1) // world
    nodes = [(ix, iy, iz) for iz in range(z0, z1) for iy in range(geom.ny) for ix in range(geom.nx)]
    a_part = oracle.Gt_nodes(geom, oracle.Dt(geom, y), nodes)
    parts = [None] * world
    dist.all_gather_object(parts, (qs, u_part, (z0, z1), a_part))
    if rank == 0:
        u = np.zeros(geom.data_shape)
        a = np.zeros(geom.vol_shape)
        for q_r, u_r, (s0, s1), a_r in parts:
            u[q_r] = u_r
            a[s0:s1] = a_r.reshape(s1 - s0, geom.ny, geom.nx)
        u_ref = oracle.H(geom, alpha)
        a_ref = oracle.Ht(geom, y)
        out["H"] = float(np.abs(u - u_ref).max() / np.abs(u_ref).max())
        out["Ht"] = float(np.abs(a - a_ref).max() / np.abs(a_ref).max())
    dist.destroy_process_group()


def test_sharded_operators_equal_unsharded():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    assert out["H"] <= 1e-12 and out["Ht"] <= 1e-12, dict(out)
