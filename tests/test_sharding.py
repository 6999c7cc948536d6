"""The operator pair shards with no exchange of partial results: H over transducers (each rank
writes its own rows of u) and H^T over z-slabs of the volume (each rank gathers, for its own
nodes, every transducer's samples).  Checked with two gloo ranks on the CPU, each computing its
share with the FP64 oracle; gathered, the shares equal the unsharded operators.  FBP and the
spherical-voxel pair shard the same way (FBP and H_sph^T over node slabs, H_sph over
transducers).  (The GPU build runs replicas only: every box has one GPU.)"""
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


def _rank_other(rank, world, port, out):
    """FBP and the spherical-voxel pair sharded the same way: FBP and H_sph^T over z-slabs of the
    nodes (every transducer's data), H_sph over transducers (its own rows)."""
    import torch.distributed as dist
    from oracle import fbp as F
    from oracle import sph as S
    from paper_1304_2017_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    geom = _geom()
    rng = np.random.default_rng(6)
    p = rng.standard_normal(geom.data_shape)
    w = F.arc_weights(geom.positions_mm, 2, 3)
    alpha = W.random_volume(geom, seed=7).astype(np.float64)
    freqs = 0.25 * (np.arange(12) + 1)
    u = rng.standard_normal((geom.n_transducers, 12)) + 1j * rng.standard_normal((geom.n_transducers, 12))
    z0, z1 = geom.nz * rank // world, geom.nz * (rank + 1) // world
    nodes = np.array([(ix, iy, iz) for iz in range(z0, z1) for iy in range(geom.ny) for ix in range(geom.nx)])
    qs = list(range(rank, geom.n_transducers, world))
    part = (qs, (z0, z1), F.fbp(geom, p, w, nodes=nodes), S.H_sph(geom, alpha, freqs, qs=qs),
            S.H_sph_t(geom, u, freqs, nodes=nodes))
    parts = [None] * world
    dist.all_gather_object(parts, part)
    if rank == 0:
        fb = np.zeros(geom.vol_shape)
        us = np.zeros((geom.n_transducers, 12), complex)
        at = np.zeros(geom.vol_shape)
        for q_r, (s0, s1), f_r, u_r, a_r in parts:
            fb[s0:s1] = f_r.reshape(s1 - s0, geom.ny, geom.nx)
            us[q_r] = u_r
            at[s0:s1] = a_r.reshape(s1 - s0, geom.ny, geom.nx)
        f_ref = F.fbp(geom, p, w)
        u_ref = S.H_sph(geom, alpha, freqs)
        a_ref = S.H_sph_t(geom, u, freqs)
        out["fbp"] = float(np.abs(fb - f_ref).max() / np.abs(f_ref).max())
        out["sph"] = float(np.abs(us - u_ref).max() / np.abs(u_ref).max())
        out["spht"] = float(np.abs(at - a_ref).max() / np.abs(a_ref).max())
    dist.destroy_process_group()


def test_sharded_fbp_and_spherical_voxel_model_equal_unsharded():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_other, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    assert out["fbp"] <= 1e-12 and out["sph"] <= 1e-12 and out["spht"] <= 1e-12, dict(out)
