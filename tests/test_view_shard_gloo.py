"""The view-sharded decomposition of Algorithm 1 on two gloo ranks (CPU).

Sharding the operator by views splits A into row blocks A_r (one per rank,
each a contiguous run of views): p_b = A d_x needs no exchange, r_x = A^T e_b
is the sum over ranks of A_r^T e_r (one volume all-reduce), and every norm
over the sinogram (||b||, ||p_b||^2, ||e_b||) is a sum of per-rank partial
sums (a scalar all-reduce).  Run that way on the FP64 oracle's operator,
CGLS must give the unsharded oracle's iterates and discrepancy history to
rounding.  This pins the exchange pattern a multi-GPU run would use; the
library itself runs one GPU per process and shards nothing (replicas)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

CFG = dict(nx=14, ny=12, nz=9, vx=1.0, vy=1.1, vz=1.2, nu=22, nv=16, du=1.0, dv=1.0,
           sid=120.0, sdd=200.0, nviews=11)
K = 8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def shard(nviews, rank, world):
    """Contiguous view block of one rank (the first nviews % world ranks take
    one view more)."""
    q, r = divmod(nviews, world)
    lo = rank * q + min(rank, r)
    return list(range(lo, lo + q + (1 if rank < r else 0)))


def _problem():
    import oracle
    import synth
    og = oracle.OGeom(**CFG)
    ells = synth.random_ellipsoids(4, 21, *synth.box_of(CFG), axis_range=(2.0, 6.0))
    x = synth.voxelize(ells, CFG).astype(np.float64)
    b = synth.gaussian_noise(oracle.project(og, x), 0.01, seed=22)
    return og, b


def _allsum(v):
    if np.ndim(v) == 0:
        t = torch.tensor([float(v)], dtype=torch.float64)
        dist.all_reduce(t)
        return float(t[0])
    t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def sharded_cgls(og, b, views, k_max):
    """Algorithm 1 with this rank's views; exchanges as in the module doc."""
    import oracle
    g = og.subset(views)
    br = b[views]
    A = lambda z: oracle.project(g, z)                       # p_r = A_r z, no exchange
    AT = lambda e: _allsum(oracle.backproject(g, e))         # sum_r A_r^T e_r
    nrm = lambda s: np.sqrt(_allsum(np.sum(s * s)))
    NB0 = nrm(br)
    e = br.copy()
    x = np.zeros(og.vol_shape)
    r = AT(e)
    d = r.copy()
    NR2_old = float(np.sum(r * r))                           # volume: same on every rank
    hist = []
    for i in range(k_max):
        if i > 0:
            r = AT(e)
            NR2_now = float(np.sum(r * r))
            d = r + (NR2_now / NR2_old) * d
            NR2_old = NR2_now
        p = A(d)
        alpha = NR2_old / _allsum(np.sum(p * p))
        x = x + alpha * d
        e = e - alpha * p
        hist.append(nrm(e) / NB0)
    return x, hist


def _worker(rank, world, port, out_x, out_h):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    og, b = _problem()
    x, hist = sharded_cgls(og, b, shard(og.nviews, rank, world), K)
    out_x[rank].copy_(torch.from_numpy(x.ravel()))
    out_h[rank].copy_(torch.tensor(hist, dtype=torch.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_covers_every_view_once():
    for n in (1, 7, 11, 360):
        for w in (1, 2, 3, 8):
            got = [v for r in range(w) for v in shard(n, r, w)]
            assert got == list(range(n))


def test_view_sharded_cgls_equals_unsharded_oracle():
    import oracle
    from oracle.solvers import cgls
    oracle.build()
    og, b = _problem()
    ref = cgls(oracle.Operator(og), b, K=K)
    world, port = 2, _free_port()
    n = CFG["nx"] * CFG["ny"] * CFG["nz"]
    out_x = torch.zeros(world, n, dtype=torch.float64).share_memory_()
    out_h = torch.zeros(world, K, dtype=torch.float64).share_memory_()
    mp.spawn(_worker, args=(world, port, out_x, out_h), nprocs=world, join=True)
    for r in range(world):
        np.testing.assert_allclose(out_x[r].numpy(), ref.x.ravel(), rtol=1e-9,
                                   atol=1e-12 * np.abs(ref.x).max())
        np.testing.assert_allclose(out_h[r].numpy(), ref.history, rtol=1e-9)
    assert torch.equal(out_x[0], out_x[1])
