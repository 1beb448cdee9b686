"""Batched CGLS (ct_batch): several solves advanced in lock step, the
projectors of all column-major Siddon jobs in one persistent launch per
operator.  Each job must give what ct_cgls gives alone: bitwise with
fixed-point backprojection, and within the solver bar (1e-4 relative L2 of
the iterate after k updates) of the FP64 oracle otherwise."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.solvers import cgls as ocgls

pytestmark = pytest.mark.gpu

TOL_X = 1e-4

# column-major geometries of different sizes (tiles of several grids in one
# launch, ragged tails), one off-centre, and one whose rays advance mostly
# along z (ray-major kernels: launched on its own inside the batched step)
GEOMS = {
    "small": dict(nx=30, ny=26, nz=18, vx=1.0, vy=1.0, vz=1.2, nu=44, nv=28, du=1.0, dv=1.0,
                  sid=250.0, sdd=400.0, nviews=24),
    "ragged": dict(nx=37, ny=29, nz=21, vx=1.1, vy=0.9, vz=1.3, nu=71, nv=45, du=1.0, dv=1.2,
                   sid=300.0, sdd=520.0, nviews=17),
    "offcentre": dict(nx=32, ny=24, nz=16, vx=1.0, vy=1.0, vz=1.0, nu=64, nv=33, du=0.8,
                      dv=0.8, sid=200.0, sdd=380.0, nviews=11, ox=14.0, oy=-9.0, oz=3.0,
                      det_off_u=3.3, det_off_v=-2.1),
    "bigcone": dict(nx=16, ny=16, nz=40, vx=1.0, vy=1.0, vz=1.0, nu=24, nv=70, du=1.5, dv=2.5,
                    sid=30.0, sdd=60.0, nviews=5),
}


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2110_13526_gb300 as m
    m.lib()
    oracle.build()
    return m


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def problem(name, seed):
    cfg = GEOMS[name]
    og = oracle.OGeom(**cfg)
    lo, hi = synth.box_of(cfg)
    ells = synth.random_ellipsoids(5, seed, lo, hi, axis_range=(2.0, 8.0))
    x = synth.voxelize(ells, cfg)
    b = synth.gaussian_noise(oracle.project(og, x.astype(np.float64)), 0.01, seed=seed)
    return cfg, og, b.astype(np.float32)


@pytest.fixture(scope="module")
def problems():
    return {name: problem(name, k + 3) for k, name in enumerate(GEOMS)}


# (geometry, max_iter, err_tol, precond, tikhonov, step at which it joins)
JOBS = [("small", 12, 0.0, "none", 0.0, 0), ("ragged", 7, 0.0, "rowcol", 0.0, 0),
        ("offcentre", 30, 0.1, "none", 0.0, 0), ("bigcone", 6, 0.0, "jacobi", 0.0, 2),
        ("small", 9, 0.0, "none", 0.3, 3), ("ragged", 10, 0.0, "none", 0.0, 5)]


def run_batch(ct, problems, jobs, deterministic):
    geoms = {}
    for name, *_ in jobs:
        if name not in geoms:
            geoms[name] = ct.Geometry(**GEOMS[name], deterministic=deterministic)
    bt = ct.Batch()
    ids, results, step = {}, {}, 0
    pending = list(enumerate(jobs))
    while pending or any(k not in results for k in ids):
        for k, (name, K, err, pc, lam, at) in list(pending):
            if at <= step:
                b = torch.from_numpy(problems[name][2]).cuda()
                ids[k] = bt.add(geoms[name], b, max_iter=K, err_tol=err, precond=pc,
                                tikhonov=lam)
                pending.remove((k, (name, K, err, pc, lam, at)))
        for k, jid in ids.items():
            if k not in results and bt.done(jid):
                results[k] = bt.result(jid)
        if pending or any(k not in results for k in ids):
            bt.step()
            step += 1
        assert step < 100
    bt.close()
    return geoms, results


def test_batch_bitwise_equals_solo_deterministic(ct, problems):
    geoms, res = run_batch(ct, problems, JOBS, deterministic=True)
    for k, (name, K, err, pc, lam, _) in enumerate(JOBS):
        b = torch.from_numpy(problems[name][2]).cuda()
        xs, rs = ct.cgls(geoms[name], b, max_iter=K, err_tol=err, precond=pc, tikhonov=lam)
        xb, rb = res[k]
        assert rb.iterations == rs.iterations, (name, rb.iterations, rs.iterations)
        assert torch.equal(xb, xs), (name, (xb - xs).abs().max().item())
        assert rb.history == rs.history
        assert (rb.nb0, rb.nb) == (rs.nb0, rs.nb)
        assert (rb.n_forward, rb.n_back) == (rs.n_forward, rs.n_back)
    # the tolerance-stopped job stopped early, the others ran to max_iter
    assert res[2][1].iterations < 30
    assert [res[k][1].iterations for k in (0, 1, 3, 4, 5)] == [12, 7, 6, 9, 10]


def test_batch_float_parity_with_oracle(ct, problems):
    """Float-atomic backprojection: each batched job within 1e-4 of the FP64
    oracle's CGLS after K updates."""
    jobs = [("small", 10, 0.0, "none", 0.0, 0), ("ragged", 8, 0.0, "none", 0.0, 0),
            ("offcentre", 6, 0.0, "none", 0.0, 1)]
    _, res = run_batch(ct, problems, jobs, deterministic=False)
    for k, (name, K, *_rest) in enumerate(jobs):
        cfg, og, b = problems[name]
        ref = ocgls(oracle.Operator(og), b.astype(np.float64), K=K)
        x, r = res[k]
        assert r.iterations == K
        assert rel(x.cpu().numpy(), ref.x) < TOL_X, name
        np.testing.assert_allclose(r.history, ref.history, rtol=TOL_X)


def test_batch_launches_one_projector_kernel_per_operator(ct, problems):
    """N column-major jobs share one A^T and one A launch per step: a step of
    N jobs launches 2 (N - 1) fewer kernels than N steps of one job."""
    g = ct.Geometry(**GEOMS["small"])
    b = torch.from_numpy(problems["small"][2]).cuda()

    def per_step(n):
        bt = ct.Batch()
        for _ in range(n):
            bt.add(g, b, max_iter=50)
        bt.step()                      # captures the step's graph
        torch.cuda.synchronize()
        k0 = ct.kernel_launches()
        for _ in range(3):
            bt.step()
        torch.cuda.synchronize()
        k = (ct.kernel_launches() - k0) / 3
        bt.close()
        return k

    one, three = per_step(1), per_step(3)
    assert three == 3 * one - 2 * 2, (one, three)


def test_batch_footprint_and_errors(ct, problems):
    cfg = GEOMS["small"]
    gs = ct.Geometry(**cfg, projector="sf_tt")
    g = ct.Geometry(**cfg)
    b = torch.from_numpy(problems["small"][2]).cuda()
    # a footprint job runs its own projectors inside the batched step
    bs = ct.project(gs, torch.from_numpy(synth.voxelize(
        synth.random_ellipsoids(4, 9, *synth.box_of(cfg), axis_range=(2.0, 8.0)), cfg)).cuda())
    bt = ct.Batch()
    j1 = bt.add(gs, bs, max_iter=6)
    j2 = bt.add(g, b, max_iter=4)
    while bt.step():
        pass
    x1, r1 = bt.result(j1)
    x2, r2 = bt.result(j2)
    xs1, rs1 = ct.cgls(gs, bs, max_iter=6)
    assert r1.iterations == 6 and r2.iterations == 4
    assert rel(x1.cpu().numpy(), xs1.cpu().numpy()) < 1e-4
    np.testing.assert_allclose(r1.history, rs1.history, rtol=1e-4)
    # options a batch does not take (BF16 storage), unknown ids, removal of a
    # running job
    x = torch.zeros(g.vol_shape, device="cuda")
    bad = ct.SolverOpts(4, 0.0, 0, 0.0, 0, 0, 1)
    jid = ctypes.c_int32()
    with pytest.raises(ct.CTError):
        ct._check(ct.lib().ct_batch_add_cgls(bt.handle, g.handle, ct._ptr(b), ct._ptr(x),
                                             ctypes.byref(bad), ctypes.byref(jid)))
    with pytest.raises(ct.CTError):
        bt.done(12345)
    j3 = bt.add(g, b, max_iter=20)
    bt.step()
    bt.remove(j3)
    assert bt.step() == 0
    bt.close()
