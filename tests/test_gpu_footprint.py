"""GPU parity of the separable-footprint projectors (ct_geometry_set_projector
SF-TR / SF-TT) with the FP64 oracle ``oracle.footprint``, through the C ABI:
A and A^T element by element, the adjoint identity, nnz, the solvers and
the preconditioner weights on top of them, and the combinations rejected."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import footprint as ofp
from oracle.solvers import cgls as ocgls, inv_sqrt_guarded, lsqr as olsqr, sirt as osirt

pytestmark = pytest.mark.gpu

# FP32 breakpoints: a projected edge |u| pixels from the detector centre is
# rounded by ~2^-24 |u| (plus the depth division), which moves footprint mass
# between neighbouring cells; the parity bar of the Siddon pair holds.
TOL = 1e-5

CASES = {
    "ragged": dict(nx=37, ny=29, nz=21, vx=1.1, vy=0.9, vz=1.3, nu=71, nv=45, du=1.0, dv=1.2,
                   sid=300.0, sdd=520.0, nviews=17),
    "offcentre": dict(nx=32, ny=24, nz=16, vx=1.0, vy=1.0, vz=1.0, nu=64, nv=33, du=0.8,
                      dv=0.8, sid=200.0, sdd=380.0, nviews=11, ox=14.0, oy=-9.0, oz=3.0,
                      det_off_u=3.3, det_off_v=-2.1),
    # coarse detector: footprints narrower than a cell; fine detector: wider
    # than the 8 cells a pass keeps in registers
    "coarse": dict(nx=20, ny=20, nz=12, vx=1.0, vy=1.0, vz=1.0, nu=13, nv=9, du=4.0, dv=4.0,
                   sid=150.0, sdd=250.0, nviews=7),
    "fine": dict(nx=10, ny=9, nz=8, vx=3.0, vy=3.0, vz=3.0, nu=150, nv=120, du=0.25, dv=0.3,
                 sid=100.0, sdd=180.0, nviews=5),
    # source 2.7 mm from the nearest voxel corner: in TT the projections of a
    # z face at the nearest and farthest depth spread wider than the voxel's
    # height, so neighbouring faces overlap (about half the voxel-views)
    "steep": dict(nx=8, ny=8, nz=24, vx=2.0, vy=2.0, vz=1.0, nu=40, nv=40, du=3.0, dv=3.0,
                  sid=14.0, sdd=30.0, nviews=5, det_off_u=0.7, det_off_v=-1.1),
}


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2110_13526_gb300 as m
    m.lib()
    return m


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


class SFOperator:
    """The oracle's SF pair behind the interface of oracle.solvers."""

    def __init__(self, g, kind):
        self.g, self.kind = g, kind

    def A(self, x):
        return ofp.project(self.g, x, self.kind)

    def AT(self, y):
        return ofp.backproject(self.g, y, self.kind)


@pytest.mark.parametrize("kind", ["sf_tr", "sf_tt"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_forward_backward_parity(ct, name, kind):
    cfg = CASES[name]
    g, og = ct.Geometry(**cfg, projector=kind), oracle.OGeom(**cfg)
    k = kind[3:]
    x = np.abs(synth.random_field(g.vol_shape, seed=50))
    p = ct.project(g, torch.from_numpy(x).cuda()).cpu().numpy()
    want = ofp.project(og, x, k)
    assert np.count_nonzero(want) > 0.3 * want.size
    assert rel(p, want) < TOL
    y = synth.random_field(g.sino_shape, seed=51)
    r = ct.backproject(g, torch.from_numpy(y).cuda()).cpu().numpy()
    assert rel(r, ofp.backproject(og, y, k)) < TOL
    # alpha / beta epilogues
    out = torch.from_numpy(synth.random_field(g.sino_shape, seed=52)).cuda()
    o0 = out.cpu().numpy()
    ct.project(g, torch.from_numpy(x).cuda(), out=out, alpha=-0.5, beta=2.0)
    assert rel(out.cpu().numpy(), -0.5 * want + 2.0 * o0) < TOL
    vo = torch.from_numpy(synth.random_field(g.vol_shape, seed=53)).cuda()
    v0 = vo.cpu().numpy()
    ct.backproject(g, torch.from_numpy(y).cuda(), out=vo, alpha=0.25, beta=-1.0)
    assert rel(vo.cpu().numpy(), 0.25 * ofp.backproject(og, y, k) - v0) < TOL


# degenerate sizes: one voxel, one slice (a single segment with one face pair
# per column), one detector row (most faces' ramps clipped off the detector)
DEGENERATE = {
    "single_voxel": dict(nx=1, ny=1, nz=1, vx=3.0, vy=3.0, vz=3.0, nu=5, nv=3, du=1.0, dv=1.0,
                         sid=50.0, sdd=90.0, nviews=4, angles=[0.1, 1.3, 2.9, 4.4]),
    "one_slice": dict(nx=12, ny=9, nz=1, vx=1.0, vy=1.1, vz=2.0, nu=20, nv=4, du=1.0, dv=1.0,
                      sid=60.0, sdd=100.0, nviews=5, det_off_v=0.3),
    "one_row": dict(nx=10, ny=10, nz=6, vx=1.0, vy=1.0, vz=1.0, nu=18, nv=1, du=1.2, dv=3.0,
                    sid=60.0, sdd=100.0, nviews=5, det_off_v=0.4),
}


@pytest.mark.parametrize("kind", ["sf_tr", "sf_tt"])
@pytest.mark.parametrize("name", sorted(DEGENERATE))
def test_degenerate_sizes(ct, name, kind):
    cfg = DEGENERATE[name]
    og = oracle.OGeom(**cfg)
    k = kind[3:]
    x = np.abs(synth.random_field((cfg["nz"], cfg["ny"], cfg["nx"]), seed=70))
    want = ofp.project(og, x, k)
    y = synth.random_field(want.shape, seed=71)
    want_r = ofp.backproject(og, y, k)
    for det in (False, True):
        g = ct.Geometry(**cfg, projector=kind, deterministic=det)
        assert rel(ct.project(g, torch.from_numpy(x).cuda()).cpu().numpy(), want) < TOL
        assert rel(ct.backproject(g, torch.from_numpy(y).cuda()).cpu().numpy(), want_r) < TOL


@pytest.mark.parametrize("kind", ["sf_tr", "sf_tt"])
def test_adjoint_nnz_and_norm(ct, kind):
    cfg = CASES["ragged"]
    g = ct.Geometry(**cfg, projector=kind)
    x = torch.from_numpy(synth.random_field(g.vol_shape, seed=54)).cuda()
    y = torch.from_numpy(synth.random_field(g.sino_shape, seed=55)).cuda()
    lhs = float((ct.project(g, x).double() * y.double()).sum())
    rhs = float((x.double() * ct.backproject(g, y).double()).sum())
    scale = float((ct.project(g, x.abs()).double() * y.double().abs()).sum())
    assert abs(lhs - rhs) <= 2e-6 * scale
    _, n2 = ct.project_norm2(g, x)
    assert float(n2) == pytest.approx(float((ct.project(g, x).double() ** 2).sum()), rel=1e-6)
    # nnz against the dense oracle matrix of a tiny case
    tiny = dict(nx=4, ny=3, nz=3, vx=1.0, vy=1.2, vz=0.9, nu=9, nv=7, du=0.8, dv=0.7,
                sid=30.0, sdd=50.0, nviews=3, angles=[0.2, 1.9, 4.0])
    gt = ct.Geometry(**tiny, projector=kind)
    M = ofp.dense_matrix(oracle.OGeom(**tiny), kind[3:])
    assert ct.count_nnz(gt) == int(np.count_nonzero(M))


@pytest.mark.parametrize("kind", ["sf_tr", "sf_tt"])
def test_solvers_and_weights_on_footprints(ct, kind):
    cfg = CASES["offcentre"]
    og = oracle.OGeom(**cfg)
    g = ct.Geometry(**cfg, projector=kind)
    op = SFOperator(og, kind[3:])
    x_true = synth.voxelize(synth.random_ellipsoids(5, 3, *synth.box_of(cfg),
                                                    axis_range=(3.0, 9.0)), cfg)
    b = op.A(x_true.astype(np.float64))
    b32 = b.astype(np.float32)
    bd = torch.from_numpy(b32).cuda()
    ref = ocgls(op, b32.astype(np.float64), K=10)
    x, rep = ct.cgls(g, bd, max_iter=10)
    assert rel(x.cpu().numpy(), ref.x) < 1e-4
    np.testing.assert_allclose(rep.history, ref.history, rtol=1e-4)
    ref = olsqr(op, b32.astype(np.float64), K=10)
    x, rep = ct.lsqr(g, bd, max_iter=10)
    assert rel(x.cpu().numpy(), ref.x) < 1e-4
    ref = osirt(op, b32.astype(np.float64), K=6, lam=1.5)
    x, rep = ct.sirt(g, bd, max_iter=6, relax=1.5)
    assert rel(x.cpu().numpy(), ref.x) < 1e-4
    # preconditioner weights R^-1/2, C^-1/2 with R = A 1, C = A^T 1.  A ray that
    # grazes a voxel corner has a tiny footprint sliver whose FP32 cell
    # integral carries a large relative error, magnified by the inverse square
    # root; the weights are compared where the sums are not tiny.
    wc, wr = ct.precond_weights(g, "rowcol")
    for w, sums in ((wr, op.A(np.ones(og.vol_shape))), (wc, op.AT(np.ones(og.sino_shape)))):
        ok = sums > 1e-3 * sums.max()
        assert ok.mean() > 0.5
        assert rel(w.cpu().numpy()[ok], inv_sqrt_guarded(sums)[ok]) < 1e-5
    x, _ = ct.cgls(g, bd, max_iter=8, precond="jacobi")
    assert torch.isfinite(x).all()


def test_rejected_combinations(ct):
    cfg = CASES["coarse"]
    g = ct.Geometry(**cfg, projector="sf_tt")
    bd = torch.zeros(g.sino_shape, device="cuda")
    with pytest.raises(RuntimeError, match="CT_ERR_INVALID_ARG"):
        ct.cgls(g, bd, max_iter=3, storage="bf16")
    with pytest.raises(RuntimeError, match="CT_ERR_INVALID_ARG"):
        ct.project(g, torch.zeros(g.vol_shape, device="cuda", dtype=torch.float16))
    assert ct.lib().ct_geometry_set_projector(g.handle, 7) == 1       # unknown projector
    # a volume reaching the source: the footprint's depth division is undefined
    with pytest.raises(RuntimeError, match="source circle"):
        ct.Geometry(**dict(cfg, sid=12.0, sdd=40.0), projector="sf_tt")


@pytest.mark.parametrize("kind", ["sf_tr", "sf_tt"])
@pytest.mark.parametrize("name", ["ragged", "fine"])
def test_deterministic_forward(ct, name, kind):
    """Deterministic mode sums the footprint forward projection in int64 fixed
    point: bitwise equal from call to call, within the parity bar of the
    oracle, and within FP32 rounding of the float-atomic sums.  Either order
    of setting the mode and the projector gives the same geometry."""
    cfg = CASES[name]
    og = oracle.OGeom(**cfg)
    gf = ct.Geometry(**cfg, projector=kind)
    gd = ct.Geometry(**cfg, projector=kind, deterministic=True)
    g2 = ct.Geometry(**cfg)
    assert ct.lib().ct_geometry_set_deterministic(g2.handle, 1) == 0
    assert ct.lib().ct_geometry_set_projector(g2.handle, ct.PROJECTORS[kind]) == 0
    k = kind[3:]
    x = synth.random_field(gd.vol_shape, seed=60)          # signed: sums cancel
    xd = torch.from_numpy(x).cuda()
    want = ofp.project(og, x.astype(np.float64), k)
    p1 = ct.project(gd, xd)
    for _ in range(3):
        assert torch.equal(ct.project(gd, xd), p1)
    assert torch.equal(ct.project(g2, xd), p1)
    assert rel(p1.cpu().numpy(), want) < TOL
    assert rel(p1.cpu().numpy(), ct.project(gf, xd).cpu().numpy()) < 1e-6
    # epilogue, the unit volume behind the row sums, the norm
    o0 = torch.from_numpy(synth.random_field(gd.sino_shape, seed=61)).cuda()
    out = o0.clone()
    ct.project(gd, xd, out=out, alpha=-0.5, beta=2.0)
    assert rel(out.cpu().numpy(), -0.5 * want + 2.0 * o0.cpu().numpy()) < TOL
    out2 = o0.clone()
    ct.project(gd, xd, out=out2, alpha=-0.5, beta=2.0)
    assert torch.equal(out, out2)
    wr, _ = ct.precond_weights(gd, "rowcol")
    wr2, _ = ct.precond_weights(gd, "rowcol")
    assert torch.equal(wr, wr2)
    p, n2 = ct.project_norm2(gd, xd)
    assert torch.equal(p, p1)
    assert float(n2) == float((p1.double() ** 2).sum()) or \
        float(n2) == pytest.approx(float((p1.double() ** 2).sum()), rel=1e-12)
    # the backprojection gathers in both modes: the same bits
    y = torch.from_numpy(synth.random_field(gd.sino_shape, seed=62)).cuda()
    assert torch.equal(ct.backproject(gd, y), ct.backproject(gf, y))


@pytest.mark.parametrize("precond", ["none", "rowcol"])
def test_deterministic_solvers_on_footprints(ct, precond):
    """CGLS, LSQR and a CGLS state resumed from bytes on a deterministic SF-TT
    geometry: bitwise equal between runs, and within the solver bar of the
    oracle."""
    cfg = CASES["offcentre"]
    og = oracle.OGeom(**cfg)
    g = ct.Geometry(**cfg, projector="sf_tt", deterministic=True)
    op = SFOperator(og, "tt")
    x_true = synth.voxelize(synth.random_ellipsoids(5, 3, *synth.box_of(cfg),
                                                    axis_range=(3.0, 9.0)), cfg)
    b32 = synth.gaussian_noise(op.A(x_true.astype(np.float64)), 0.01, seed=63).astype(np.float32)
    bd = torch.from_numpy(b32).cuda()
    x1, r1 = ct.cgls(g, bd, max_iter=10, precond=precond)
    x2, r2 = ct.cgls(g, bd, max_iter=10, precond=precond)
    assert torch.equal(x1, x2) and r1.history == r2.history
    if precond == "none":
        ref = ocgls(op, b32.astype(np.float64), K=10)
        assert rel(x1.cpu().numpy(), ref.x) < 1e-4
        np.testing.assert_allclose(r1.history, ref.history, rtol=1e-4)
    l1, _ = ct.lsqr(g, bd, max_iter=8, precond=precond)
    l2, _ = ct.lsqr(g, bd, max_iter=8, precond=precond)
    assert torch.equal(l1, l2)
    s = ct.CglsState(g)
    s.run(bd, 4, precond=precond)
    blob = s.to_bytes()
    s.close()
    s2 = ct.CglsState(g)
    s2.from_bytes(blob)
    x10, rep = s2.run(bd, 10, precond=precond)
    s2.close()
    assert torch.equal(x10, x1) and rep.history == r1.history
