"""GPU parity of the projector pair (ct_project / ct_backproject) with the FP64
oracle, through the C ABI.  Tolerance: 1e-5 relative L2 for FP32 projections
and backprojections at every volume size (crossing positions are exact
integer-line positions good to about 2^-23 voxel, and the FP32 sums of a few
hundred terms per ray, or a few hundred per voxel and view, stay near 1e-6)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2110_13526_gb300 as m
    m.lib()                      # raises if the CUDA library is missing
    oracle.build()
    return m


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


CASES = {
    # ragged tails in u, v, volume; anisotropic voxels; many tiles
    "ragged": dict(nx=37, ny=29, nz=21, vx=1.1, vy=0.9, vz=1.3, nu=71, nv=45, du=1.0, dv=1.2,
                   sid=300.0, sdd=520.0, nviews=17),
    # off-centre volume and shifted detector (Software section: off-centre reconstruction)
    "offcentre": dict(nx=32, ny=24, nz=16, vx=1.0, vy=1.0, vz=1.0, nu=64, nv=33, du=0.8,
                      dv=0.8, sid=200.0, sdd=380.0, nviews=11, ox=14.0, oy=-9.0, oz=3.0,
                      det_off_u=3.3, det_off_v=-2.1),
    # huge cone angle: rays that advance mostly along z
    "bigcone": dict(nx=16, ny=16, nz=40, vx=1.0, vy=1.0, vz=1.0, nu=24, nv=70, du=1.5, dv=2.5,
                    sid=30.0, sdd=60.0, nviews=5),
    # views exactly on the axes and diagonals (dominance ties, rays parallel to
    # grid planes).  Odd sizes put those rays through voxel centres: a ray lying
    # exactly IN a voxel-boundary plane is ill-posed (the side it is credited to
    # depends on the last bit of sin/cos) and is not a parity case.
    "axes": dict(nx=21, ny=21, nz=11, vx=1.0, vy=1.0, vz=1.0, nu=33, nv=9, du=1.0, dv=1.0,
                 sid=150.0, sdd=250.0, nviews=8),
    # detector rows under a voxel high (A^T pairs row blocks, a warp taking
    # every other row) with three row blocks: one pair, one unpaired, and a
    # ragged last column block
    "pairs": dict(nx=40, ny=36, nz=30, vx=1.0, vy=1.0, vz=1.0, nu=50, nv=90, du=0.9, dv=0.9,
                  sid=260.0, sdd=450.0, nviews=9),
    # single voxel and a one-pixel detector
    "tiny": dict(nx=1, ny=1, nz=1, vx=3.0, vy=3.0, vz=3.0, nu=5, nv=3, du=1.0, dv=1.0,
                 sid=50.0, sdd=90.0, nviews=4, angles=[0.1, 1.3, 2.9, 4.4]),
    # one slice and one detector row: column-major warps with a single ray
    "slice_row": dict(nx=24, ny=17, nz=1, vx=1.0, vy=1.2, vz=2.0, nu=40, nv=1, du=1.0, dv=1.5,
                      sid=80.0, sdd=140.0, nviews=7),
    # one slice under a cone whose outer rows advance mostly along z (the
    # ray-major kernels): only the rows near the source's height reach it
    "slice_cone": dict(nx=20, ny=18, nz=1, vx=1.0, vy=1.0, vz=3.0, nu=30, nv=60, du=1.5,
                       dv=2.5, sid=30.0, sdd=60.0, nviews=5, det_off_v=0.37),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_forward_parity(ct, name):
    cfg = CASES[name]
    g, og = ct.Geometry(**cfg), oracle.OGeom(**cfg)
    x = synth.random_field(g.vol_shape, seed=10)
    p = ct.project(g, torch.from_numpy(x).cuda()).cpu().numpy()
    want = oracle.project(og, x.astype(np.float64))
    assert rel(p, want) < TOL
    # alpha/beta epilogue; beta = 0 must not read the (NaN-filled) output
    out = torch.full(g.sino_shape, float("nan"), device="cuda")
    ct.project(g, torch.from_numpy(x).cuda(), out=out, alpha=2.0, beta=0.0)
    assert rel(out.cpu().numpy(), 2 * want) < TOL
    y0 = synth.random_field(g.sino_shape, seed=11)
    out = torch.from_numpy(y0).cuda()
    ct.project(g, torch.from_numpy(x).cuda(), out=out, alpha=-0.5, beta=1.5)
    assert rel(out.cpu().numpy(), -0.5 * want + 1.5 * y0) < TOL


@pytest.mark.parametrize("name", sorted(CASES))
def test_backward_parity(ct, name):
    cfg = CASES[name]
    g, og = ct.Geometry(**cfg), oracle.OGeom(**cfg)
    y = synth.random_field(g.sino_shape, seed=12)
    r = ct.backproject(g, torch.from_numpy(y).cuda()).cpu().numpy()
    want = oracle.backproject(og, y.astype(np.float64))
    assert rel(r, want) < TOL
    x0 = synth.random_field(g.vol_shape, seed=13)
    out = torch.from_numpy(x0).cuda()
    ct.backproject(g, torch.from_numpy(y).cuda(), out=out, alpha=0.25, beta=-1.0)
    assert rel(out.cpu().numpy(), 0.25 * want - x0) < TOL


def test_adjoint_identity_gpu(ct):
    cfg = CASES["ragged"]
    g = ct.Geometry(**cfg)
    x = torch.from_numpy(synth.random_field(g.vol_shape, seed=14)).cuda()
    y = torch.from_numpy(synth.random_field(g.sino_shape, seed=15)).cuda()
    ax = ct.project(g, x).double()
    aty = ct.backproject(g, y).double()
    lhs = float((ax * y.double()).sum())
    rhs = float((x.double() * aty).sum())
    scale = float((ct.project(g, x.abs()).double() * y.double().abs()).sum())
    assert abs(lhs - rhs) <= 2e-6 * scale


def test_pr1_full_parity(ct):
    cfg = synth.CONFIGS["PR1"]
    g, og = ct.Geometry(**cfg), oracle.OGeom(**cfg)
    x = synth.voxelize(synth.nested_phantom(64.0, seed=0), cfg)
    p = ct.project(g, torch.from_numpy(x).cuda()).cpu().numpy()
    want = oracle.project(og, x.astype(np.float64))
    assert rel(p, want) < TOL
    y = synth.random_field(g.sino_shape, seed=16)
    r = ct.backproject(g, torch.from_numpy(y).cuda()).cpu().numpy()
    assert rel(r, oracle.backproject(og, y.astype(np.float64))) < TOL


def test_b256_sampled_views(ct):
    """256^3 workload in the bench's launch configuration: full A on the GPU,
    8 sampled views {0, 45, ..., 315} against the oracle; A^T of a sinogram
    that is nonzero on those 8 views only."""
    cfg = synth.CONFIGS["B256"]
    g = ct.Geometry(**cfg)
    views = [0, 45, 90, 135, 180, 225, 270, 315]
    og = oracle.OGeom(**cfg).subset(views)
    lo, hi = synth.box_of(cfg)
    x = synth.voxelize(synth.random_ellipsoids(40, 1, lo, hi), cfg)
    p = ct.project(g, torch.from_numpy(x).cuda())
    want = oracle.project(og, x.astype(np.float64))
    got = p[views].cpu().numpy()
    assert rel(got, want) < TOL
    y = np.zeros(g.sino_shape, dtype=np.float32)
    ys = synth.random_field((len(views), cfg["nv"], cfg["nu"]), seed=17)
    y[views] = ys
    r = ct.backproject(g, torch.from_numpy(y).cuda()).cpu().numpy()
    assert rel(r, oracle.backproject(og, ys.astype(np.float64))) < TOL


def test_p512_sampled_views(ct):
    """512^3 precision workload (0.5 mm voxels, 768 x 576 detector of 0.75 mm
    pixels, 720 views) in the bench's launch configuration (all views in one
    launch group): A of the phantom and A^T of a signed sinogram against the
    oracle on the 16 views k * 720 / 16, both at 1e-5.  Voxels here lie up to
    256 from the centre, where FP32 crossings relative to the centre lose
    2^-24 * 256 of a voxel."""
    cfg = synth.CONFIGS["P512"]
    g = ct.Geometry(**cfg)
    views = [int(round(k * cfg["nviews"] / 16)) % cfg["nviews"] for k in range(16)]
    og = oracle.OGeom(**cfg).subset(views)
    lo, hi = synth.box_of(cfg)
    x = synth.voxelize(synth.random_ellipsoids(40, 2, lo, hi), cfg)
    p = ct.project(g, torch.from_numpy(x).cuda())[views].cpu().numpy()
    assert rel(p, oracle.project(og, x.astype(np.float64))) < TOL
    del p
    ys = synth.random_field((len(views), cfg["nv"], cfg["nu"]), seed=42)
    y = torch.zeros(g.sino_shape, device="cuda")
    y[views] = torch.from_numpy(ys).cuda()
    r = ct.backproject(g, y).cpu().numpy()
    del y
    assert rel(r, oracle.backproject(og, ys.astype(np.float64))) < TOL


# Launch orders of the projector grid.  "wide": the volume and its transposed
# copy take more than 160 MB, so A visits all 20 views together and A^T groups
# of 16 (one full group and one of 4 with 12 idle views).  "tall": 4097 row
# blocks leave room for 15 view groups in the grid's 65535 z blocks, so the 23
# views go in groups of 2 (the last one holding a single view).
ORDER_CASES = {
    "wide": dict(nx=256, ny=256, nz=400, vx=1.0, vy=1.0, vz=1.0, nu=64, nv=48, du=8.0,
                 dv=14.0, sid=750.0, sdd=1200.0, nviews=20),
    "tall": dict(nx=12, ny=10, nz=9, vx=1.0, vy=1.0, vz=1.0, nu=3, nv=8 * 4096 + 5, du=8.0,
                 dv=0.0005, sid=100.0, sdd=160.0, nviews=23),
}


@pytest.mark.parametrize("name", sorted(ORDER_CASES))
def test_launch_orders(ct, name):
    cfg = ORDER_CASES[name]
    g, og = ct.Geometry(**cfg), oracle.OGeom(**cfg)
    # non-negative, like attenuation: a signed field summed along rays of up
    # to 500 voxels cancels to a small fraction of its terms, which would
    # magnify the FP32 rounding of the sums beyond the parity bar
    x = np.abs(synth.random_field(g.vol_shape, seed=40))
    p = ct.project(g, torch.from_numpy(x).cuda()).cpu().numpy()
    want = oracle.project(og, x.astype(np.float64))
    assert np.count_nonzero(want) > 0.5 * want.size
    assert rel(p, want) < TOL
    y = synth.random_field(g.sino_shape, seed=41)
    r = ct.backproject(g, torch.from_numpy(y).cuda()).cpu().numpy()
    # z runs to +-200 voxels from the centre here: crossings are exact
    # integer-line positions, so A^T keeps the same bar as A (with crossings
    # computed in FP32 from the volume centre this case measured 1.57e-5)
    assert rel(r, oracle.backproject(og, y.astype(np.float64))) < TOL
    # the norm partials (one per CTA, idle CTAs included) sum to ||A x||^2
    xs = torch.from_numpy(x).cuda()
    _, n2 = ct.project_norm2(g, xs)
    assert float(n2) == pytest.approx(float((want ** 2).sum()), rel=2 * TOL)


def test_count_nnz_matches_oracle(ct):
    """Counts agree to 1e-3: a segment shorter than the resolution of a
    crossing position (2^-23 of a slab) may be counted on one side only.
    Where a ray crosses two grid planes at exactly the same point (a tie,
    frequent in a symmetric geometry's axis-aligned views), FP64 sees one
    crossing and the two independently rounded integer lines may leave a
    sliver of about 1e-7 mm: a real entry of the kernels' matrix, far below
    parity, but not a count the oracle can match.  The large-cone case
    therefore runs with its detector shifted off the symmetric position."""
    cone = dict(CASES["bigcone"], det_off_u=0.137, det_off_v=0.291)
    for cfg in (CASES["ragged"], cone, synth.CONFIGS["PR1"]):
        g, og = ct.Geometry(**cfg), oracle.OGeom(**cfg)
        n_gpu, n_ref = ct.count_nnz(g), oracle.count_nnz(og)
        assert abs(n_gpu - n_ref) <= max(2, 1e-3 * n_ref)


def test_project_norm2_is_fp64_and_deterministic(ct):
    cfg = CASES["ragged"]
    g = ct.Geometry(**cfg)
    x = torch.from_numpy(synth.random_field(g.vol_shape, seed=18)).cuda()
    out, n1 = ct.project_norm2(g, x)
    want = float((out.double() ** 2).sum())
    assert float(n1) == pytest.approx(want, rel=1e-12)
    _, n2 = ct.project_norm2(g, x)
    assert float(n1) == float(n2)


def test_empty_and_missing(ct):
    # no views: nothing to do, no error
    g = ct.Geometry(nx=4, ny=4, nz=4, vx=1, vy=1, vz=1, nu=8, nv=8, du=1, dv=1, sid=50,
                    sdd=80, nviews=0)
    v = torch.ones(g.vol_shape, device="cuda")
    s = ct.project(g, v)
    assert s.numel() == 0
    r = ct.backproject(g, s)
    assert float(r.abs().sum()) == 0.0
    assert ct.count_nnz(g) == 0
    # a volume placed where no ray passes projects to exact zeros
    g2 = ct.Geometry(nx=4, ny=4, nz=4, vx=1, vy=1, vz=1, nu=6, nv=6, du=0.1, dv=0.1, sid=50,
                     sdd=80, nviews=3, oz=30.0)
    assert float(ct.project(g2, v).abs().sum()) == 0.0


@pytest.mark.parametrize("bad", [dict(nv=65535 * 8 + 1), dict(nviews=65536), dict(nz=65536),
                                 dict(sdd=40.0), dict(du=0.0)])
def test_geometry_limits_rejected(ct, bad):
    cfg = dict(nx=4, ny=4, nz=4, vx=1, vy=1, vz=1, nu=8, nv=8, du=1, dv=1, sid=50, sdd=80,
               nviews=2)
    cfg.update(bad)
    with pytest.raises(RuntimeError, match="CT_ERR_INVALID_ARG"):
        ct.Geometry(**cfg)


def test_host_tensors_round_trip(ct):
    cfg = CASES["offcentre"]
    g = ct.Geometry(**cfg)
    x = torch.from_numpy(synth.random_field(g.vol_shape, seed=19))
    p_host = ct.project(g, x)
    assert p_host.device.type == "cpu"
    p_dev = ct.project(g, x.cuda()).cpu()
    assert torch.equal(p_host, p_dev)


@pytest.mark.parametrize("name", ["ragged", "offcentre", "bigcone", "pairs", "slice_row", "slice_cone"])
def test_deterministic_backprojection(ct, name):
    """Fixed-point accumulation: bitwise repeatable, same parity bar."""
    cfg = CASES[name]
    g, og = ct.Geometry(**cfg, deterministic=True), oracle.OGeom(**cfg)
    y = torch.from_numpy(synth.random_field(g.sino_shape, seed=20)).cuda()
    r1 = ct.backproject(g, y)
    r2 = ct.backproject(g, y)
    assert torch.equal(r1, r2)
    want = oracle.backproject(og, y.cpu().double().numpy())
    assert rel(r1.cpu().numpy(), want) < TOL
    x0 = torch.from_numpy(synth.random_field(g.vol_shape, seed=21)).cuda()
    out = x0.clone()
    ct.backproject(g, y, out=out, alpha=0.25, beta=-1.0)
    assert rel(out.cpu().numpy(), 0.25 * want - x0.cpu().numpy()) < TOL


@pytest.mark.parametrize("n,nz", [(128, 256), (192, 384)])
def test_ray_major_parity_at_scale(ct, n, nz):
    """A geometry whose top and bottom rows advance mostly along z takes the
    ray-major kernels.  Their exact integer lines keep the error flat in the
    volume's extent (measured A 1.2e-7 -> 2.1e-7 and A^T 3.2e-7 -> 3.6e-7
    from 64 to 256 z-slices); the FP32 walk they replaced grew to 9.0e-6 at
    256 slices and would have passed 1e-5 at about 280."""
    cfg = dict(nx=n, ny=n, nz=nz, vx=1.0, vy=1.0, vz=1.0, nu=int(1.6 * n), nv=int(3.2 * nz),
               du=1.0, dv=1.0, sid=1.2 * n, sdd=2.0 * n, nviews=6,
               angles=[0.13, 0.9, 1.7, 2.6, 3.9, 5.2])
    g, og = ct.Geometry(**cfg), oracle.OGeom(**cfg)
    x = np.abs(synth.random_field(g.vol_shape, seed=3))
    y = synth.random_field(g.sino_shape, seed=4)
    p = ct.project(g, torch.from_numpy(x).cuda()).cpu().numpy()
    r = ct.backproject(g, torch.from_numpy(y).cuda()).cpu().numpy()
    assert rel(p, oracle.project(og, x.astype(np.float64))) < 2e-6
    assert rel(r, oracle.backproject(og, y.astype(np.float64))) < 2e-6
