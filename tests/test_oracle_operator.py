"""Pins of the FP64 Siddon oracle (A, A^T) against what mathematics fixes.

Each test checks the oracle against something other than itself: a brute
force by a different method, a closed form, a hand-built case, an invariant,
or the continuous line integral it discretises.
"""
import numpy as np
import pytest

import synth
from oracle import OGeom, backproject, count_nnz, project, ray_segments, segment_segments
from oracle.dense import dense_matrix
from oracle.ellipsoid import ray_integral


def tiny_geom(**kw):
    d = dict(nx=8, ny=8, nz=8, vx=1.0, vy=1.1, vz=0.9, nu=12, nv=10, du=1.3, dv=1.2,
             sid=40.0, sdd=70.0, nviews=3, angles=[0.3, 1.4, 2.9])
    d.update(kw)
    return OGeom(**d)


def box_chord(g, s, p):
    """Length of segment s->p inside the volume box: closed form, slab method."""
    lo = np.array([-g.nx * g.vx / 2 + g.ox, -g.ny * g.vy / 2 + g.oy, -g.nz * g.vz / 2 + g.oz])
    hi = lo + np.array([g.nx * g.vx, g.ny * g.vy, g.nz * g.vz])
    d = np.asarray(p) - np.asarray(s)
    t0, t1 = 0.0, 1.0
    for a in range(3):
        ta, tb = (lo[a] - s[a]) / d[a], (hi[a] - s[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(t1 - t0, 0.0) * np.linalg.norm(d)


@pytest.mark.parametrize("kw", [{}, dict(ox=1.7, oy=-0.6, oz=0.8),
                                dict(nx=5, ny=7, nz=6, det_off_u=0.4, det_off_v=-0.7)])
def test_dense_bruteforce_equals_siddon(oracle_lib, kw):
    """Dense A by per-voxel slab intersection == Siddon rows, entry by entry."""
    g = tiny_geom(**kw)
    A = dense_matrix(g)
    S = np.zeros_like(A)
    r = 0
    for view in range(g.nviews):
        for v in range(g.nv):
            for u in range(g.nu):
                idx, ln = ray_segments(g, view, u, v)
                np.add.at(S[r], idx, ln)
                r += 1
    scale = A.max()
    assert np.abs(S - A).max() <= 1e-12 * scale
    assert count_nnz(g) == int((A > 1e-12 * scale).sum())
    x = np.random.default_rng(0).standard_normal(g.vol_shape)
    y = np.random.default_rng(1).standard_normal(g.sino_shape)
    np.testing.assert_allclose(project(g, x).ravel(), A @ x.ravel(), rtol=0, atol=1e-12 * scale * 10)
    np.testing.assert_allclose(backproject(g, y).ravel(), A.T @ y.ravel(), rtol=0,
                               atol=1e-12 * scale * 10)


def test_constant_volume_is_box_chord(oracle_lib):
    """A 1 = the chord of each ray through the volume box."""
    g = OGeom(**synth.CONFIGS["PR1"]).subset([0, 7, 31, 52])
    b = project(g, np.ones(g.vol_shape))
    from oracle import ray_endpoints
    for view in range(g.nviews):
        for (u, v) in [(0, 0), (64, 48), (127, 95), (17, 80), (100, 3)]:
            s, p = ray_endpoints(g, view, u, v)
            assert b[view, v, u] == pytest.approx(box_chord(g, s, p), rel=1e-12, abs=1e-12)


def test_single_voxel_chords(oracle_lib):
    """Hand-computed chords through one cube of side 1 centred at the origin."""
    g = OGeom(nx=1, ny=1, nz=1, vx=1.0, vy=1.0, vz=1.0, nu=1, nv=1, du=1, dv=1,
              sid=10.0, sdd=20.0, nviews=1)
    cases = [((-2, -2, -2), (2, 2, 2), np.sqrt(3.0)),      # main diagonal
             ((-2, 0.1, 0.2), (2, 0.1, 0.2), 1.0),         # axis-parallel
             ((-2, 0.3, -2), (2, 0.3, 2), np.sqrt(2.0)),    # face diagonal
             ((-2, 0.7, 0.0), (2, 0.7, 0.0), 0.0),          # misses
             ((0.0, 0.0, -3.0), (0.0, 0.0, 0.25), 0.75)]   # ends inside
    for s, p, want in cases:
        idx, ln = segment_segments(g, s, p)
        assert ln.sum() == pytest.approx(want, rel=1e-13, abs=1e-13)
        assert all(i == 0 for i in idx)


def test_axis_aligned_ray_through_voxel_centres(oracle_lib):
    """A ray along x through voxel centres: A x = h_x * (sum along that row)."""
    g = OGeom(nx=5, ny=5, nz=5, vx=1.5, vy=1.0, vz=2.0, nu=1, nv=1, du=1, dv=1,
              sid=10.0, sdd=20.0, nviews=1)
    x = np.random.default_rng(3).standard_normal(g.vol_shape)
    for j, k in [(2, 2), (0, 4), (3, 1)]:
        y = (j - 2) * 1.0
        z = (k - 2) * 2.0
        idx, ln = segment_segments(g, (-20.0, y, z), (20.0, y, z))
        got = float(np.sum(ln * x.ravel()[idx]))
        assert got == pytest.approx(1.5 * x[k, j, :].sum(), rel=1e-13, abs=1e-13)
        assert len(idx) == 5


def test_tie_on_voxel_face_goes_to_upper_index(oracle_lib):
    """A ray lying in a y-plane between rows j = 1 and j = 2 is credited to j = 2."""
    g = OGeom(nx=4, ny=4, nz=4, vx=1.0, vy=1.0, vz=1.0, nu=1, nv=1, du=1, dv=1,
              sid=10.0, sdd=20.0, nviews=1)
    idx, ln = segment_segments(g, (-5.0, 0.0, 0.5), (5.0, 0.0, 0.5))
    j = (idx // 4) % 4
    assert np.all(j == 2) and ln.sum() == pytest.approx(4.0)


def test_geometry_orientation(oracle_lib):
    """Source at SID (cos, sin, 0), view rotation counter-clockwise about +z,
    detector centre ray through the isocentre."""
    from oracle import ray_endpoints
    g = OGeom(nx=1, ny=1, nz=1, vx=2.0, vy=2.0, vz=2.0, nu=3, nv=3, du=1.0, dv=1.0,
              sid=100.0, sdd=150.0, nviews=4)
    for view, (cx, cy) in enumerate([(1, 0), (0, 1), (-1, 0), (0, -1)]):
        s, p = ray_endpoints(g, view, 1, 1)
        np.testing.assert_allclose(s, [100 * cx, 100 * cy, 0], atol=1e-12)
        np.testing.assert_allclose(p, [-50 * cx, -50 * cy, 0], atol=1e-12)
        # the central ray crosses the 2 mm voxel at the isocentre straight through
        idx, ln = ray_segments(g, view, 1, 1)
        assert ln.sum() == pytest.approx(2.0, rel=1e-12)
    # u increases along e_u = (-sin, cos, 0), v along +z
    s, p = ray_endpoints(g, 0, 2, 0)
    np.testing.assert_allclose(p, [-50, 1.0, -1.0], atol=1e-12)
    # an off-centre volume shifted away from every ray is never hit
    g2 = OGeom(nx=2, ny=2, nz=2, vx=1.0, vy=1.0, vz=1.0, nu=3, nv=3, du=0.1, dv=0.1,
               sid=100.0, sdd=150.0, nviews=1, oy=5.0)
    assert np.all(project(g2, np.ones(g2.vol_shape)) == 0)


def test_adjoint_identity_pr1(oracle_lib):
    """<A x, y> = <x, A^T y> to 1e-12 relative (random signed x, y)."""
    g = OGeom(**synth.CONFIGS["PR1"])
    x = np.random.default_rng(5).standard_normal(g.vol_shape)
    y = np.random.default_rng(6).standard_normal(g.sino_shape)
    lhs = float(np.sum(project(g, x) * y))
    rhs = float(np.sum(x * backproject(g, y)))
    scale = float(np.sqrt(np.sum(project(g, np.abs(x)) * np.abs(y))))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs), scale)


def test_adjoint_identity_b256_sampled_views(oracle_lib):
    """Adjoint identity on 2 of the 8 sampled views of the 256^3 workload."""
    g = OGeom(**synth.CONFIGS["B256"]).subset([0, 135])
    x = np.random.default_rng(7).standard_normal(g.vol_shape)
    y = np.random.default_rng(8).standard_normal(g.sino_shape)
    lhs = float(np.sum(project(g, x) * y))
    rhs = float(np.sum(x * backproject(g, y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-9


def test_squared_length_backprojection_is_jacobi_diagonal(oracle_lib):
    """(A o A)^T 1 = diag(A^T A): column sums of squared dense entries."""
    g = tiny_geom()
    A = dense_matrix(g)
    D = backproject(g, np.ones(g.sino_shape), power=2)
    np.testing.assert_allclose(D.ravel(), (A * A).sum(axis=0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(D.ravel(), np.diag(A.T @ A), rtol=1e-12, atol=1e-12)


def test_ellipsoid_line_integrals_converge_under_refinement(oracle_lib):
    """A voxelise(E) -> analytic ray integral of E as h -> 0 (roughly O(h))."""
    ells = synth.random_ellipsoids(6, 4, [-32.0] * 3, [32.0] * 3, axis_range=(6.0, 20.0))
    errs = []
    for n in (16, 32, 64):
        h = 64.0 / n
        cfg = dict(nx=n, ny=n, nz=n, vx=h, vy=h, vz=h, nu=64, nv=48, du=2.0, dv=2.0,
                   sid=750.0, sdd=1200.0, nviews=6)
        g = OGeom(**cfg)
        vol = synth.voxelize(ells, cfg, dtype=np.float64)
        b = project(g, vol)
        rays = [(vw, u, v) for vw in range(6) for u in range(0, 64, 5) for v in range(0, 48, 5)]
        num = np.array([b[vw, v, u] for vw, u, v in rays])
        ana = np.array([ray_integral(g, ells, vw, u, v) for vw, u, v in rays])
        errs.append(np.linalg.norm(num - ana) / np.linalg.norm(ana))
    # measured: 0.112, 0.064, 0.025 (and 0.011 at 128^3)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.35 * errs[0] and errs[2] < 0.04


def test_sphere_voxelisation_volume():
    """Voxelised sphere: total mass -> 4/3 pi r^3 rho within voxelisation error."""
    e = synth.Ellipsoid(np.array([1.3, -0.4, 0.7]), np.array([9.0, 9.0, 9.0]), np.eye(3), 0.5)
    cfg = dict(nx=32, ny=32, nz=32, vx=1.0, vy=1.0, vz=1.0)
    vol = synth.voxelize([e], cfg, dtype=np.float64)
    want = 4.0 / 3.0 * np.pi * 9.0 ** 3 * 0.5
    assert vol.sum() == pytest.approx(want, rel=0.02)
    # additivity of overlapping ellipsoids
    e2 = synth.Ellipsoid(np.array([-3.0, 2.0, 0.0]), np.array([5.0, 7.0, 4.0]), np.eye(3), -0.25)
    both = synth.voxelize([e, e2], cfg, dtype=np.float64)
    np.testing.assert_allclose(both, vol + synth.voxelize([e2], cfg, dtype=np.float64), atol=1e-12)


def test_nnz_pr1_matches_dense_count_scaling(oracle_lib):
    """nnz(A) of the 64^3 workload: about 68 nonzeros per ray (7.29e7 in total)."""
    g = OGeom(**synth.CONFIGS["PR1"])
    n = count_nnz(g)
    assert 7.0e7 < n < 7.6e7
