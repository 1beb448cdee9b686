"""Pins of the separable-footprint (SF) oracle, ``oracle.footprint``.

The paper's results use Long et al.'s TT footprint projector, which it names
but does not write out; the oracle restates it (module doc there).  These
tests pin that restatement to something other than itself: the exact
cell-averaged chord of a voxel, computed here by brute force (every detector
cell sampled by a grid of rays, each ray clipped against the voxel box).

* In the parallel-beam limit the separable footprint is exact: a square
  voxel's transaxial projection is exactly the trapezoid of its corner
  projections with the centre chord as height, and the axial one a
  rectangle, so SF-TR and SF-TT equal the brute force at any view angle and
  detector offset (up to the 5e-6 magnification left at SID = 1e7 mm).
* In a steep cone beam SF is an approximation: the measured error against
  the brute force is 2.7 % (TT) and 5.4 % (TR) at worst, and TT is the more
  accurate, which is why it is the default.
* In a steep cone the separable footprint of every voxel equals, to
  rounding, the one rebuilt here by another route: the detector point of
  each of the voxel's eight corners found by intersecting the ray from the
  source with the detector plane in 3-D; the transaxial breakpoints the
  corners' u, the TT axial breakpoints the v of the bottom and top faces
  seen at the nearest and farthest vertical edge (depth along the central
  ray), the TR ones those faces at the centre's depth; each cell's average
  integrated piece by piece (exact for a piecewise-linear profile); the
  amplitude the centre ray clipped against the voxel's x and y slabs.  A
  slip in any factor (a breakpoint at the wrong depth, a swapped face, a
  mis-signed offset) fails it exactly, where the brute-force bound above
  could let it through.
* A and A^T use the same entries (adjoint to rounding); ``project`` equals
  the dense matrix; the footprint of a voxel carries its volume in the
  parallel limit; mirroring the volume in z mirrors every view in v.
"""
import numpy as np
import pytest

from oracle import OGeom
from oracle import footprint as fp


def chord(s, p, lo, hi):
    """Length of the segment s -> p inside the box [lo, hi] (slab clipping)."""
    d = p - s
    t0 = np.zeros(d.shape[:-1])
    t1 = np.ones(d.shape[:-1])
    for a in range(3):
        da = d[..., a]
        with np.errstate(divide="ignore", invalid="ignore"):
            ta, tb = (lo[a] - s[a]) / da, (hi[a] - s[a]) / da
        par = da == 0
        t0 = np.maximum(t0, np.where(par, -np.inf, np.minimum(ta, tb)))
        t1 = np.minimum(t1, np.where(par, np.inf, np.maximum(ta, tb)))
        if lo[a] > s[a] or hi[a] < s[a]:
            t1 = np.where(par, -1.0, t1)
    return np.maximum(t1 - t0, 0.0) * np.linalg.norm(d, axis=-1)


def brute(g, view, j, S):
    """Cell-averaged chord of voxel j in every detector cell of one view."""
    th = g.angle_array()[view]
    ct, st = np.cos(th), np.sin(th)
    s = np.array([g.sid * ct, g.sid * st, 0.0])
    eu, ev = np.array([-st, ct, 0.0]), np.array([0.0, 0.0, 1.0])
    c = -(g.sdd - g.sid) * np.array([ct, st, 0.0])
    k, jj, i = np.unravel_index(j, g.vol_shape)
    cen = np.array([(i - 0.5 * (g.nx - 1)) * g.vx + g.ox, (jj - 0.5 * (g.ny - 1)) * g.vy + g.oy,
                    (k - 0.5 * (g.nz - 1)) * g.vz + g.oz])
    h = np.array([g.vx, g.vy, g.vz])
    out = np.zeros((g.nv, g.nu))
    sub = (np.arange(S) + 0.5) / S - 0.5
    for l in range(g.nv):
        for u in range(g.nu):
            uu = (u + sub - 0.5 * (g.nu - 1)) * g.du + g.det_off_u
            vv = (l + sub - 0.5 * (g.nv - 1)) * g.dv + g.det_off_v
            U, V = np.meshgrid(uu, vv)
            P = c + U[..., None] * eu + V[..., None] * ev
            out[l, u] = chord(s, P, cen - h / 2, cen + h / 2).mean()
    return out


@pytest.mark.parametrize("kind", ["tr", "tt"])
@pytest.mark.parametrize("angle,off", [(0.0, 0.0), (0.0, 1.0), (np.pi / 4, 0.0), (0.3, 0.37),
                                       (2.2, -0.61)])
def test_parallel_limit_is_exact(kind, angle, off):
    g = OGeom(nx=1, ny=1, nz=1, vx=2.0, vy=2.0, vz=2.0, nu=5, nv=3, du=2.0, dv=2.0,
              sid=1e7, sdd=1e7 + 50.0, nviews=1, angles=[angle], det_off_u=off)
    a = fp.project(g, np.ones((1, 1, 1)), kind)[0]
    b = brute(g, 0, 0, S=400)
    assert np.abs(a - b).max() < 2e-5 * b.max()
    # the footprint carries the voxel volume (magnification 1 + 5e-6)
    assert a.sum() * g.du * g.dv == pytest.approx(8.0, rel=2e-5)


def test_cone_beam_approximation_and_tt_beats_tr():
    g = OGeom(nx=3, ny=3, nz=3, vx=2.0, vy=2.0, vz=2.0, nu=24, nv=24, du=0.6, dv=0.6,
              sid=30.0, sdd=60.0, nviews=3, angles=[0.2, 1.1, 2.5])
    errs = {"tr": [], "tt": []}
    for v in range(3):
        gv = g.subset([v])
        for j in (0, 4, 13, 26):
            b = brute(gv, 0, j, S=60)
            e = np.zeros(27)
            e[j] = 1.0
            for kind in errs:
                a = fp.project(gv, e.reshape(3, 3, 3), kind)[0]
                errs[kind].append(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert max(errs["tt"]) < 0.04 and max(errs["tr"]) < 0.08
    assert np.mean(errs["tt"]) < np.mean(errs["tr"])


@pytest.mark.parametrize("kind", ["tr", "tt"])
def test_adjoint_and_dense(kind):
    g = OGeom(nx=5, ny=4, nz=3, vx=1.1, vy=0.9, vz=1.3, nu=9, nv=7, du=1.2, dv=1.4,
              sid=40.0, sdd=70.0, nviews=4, angles=[0.1, 0.8, 2.0, 4.4], ox=0.7, oz=-0.4,
              det_off_u=0.3)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(g.vol_shape)
    y = rng.standard_normal(g.sino_shape)
    ax, aty = fp.project(g, x, kind), fp.backproject(g, y, kind)
    assert abs(np.sum(ax * y) - np.sum(x * aty)) < 1e-12 * np.sum(np.abs(ax) * np.abs(y))
    M = fp.dense_matrix(g, kind)
    np.testing.assert_allclose(M @ x.ravel(), ax.ravel(), rtol=1e-12, atol=1e-12)
    assert np.count_nonzero(M) > 0 and np.all(M >= 0)


def _frame(g, th):
    ct, st = np.cos(th), np.sin(th)
    s = np.array([g.sid * ct, g.sid * st, 0.0])
    n = np.array([-ct, -st, 0.0])                        # central ray direction
    c = s + g.sdd * n                                    # detector centre
    return s, n, c, np.array([-st, ct, 0.0]), np.array([0.0, 0.0, 1.0])


def _hit(g, th, q):
    """Pixel-index (u, v) where the ray from the source through q meets the
    detector plane, and the depth of q along the central ray."""
    s, n, c, eu, ev = _frame(g, th)
    d = q - s
    lam = np.dot(c - s, n) / np.dot(d, n)
    p = s + lam * d - c
    u = (np.dot(p, eu) - g.det_off_u) / g.du + 0.5 * (g.nu - 1)
    v = (np.dot(p, ev) - g.det_off_v) / g.dv + 0.5 * (g.nv - 1)
    return u, v, np.dot(d, n)


def _piece_avg(b, k):
    """Integral over [k - 1/2, k + 1/2] of the unit trapezoid with breakpoints
    b[0] <= .. <= b[3]: split at the breakpoints, trapezoid rule on each
    linear piece."""
    def f(x, m):                                         # the piece containing m, at x
        if m < b[0] or m >= b[3]:
            return 0.0
        if m < b[1]:
            return (x - b[0]) / (b[1] - b[0])
        if m < b[2]:
            return 1.0
        return (b[3] - x) / (b[3] - b[2])
    pts = sorted({k - 0.5, k + 0.5, *[t for t in b if k - 0.5 < t < k + 0.5]})
    tot = 0.0
    for p, q in zip(pts[:-1], pts[1:]):
        m = 0.5 * (p + q)
        tot += 0.5 * (q - p) * (f(p, m) + f(q, m))
    return tot


def rebuilt_footprint(g, th, i, j, k, kind):
    """A_ij of voxel (i, j, k) in every cell of view th, from the corners."""
    cen = np.array([(i - 0.5 * (g.nx - 1)) * g.vx + g.ox, (j - 0.5 * (g.ny - 1)) * g.vy + g.oy,
                    (k - 0.5 * (g.nz - 1)) * g.vz + g.oz])
    h = np.array([g.vx, g.vy, g.vz]) / 2
    edges = []                                           # per vertical edge: (u, depth, v_bot, v_top)
    for sx in (-1, 1):
        for sy in (-1, 1):
            lo = cen + h * np.array([sx, sy, -1])
            hi = cen + h * np.array([sx, sy, 1])
            u0, vb, t0 = _hit(g, th, lo)
            u1, vt, t1 = _hit(g, th, hi)
            assert abs(u0 - u1) < 1e-9 and abs(t0 - t1) < 1e-9
            edges.append((u0, t0, vb, vt))
    bu = sorted(e[0] for e in edges)
    if kind == "tt":
        near = min(edges, key=lambda e: e[1])
        far = max(edges, key=lambda e: e[1])
        bv = sorted([near[2], near[3], far[2], far[3]])
    else:
        _, vlo, _ = _hit(g, th, cen - np.array([0.0, 0.0, h[2]]))
        _, vhi, _ = _hit(g, th, cen + np.array([0.0, 0.0, h[2]]))
        bv = [min(vlo, vhi)] * 2 + [max(vlo, vhi)] * 2
    # amplitude: the line source -> centre inside the voxel's x and y slabs
    s = _frame(g, th)[0]
    d = cen - s
    t0, t1 = -np.inf, np.inf
    for a in (0, 1):
        if d[a] != 0:
            ta, tb = (cen[a] - h[a] - s[a]) / d[a], (cen[a] + h[a] - s[a]) / d[a]
            t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    amp = (t1 - t0) * np.linalg.norm(d)
    fu = np.array([_piece_avg(bu, c) for c in range(g.nu)])
    fv = np.array([_piece_avg(bv, r) for r in range(g.nv)])
    return amp * np.outer(fv, fu)


@pytest.mark.parametrize("kind", ["tr", "tt"])
def test_cone_beam_footprint_equals_corner_rebuild(kind):
    # steep cone (SID 3.5 voxel pitches from the far corner), anisotropic
    # voxels, every offset set, views on all four sides and on diagonals
    g = OGeom(nx=4, ny=3, nz=5, vx=1.7, vy=1.1, vz=1.4, nu=40, nv=46, du=0.55, dv=0.6,
              sid=9.0, sdd=21.0, nviews=6, angles=[0.15, 0.785398, 1.9, 3.3, 4.1, 5.6],
              ox=0.6, oy=-0.35, oz=0.9, det_off_u=0.8, det_off_v=-1.1)
    rng = np.random.default_rng(7)
    n = g.nx * g.ny * g.nz
    for jv in rng.choice(n, size=12, replace=False):
        e = np.zeros(n)
        e[jv] = 1.0
        got = fp.project(g, e.reshape(g.vol_shape), kind)
        k, j, i = np.unravel_index(jv, g.vol_shape)
        for vi, th in enumerate(g.angle_array()):
            want = rebuilt_footprint(g, th, i, j, k, kind)
            assert want.max() > 0
            np.testing.assert_allclose(got[vi], want, rtol=1e-10, atol=1e-12 * want.max())


@pytest.mark.parametrize("kind", ["tr", "tt"])
def test_z_mirror_symmetry(kind):
    """Mirroring the volume in z (centred, no z offset, centred rows) mirrors
    every view's projection in v, for any transaxial placement."""
    g = OGeom(nx=5, ny=4, nz=6, vx=1.2, vy=0.8, vz=1.1, nu=21, nv=17, du=0.9, dv=1.0,
              sid=14.0, sdd=30.0, nviews=5, angles=[0.3, 1.2, 2.0, 3.9, 5.1], ox=0.4,
              oy=-0.7, det_off_u=0.35)
    x = np.random.default_rng(3).random(g.vol_shape)
    a = fp.project(g, x, kind)
    b = fp.project(g, x[::-1], kind)
    np.testing.assert_allclose(b, a[:, ::-1, :], rtol=1e-12, atol=1e-12 * a.max())
