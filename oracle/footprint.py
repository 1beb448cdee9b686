"""FP64 oracle of the separable-footprint projector (test infrastructure only).

The paper computes its results with the "TT" footprint projector of Long,
Fessler and Balter (2010), named in Materials and Methods but not written out
there.  This module restates that method as read here (the reading is the
one the CUDA library implements; neither side imports the other):

For voxel j (centre c_j, pitch hx, hy, hz) and view theta, with the
conventions of ``OGeom`` (source s = SID (cos th, sin th, 0), flat detector
at depth SDD along the central ray, e_u = (-sin th, cos th, 0), e_v = z):

* a point P projects to detector coordinates a = SDD (P - s).e_u / t(P),
  b = SDD P_z / t(P), with the depth t(P) = (P - s).(-cos th, -sin th, 0);
  in pixel-index units u = (a - det_off_u) / du + (nu - 1) / 2, likewise v.
* transaxial footprint F_u: the trapezoid of unit height whose breakpoints
  are the sorted projections u of the voxel's four vertical edges (the
  projection does not depend on z);
* axial footprint F_v: "TR" -- the unit rectangle between the projections of
  the two z faces at the depth of the voxel centre; "TT" -- the trapezoid
  whose breakpoints are the sorted projections of the two z faces at the
  smallest and the largest depth of the voxel's corners;
* amplitude (Long et al.'s first method): the chord of the ray through the
  voxel centre across the voxel's x and y faces,
  l_j = min(hx / |d_x|, hy / |d_y|) for the unit direction d from the source
  to c_j (for hx = hy this is the transaxial chord divided by the cosine of
  the ray's elevation);
* detector cells average the footprint:
  A_ij = l_j * Fbar_u(k) * Fbar_v(l), Fbar(k) = integral of F over
  [k - 1/2, k + 1/2] (pixel-index units, cell width 1).

A^T uses the same entries, so the pair is exactly adjoint.
"""
from __future__ import annotations

import numpy as np

KINDS = ("tr", "tt")


def _trap_integral(t0, t1, t2, t3, x):
    """Integral from -inf to x of the unit-height trapezoid t0<=t1<=t2<=t3."""
    x = np.asarray(x, dtype=np.float64)
    r = np.zeros(np.broadcast(t0, x).shape)
    w01 = t1 - t0
    w23 = t3 - t2
    rise = 0.5 * w01                                     # area of the rising ramp
    flat = t2 - t1
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(w01 > 0, (x - t0) ** 2 / (2 * np.where(w01 > 0, w01, 1.0)), 0.0)
        c = np.where(w23 > 0, (t3 - x) ** 2 / (2 * np.where(w23 > 0, w23, 1.0)), 0.0)
    r = np.where(x <= t0, 0.0, r)
    r = np.where((x > t0) & (x <= t1), a, r)
    r = np.where((x > t1) & (x <= t2), rise + (x - t1), r)
    r = np.where((x > t2) & (x <= t3), rise + flat + 0.5 * w23 - c, r)
    r = np.where(x > t3, rise + flat + 0.5 * w23, r)
    return r


def _cell_avg(t0, t1, t2, t3, k):
    """Fbar(k): the trapezoid integrated over the cell [k - 1/2, k + 1/2]."""
    return _trap_integral(t0, t1, t2, t3, k + 0.5) - _trap_integral(t0, t1, t2, t3, k - 0.5)


def _view_terms(g, th, kind):
    """Per-voxel footprints of one view: (tau[4, ny, nx], vb[4, nz, ny, nx], amp[nz, ny, nx])."""
    ct, st = np.cos(th), np.sin(th)
    s = np.array([g.sid * ct, g.sid * st, 0.0])
    eu = np.array([-st, ct, 0.0])
    ec = np.array([-ct, -st, 0.0])
    xs = (np.arange(g.nx) - 0.5 * (g.nx - 1)) * g.vx + g.ox
    ys = (np.arange(g.ny) - 0.5 * (g.ny - 1)) * g.vy + g.oy
    zs = (np.arange(g.nz) - 0.5 * (g.nz - 1)) * g.vz + g.oz
    X, Y = np.meshgrid(xs, ys)                           # [ny, nx]

    def u_of(px, py):
        rel = np.stack([px - s[0], py - s[1]])
        t = rel[0] * ec[0] + rel[1] * ec[1]
        a = g.sdd * (rel[0] * eu[0] + rel[1] * eu[1]) / t
        return (a - g.det_off_u) / g.du + 0.5 * (g.nu - 1), t

    corners = [(X + sx * 0.5 * g.vx, Y + sy * 0.5 * g.vy) for sx in (-1, 1) for sy in (-1, 1)]
    us, ts = zip(*[u_of(cx, cy) for cx, cy in corners])
    tau = np.sort(np.stack(us), axis=0)                  # [4, ny, nx]
    tmin, tmax = np.min(np.stack(ts), axis=0), np.max(np.stack(ts), axis=0)
    _, tc = u_of(X, Y)

    def v_of(z, t):
        return (g.sdd * z / t - g.det_off_v) / g.dv + 0.5 * (g.nv - 1)

    Z = zs[:, None, None]
    zlo, zhi = Z - 0.5 * g.vz, Z + 0.5 * g.vz
    if kind == "tr":
        vlo, vhi = v_of(zlo, tc[None]), v_of(zhi, tc[None])
        lo, hi = np.minimum(vlo, vhi), np.maximum(vlo, vhi)
        vb = np.stack([lo, lo, hi, hi])                  # a rectangle as a trapezoid
    elif kind == "tt":
        vb = np.sort(np.stack([v_of(zlo, tmin[None]), v_of(zlo, tmax[None]),
                               v_of(zhi, tmin[None]), v_of(zhi, tmax[None])]), axis=0)
    else:
        raise ValueError("kind must be 'tr' or 'tt'")
    # amplitude: chord through the centre across the x and y faces
    dx, dy = X - s[0], Y - s[1]
    dz = Z - s[2]
    nrm = np.sqrt(dx[None] ** 2 + dy[None] ** 2 + dz ** 2)
    with np.errstate(divide="ignore"):
        lx = np.where(dx[None] != 0, g.vx * nrm / np.abs(dx[None]), np.inf)
        ly = np.where(dy[None] != 0, g.vy * nrm / np.abs(dy[None]), np.inf)
    amp = np.minimum(lx, ly)
    return tau, vb, amp


def _cells(b0, b3, n):
    """First cell overlapping [b0, b3] and the largest number of cells any voxel spans."""
    k0 = np.floor(b0 + 0.5).astype(np.int64)
    k1 = np.floor(b3 + 0.5).astype(np.int64)
    w = int(np.max(k1 - k0)) + 1 if k0.size else 0
    return k0, w


def _apply(g, kind, x=None, y=None):
    if kind not in KINDS:
        raise ValueError("kind must be 'tr' or 'tt'")
    ang = g.angle_array()
    forward = y is None
    out = np.zeros(g.sino_shape if forward else g.vol_shape)
    for vi, th in enumerate(ang):
        tau, vb, amp = _view_terms(g, th, kind)
        ku0, wu = _cells(tau[0], tau[3], g.nu)
        kv0, wv = _cells(vb[0], vb[3], g.nv)
        shape3 = amp.shape
        for du_ in range(wu):
            ku = ku0 + du_                                # [ny, nx]
            fu = _cell_avg(tau[0], tau[1], tau[2], tau[3], ku)
            ok_u = (ku >= 0) & (ku < g.nu) & (fu != 0)
            for dv_ in range(wv):
                kv = kv0 + dv_                            # [nz, ny, nx]
                fv = _cell_avg(vb[0], vb[1], vb[2], vb[3], kv)
                ok = ok_u[None] & (kv >= 0) & (kv < g.nv) & (fv != 0)
                if not np.any(ok):
                    continue
                a = amp * fu[None] * fv                   # A_ij of these (voxel, cell) pairs
                kuu = np.broadcast_to(ku[None], shape3)[ok]
                kvv = kv[ok]
                if forward:
                    np.add.at(out[vi], (kvv, kuu), (a * x)[ok])
                else:
                    out[ok] += a[ok] * y[vi][kvv, kuu]
    return out


def project(g, vol, kind: str = "tt") -> np.ndarray:
    """b = A_SF x, FP64.  vol: (nz, ny, nx) -> (nviews, nv, nu)."""
    x = np.asarray(vol, dtype=np.float64).reshape(g.vol_shape)
    return _apply(g, kind, x=x)


def backproject(g, sino, kind: str = "tt") -> np.ndarray:
    """x = A_SF^T b, FP64 (the same entries as ``project``)."""
    y = np.asarray(sino, dtype=np.float64).reshape(g.sino_shape)
    return _apply(g, kind, y=y)


def dense_matrix(g, kind: str = "tt") -> np.ndarray:
    """A_SF as a dense (rays x voxels) matrix, column by column (tiny cases)."""
    n = g.nx * g.ny * g.nz
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(project(g, e.reshape(g.vol_shape), kind).ravel())
    return np.stack(cols, axis=1)
