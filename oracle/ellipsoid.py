"""Closed-form line integrals of ellipsoid phantoms (test infrastructure only).

For an ellipsoid {p : ||S^-1 R^T (p - c)|| <= 1} of density rho, the ray
r(t) = s + t (p - s) maps to q(t) = q0 + t w with q0 = S^-1 R^T (s - c) and
w = S^-1 R^T (p - s).  Its chord is where ||q0 + t w||^2 <= 1, a quadratic
in t.  The integral of the phantom along the ray, restricted to the volume
box and to t in [0, 1], is rho * L * |[t1, t2] n [t_box_in, t_box_out]|.
This is the continuous counterpart of A x for a voxelised phantom, so A
applied to finer and finer voxelisations must converge to it.
"""
from __future__ import annotations

import numpy as np

from . import OGeom, ray_endpoints


def _box_interval(g: OGeom, s, d):
    lo = np.array([-0.5 * g.nx * g.vx + g.ox, -0.5 * g.ny * g.vy + g.oy,
                   -0.5 * g.nz * g.vz + g.oz])
    hi = lo + np.array([g.nx * g.vx, g.ny * g.vy, g.nz * g.vz])
    t0, t1 = 0.0, 1.0
    for a in range(3):
        if d[a] != 0:
            ta, tb = (lo[a] - s[a]) / d[a], (hi[a] - s[a]) / d[a]
            t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
        elif not (lo[a] <= s[a] < hi[a]):
            return 0.0, 0.0
    return t0, t1


def ray_integral(g: OGeom, ells, view: int, u: int, v: int, clip_to_box: bool = True) -> float:
    """Integral of the additive ellipsoid phantom along detector ray (view, u, v)."""
    s, p = ray_endpoints(g, view, u, v)
    d = p - s
    L = float(np.linalg.norm(d))
    tb0, tb1 = _box_interval(g, s, d) if clip_to_box else (0.0, 1.0)
    if tb1 <= tb0:
        return 0.0
    total = 0.0
    for e in ells:
        Minv = (np.asarray(e.rot) / np.asarray(e.semi_axes)[None, :]).T
        q0 = Minv @ (s - np.asarray(e.center))
        w = Minv @ d
        a = float(w @ w)
        b = 2.0 * float(q0 @ w)
        c = float(q0 @ q0) - 1.0
        disc = b * b - 4 * a * c
        if disc <= 0:
            continue
        sq = np.sqrt(disc)
        t1, t2 = (-b - sq) / (2 * a), (-b + sq) / (2 * a)
        lo, hi = max(t1, tb0), min(t2, tb1)
        if hi > lo:
            total += e.rho * (hi - lo) * L
    return total
