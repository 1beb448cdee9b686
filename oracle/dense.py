"""Brute-force dense system matrix A for tiny problems (test infrastructure only).

A third, independent way to get A_ij = length of ray i inside voxel j: for
every (ray, voxel) pair intersect the segment source -> pixel centre with the
voxel's cube by the slab method and take the length of the overlap.  No plane
crossings are enumerated, nothing is sorted, there is no midpoint rule.  Used
only as a pin for the Siddon oracle on volumes of at most a few hundred voxels.
"""
from __future__ import annotations

import numpy as np

from . import OGeom, ray_endpoints


def segment_box_length(s, p, lo, hi):
    """Length of segment s->p inside the boxes [lo, hi] (lo, hi: (n, 3))."""
    s = np.asarray(s, dtype=np.float64)
    d = np.asarray(p, dtype=np.float64) - s
    L = float(np.linalg.norm(d))
    t0 = np.zeros(lo.shape[0])
    t1 = np.ones(lo.shape[0])
    for a in range(3):
        if d[a] != 0.0:
            ta = (lo[:, a] - s[a]) / d[a]
            tb = (hi[:, a] - s[a]) / d[a]
            t0 = np.maximum(t0, np.minimum(ta, tb))
            t1 = np.minimum(t1, np.maximum(ta, tb))
        else:
            inside = (s[a] >= lo[:, a]) & (s[a] < hi[:, a])
            t1 = np.where(inside, t1, -np.inf)
    return np.maximum(t1 - t0, 0.0) * L


def voxel_boxes(g: OGeom):
    """Lower and upper corners of every voxel, in storage order (z, y, x)."""
    k, j, i = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    h = np.array([g.vx, g.vy, g.vz])
    lo0 = np.array([-0.5 * g.nx * g.vx + g.ox, -0.5 * g.ny * g.vy + g.oy,
                    -0.5 * g.nz * g.vz + g.oz])
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    lo = lo0 + ijk * h
    return lo, lo + h


def dense_matrix(g: OGeom) -> np.ndarray:
    """A as an (nviews*nv*nu, nz*ny*nx) FP64 array."""
    nvox = g.nx * g.ny * g.nz
    if nvox * g.nviews * g.nu * g.nv > 5e7:
        raise ValueError("dense A is for tiny problems only")
    lo, hi = voxel_boxes(g)
    A = np.zeros((g.nviews * g.nv * g.nu, nvox))
    r = 0
    for view in range(g.nviews):
        for v in range(g.nv):
            for u in range(g.nu):
                s, p = ray_endpoints(g, view, u, v)
                A[r] = segment_box_length(s, p, lo, hi)
                r += 1
    return A
