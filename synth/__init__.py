"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module generates inputs only: workload shapes, ellipsoid phantoms, their
voxelisation and measurement noise.  It holds none of the operator's or the
solvers' arithmetic, and neither the CUDA library nor the oracle imports it.

Workloads (the paper's own phantom and detector size are not all stated; the
numbers below are the synthetic stand-ins, with the paper's geometry class:
C-arm-like circular orbit, SID 750 mm, SDD 1200 mm, Results section):

* ``PR1``  -- 64^3 voxels of 1 mm, 128 x 96 detector of 1 mm pixels,
  90 views over 360 degrees; a seeded 10-ellipsoid nested phantom that stands
  in for the 3D Shepp-Logan phantom; b = A x + N(0, (0.01 max b)^2).
* ``B256`` -- 256^3 voxels of 1 mm, 384 x 288 detector of 1 mm pixels,
  360 views; 40 random ellipsoids (seed 1).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Sequence

import numpy as np

CONFIGS: Dict[str, dict] = {
    "PR1": dict(nx=64, ny=64, nz=64, vx=1.0, vy=1.0, vz=1.0, nu=128, nv=96, du=1.0, dv=1.0,
                sid=750.0, sdd=1200.0, nviews=90),
    "B256": dict(nx=256, ny=256, nz=256, vx=1.0, vy=1.0, vz=1.0, nu=384, nv=288, du=1.0,
                 dv=1.0, sid=750.0, sdd=1200.0, nviews=360),
    "P512": dict(nx=512, ny=512, nz=512, vx=0.5, vy=0.5, vz=0.5, nu=768, nv=576, du=0.75,
                 dv=0.75, sid=750.0, sdd=1200.0, nviews=720),
    # the differentiation workload: one geometry for a batch of 8 volumes
    "DIFF": dict(nx=128, ny=128, nz=128, vx=1.0, vy=1.0, vz=1.0, nu=192, nv=144, du=1.6,
                 dv=1.6, sid=750.0, sdd=1200.0, nviews=180),
}


@dataclass
class Ellipsoid:
    """Indicator of {p : ||S^-1 R^T (p - c)|| <= 1} times ``rho`` (mm, additive)."""
    center: np.ndarray      # (3,)
    semi_axes: np.ndarray   # (3,)
    rot: np.ndarray         # (3, 3), columns = the ellipsoid's axes in world frame
    rho: float


def _quat_to_rot(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def random_ellipsoids(n: int, seed: int, box_lo, box_hi, axis_range=(5.0, 60.0),
                      rho_range=(0.1, 1.0), axis_scale: float = 1.0) -> List[Ellipsoid]:
    """Random-ellipsoid phantom.

    numpy ``default_rng(seed)`` (PCG64); per ellipsoid, in this order: three
    semi-axes U[axis_range] (times ``axis_scale``), a rotation from a uniform
    random unit quaternion (four standard normals, normalised), a centre
    uniform in the volume box shrunk by 25 % of its extent on every side, and
    a density U[rho_range].
    """
    rng = np.random.default_rng(seed)
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    ext = hi - lo
    out = []
    for _ in range(n):
        ax = rng.uniform(axis_range[0], axis_range[1], size=3) * axis_scale
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        c = rng.uniform(lo + 0.25 * ext, hi - 0.25 * ext)
        rho = rng.uniform(rho_range[0], rho_range[1])
        out.append(Ellipsoid(c, ax, _quat_to_rot(q), float(rho)))
    return out


def nested_phantom(extent_mm: float = 64.0, seed: int = 0) -> List[Ellipsoid]:
    """Ten-ellipsoid nested head-like phantom (a stand-in, not Shepp-Logan's table).

    An outer shell (density 1), an inner body that lowers the interior to 0.2,
    and eight small seeded features of density in [-0.2, 0.3] inside the body.
    Values are additive, so the volume holds values in roughly [0, 1.3].
    """
    r = extent_mm / 2.0
    eye = np.eye(3)
    out = [Ellipsoid(np.zeros(3), np.array([0.69, 0.92, 0.81]) * r * 0.95, eye, 1.0),
           Ellipsoid(np.array([0.0, -0.0184 * r, 0.0]),
                     np.array([0.6624, 0.874, 0.78]) * r * 0.95, eye, -0.8)]
    rng = np.random.default_rng(seed)
    for _ in range(8):
        c = rng.uniform(-0.4, 0.4, size=3) * r
        ax = rng.uniform(0.05, 0.25, size=3) * r
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        rho = rng.uniform(-0.2, 0.3)
        out.append(Ellipsoid(c, ax, _quat_to_rot(q), float(rho)))
    return out


def box_of(cfg: dict):
    """Volume box (lo, hi) in mm of a config dict (centred, optional offsets)."""
    n = np.array([cfg["nx"], cfg["ny"], cfg["nz"]], dtype=np.float64)
    h = np.array([cfg["vx"], cfg["vy"], cfg["vz"]], dtype=np.float64)
    o = np.array([cfg.get("ox", 0.0), cfg.get("oy", 0.0), cfg.get("oz", 0.0)])
    lo = -0.5 * n * h + o
    return lo, lo + n * h


def voxelize(ells: Sequence[Ellipsoid], cfg: dict, supersample: int = 2,
             dtype=np.float32) -> np.ndarray:
    """Mean of the phantom over ``supersample^3`` points per voxel.

    With supersample = 2 the points sit at +-h/4 from the voxel centre on every
    axis.  Returns (nz, ny, nx).  Work is confined to each ellipsoid's bounding
    box.
    """
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    h = np.array([cfg["vx"], cfg["vy"], cfg["vz"]], dtype=np.float64)
    lo, _ = box_of(cfg)
    ss = int(supersample)
    offs = (np.arange(ss) + 0.5) / ss - 0.5          # in voxel units, +-1/4 for ss = 2
    acc = np.zeros((nz, ny, nx), dtype=np.float64)
    n = np.array([nx, ny, nz])
    for e in ells:
        M = (e.rot / e.semi_axes[None, :]).T          # p -> S^-1 R^T p
        half = np.sqrt(((e.rot * e.semi_axes[None, :]) ** 2).sum(axis=1))
        i0 = np.maximum(np.floor((e.center - half - lo) / h).astype(int) - 1, 0)
        i1 = np.minimum(np.ceil((e.center + half - lo) / h).astype(int) + 1, n)
        if np.any(i1 <= i0):
            continue
        xs = lo[0] + (np.arange(i0[0], i1[0])[None, :] + 0.5 + offs[:, None]) * h[0]
        ys = lo[1] + (np.arange(i0[1], i1[1])[None, :] + 0.5 + offs[:, None]) * h[1]
        zs = lo[2] + (np.arange(i0[2], i1[2])[None, :] + 0.5 + offs[:, None]) * h[2]
        # coordinates relative to the centre, shape (ss, n_axis)
        X, Y, Z = xs - e.center[0], ys - e.center[1], zs - e.center[2]
        cnt = np.zeros((i1[2] - i0[2], i1[1] - i0[1], i1[0] - i0[0]))
        for a in range(ss):
            for b_ in range(ss):
                # q = M @ (x, y, z): separable sums over the three axes
                zq = M[:, 2][:, None] * Z[a][None, :]              # (3, nzb)
                yq = M[:, 1][:, None] * Y[b_][None, :]             # (3, nyb)
                zy = zq[:, :, None] + yq[:, None, :]               # (3, nzb, nyb)
                for c_ in range(ss):
                    xq = M[:, 0][:, None] * X[c_][None, :]         # (3, nxb)
                    q2 = np.zeros(cnt.shape)
                    for r in range(3):
                        q2 += (zy[r][:, :, None] + xq[r][None, None, :]) ** 2
                    cnt += q2 <= 1.0
        acc[i0[2]:i1[2], i0[1]:i1[1], i0[0]:i1[0]] += e.rho * cnt / ss ** 3
    return acc.astype(dtype)


def gaussian_noise(b: np.ndarray, frac: float, seed: int) -> np.ndarray:
    """b + N(0, sigma^2), sigma = frac * max(b); normals drawn in FP64, seeded."""
    rng = np.random.default_rng(seed)
    sigma = frac * float(np.max(b))
    return (np.asarray(b, dtype=np.float64) + sigma * rng.standard_normal(b.shape))


def serving_geometry(n: int, views: int) -> dict:
    """Serving scan of an n^3 volume of 1 mm voxels, detector scaled to the
    magnification 1.6: pixels of 1.6 mm, 1.5 n x 1.125 n of them."""
    return dict(nx=n, ny=n, nz=n, vx=1.0, vy=1.0, vz=1.0, nu=int(1.5 * n), nv=int(1.125 * n),
                du=1.6, dv=1.6, sid=750.0, sdd=1200.0, nviews=views)


def serving_stream(n_requests: int = 128, rate: float = 20.0, seed: int = 3,
                   sizes=(64, 128, 192, 256), views=(60, 120, 180, 360)):
    """Poisson request stream: per request, in this order from
    default_rng(seed): exponential inter-arrival time (mean 1/rate), volume
    size, view count, solver (CGLS or LSQR), phantom seed."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate)
        n = int(rng.choice(sizes))
        v = int(rng.choice(views))
        solver = str(rng.choice(["cgls", "lsqr"]))
        out.append(dict(rid=rid, arrival=t, n=n, views=v, solver=solver,
                        phantom_seed=int(rng.integers(1 << 31))))
    return out


def serving_phantom(n: int, seed: int, n_ellipsoids: int = 8) -> np.ndarray:
    """Random-ellipsoid phantom for an n^3 serving volume (semi-axes scaled by n/256)."""
    cfg = serving_geometry(n, 1)
    lo, hi = box_of(cfg)
    return voxelize(random_ellipsoids(n_ellipsoids, seed, lo, hi, axis_scale=n / 256.0), cfg)


def random_field(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """Signed standard-normal test vector (negative values are allowed, Discussion)."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)
