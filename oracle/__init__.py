"""FP64 CPU oracle for the cone-beam CT operator and the Krylov solvers.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2110_13526_gb300``)
and neither imports the other.

Contents
--------
* ``OGeom``           -- the geometry as plain FP64 numbers (own copy of the
                         conventions, independent of the library's).
* ``project`` / ``backproject`` / ``count_nnz`` / ``ray_segments``
                      -- Siddon A and A^T in C (``siddon_ref.c``), FP64.
* ``oracle.dense``    -- brute-force dense A (ray x voxel-cube slab
                         intersection), a third independent method, for <= 8^3.
* ``oracle.solvers``  -- CGLS (Algorithm 1), LSQR (Paige & Saunders 1982),
                         SIRT / PSIRT, preconditioners, in NumPy FP64.
* ``oracle.ellipsoid``-- closed-form line integrals of ellipsoids (a pin).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siddon_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboref.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP, IEEE FP64, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _CGeom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("vz", ctypes.c_double),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double),
                ("nu", ctypes.c_int32), ("nv", ctypes.c_int32),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("det_off_u", ctypes.c_double), ("det_off_v", ctypes.c_double),
                ("sid", ctypes.c_double), ("sdd", ctypes.c_double),
                ("nviews", ctypes.c_int32),
                ("angles", ctypes.POINTER(ctypes.c_double))]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.oref_project.argtypes = [P(_CGeom), P(ctypes.c_double), P(ctypes.c_double),
                                     ctypes.c_int]
        lib.oref_backproject.argtypes = [P(_CGeom), P(ctypes.c_double), P(ctypes.c_double),
                                         ctypes.c_int, ctypes.c_int]
        lib.oref_count_nnz.argtypes = [P(_CGeom), P(ctypes.c_int64), ctypes.c_int]
        lib.oref_ray.argtypes = [P(_CGeom), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 P(ctypes.c_int64), P(ctypes.c_double), ctypes.c_int]
        lib.oref_segment.argtypes = [P(_CGeom), P(ctypes.c_double), P(ctypes.c_double),
                                     P(ctypes.c_int64), P(ctypes.c_double), ctypes.c_int]
        for f in (lib.oref_project, lib.oref_backproject, lib.oref_count_nnz, lib.oref_ray,
                  lib.oref_segment):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


@dataclass
class OGeom:
    """Circular cone-beam geometry, all lengths in mm, angles in radians.

    Volume ``nx x ny x nz`` voxels of pitch ``vx, vy, vz`` centred at
    ``(ox, oy, oz)`` (off-centre reconstruction, Software section); flat
    detector ``nu x nv`` pixels of pitch ``du, dv``; source-isocentre ``sid``,
    source-detector ``sdd`` (Results section: C-arm-like geometry).  Without
    ``angles`` the views are uniform over 360 degrees, 2 pi k / nviews.
    """
    nx: int
    ny: int
    nz: int
    vx: float
    vy: float
    vz: float
    nu: int
    nv: int
    du: float
    dv: float
    sid: float
    sdd: float
    nviews: int
    ox: float = 0.0
    oy: float = 0.0
    oz: float = 0.0
    det_off_u: float = 0.0
    det_off_v: float = 0.0
    angles: Optional[Sequence[float]] = field(default=None)

    def angle_array(self) -> np.ndarray:
        if self.angles is not None:
            a = np.asarray(self.angles, dtype=np.float64)
            assert a.shape == (self.nviews,)
            return np.ascontiguousarray(a)
        return 2.0 * np.pi * np.arange(self.nviews, dtype=np.float64) / max(self.nviews, 1)

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.nviews, self.nv, self.nu)

    def subset(self, views: Sequence[int]) -> "OGeom":
        """The same geometry restricted to the given view indices."""
        a = self.angle_array()[np.asarray(views, dtype=np.int64)]
        d = dict(self.__dict__)
        d["nviews"] = len(a)
        d["angles"] = a.tolist()
        return OGeom(**d)

    def _c(self):
        ang = self.angle_array()
        cg = _CGeom(self.nx, self.ny, self.nz, self.vx, self.vy, self.vz,
                    self.ox, self.oy, self.oz, self.nu, self.nv, self.du, self.dv,
                    self.det_off_u, self.det_off_v, self.sid, self.sdd, self.nviews,
                    ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return cg, ang  # keep ang alive with the struct


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def project(g: OGeom, vol, threads: Optional[int] = None) -> np.ndarray:
    """b = A x in FP64 (Eq. 1).  vol: (nz, ny, nx) -> (nviews, nv, nu)."""
    lib = _load()
    v = np.ascontiguousarray(vol, dtype=np.float64).reshape(g.vol_shape)
    out = np.zeros(g.sino_shape, dtype=np.float64)
    cg, _keep = g._c()
    rc = lib.oref_project(ctypes.byref(cg), _dptr(v), _dptr(out), threads or default_threads())
    if rc != 0:
        raise RuntimeError("oref_project failed with %d" % rc)
    return out


def backproject(g: OGeom, sino, threads: Optional[int] = None, power: int = 1) -> np.ndarray:
    """x = A^T b in FP64 (power=1); power=2 uses squared lengths, (A o A)^T b."""
    lib = _load()
    s = np.ascontiguousarray(sino, dtype=np.float64).reshape(g.sino_shape)
    out = np.zeros(g.vol_shape, dtype=np.float64)
    cg, _keep = g._c()
    rc = lib.oref_backproject(ctypes.byref(cg), _dptr(s), _dptr(out),
                              threads or default_threads(), power)
    if rc != 0:
        raise RuntimeError("oref_backproject failed with %d" % rc)
    return out


def count_nnz(g: OGeom, threads: Optional[int] = None) -> int:
    """Number of (ray, voxel) pairs with positive intersection length."""
    lib = _load()
    out = ctypes.c_int64(0)
    cg, _keep = g._c()
    rc = lib.oref_count_nnz(ctypes.byref(cg), ctypes.byref(out), threads or default_threads())
    if rc != 0:
        raise RuntimeError("oref_count_nnz failed with %d" % rc)
    return int(out.value)


def ray_segments(g: OGeom, view: int, u: int, v: int):
    """(linear voxel indices, lengths in mm) of one detector ray."""
    lib = _load()
    cap = g.nx + g.ny + g.nz + 5
    idx = np.zeros(cap, dtype=np.int64)
    ln = np.zeros(cap, dtype=np.float64)
    cg, _keep = g._c()
    n = lib.oref_ray(ctypes.byref(cg), view, u, v,
                     idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(ln), cap)
    if n < 0:
        raise RuntimeError("oref_ray failed")
    return idx[:n].copy(), ln[:n].copy()


def segment_segments(g: OGeom, s, p):
    """(linear voxel indices, lengths) of the straight segment s -> p."""
    lib = _load()
    cap = g.nx + g.ny + g.nz + 5
    idx = np.zeros(cap, dtype=np.int64)
    ln = np.zeros(cap, dtype=np.float64)
    sa = np.ascontiguousarray(s, dtype=np.float64)
    pa = np.ascontiguousarray(p, dtype=np.float64)
    cg, _keep = g._c()
    n = lib.oref_segment(ctypes.byref(cg), _dptr(sa), _dptr(pa),
                         idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(ln), cap)
    if n < 0:
        raise RuntimeError("oref_segment failed")
    return idx[:n].copy(), ln[:n].copy()


def ray_endpoints(g: OGeom, view: int, u: int, v: int):
    """Source and pixel-centre position of one ray (same conventions as the C code)."""
    th = float(g.angle_array()[view])
    c, s_ = np.cos(th), np.sin(th)
    src = np.array([g.sid * c, g.sid * s_, 0.0])
    cd = -(g.sdd - g.sid)
    uu = (u - 0.5 * (g.nu - 1)) * g.du + g.det_off_u
    vv = (v - 0.5 * (g.nv - 1)) * g.dv + g.det_off_v
    pix = np.array([cd * c - uu * s_, cd * s_ + uu * c, vv])
    return src, pix


class Operator:
    """A and A^T of one geometry with call counters (the op-count pin of Alg. 1)."""

    def __init__(self, g: OGeom, threads: Optional[int] = None):
        self.g = g
        self.threads = threads
        self.n_forward = 0
        self.n_back = 0

    def A(self, x):
        self.n_forward += 1
        return project(self.g, x, self.threads)

    def AT(self, y):
        self.n_back += 1
        return backproject(self.g, y, self.threads)

    @property
    def calls(self):
        return self.n_forward + self.n_back
