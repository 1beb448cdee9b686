"""GPU parity on a seeded sweep of random geometries, through the C ABI.

Sixteen geometries drawn from a fixed seed: ragged volumes of anisotropic
voxels, off-centre volumes, shifted detectors of any aspect, short and long
source distances (some with rays that advance mostly along z, which take the
ray-major kernels), explicit view angles anywhere on the circle.  For each,
A and A^T of random fields match the FP64 oracle within the projector
tolerance (1e-5 relative L2), the GPU pair satisfies the adjoint identity,
the nonzero count matches the oracle's, and, on half of them, the
deterministic mode gives the same results.  Both footprint projectors are
held to their oracle on every geometry.  Angles and offsets are generic, so
no ray lies exactly in a voxel-boundary plane (an ill-posed case, see
tests/test_gpu_operator.py)."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import footprint as ofp

pytestmark = pytest.mark.gpu

TOL = 1e-5
N_GEOMETRIES = 16


def random_geometry(rng):
    nx, ny, nz = (int(v) for v in rng.integers(3, 37, size=3))
    vx, vy, vz = (float(v) for v in rng.uniform(0.6, 1.8, size=3))
    ext = np.array([nx * vx, ny * vy, nz * vz])
    ox, oy, oz = (float(v) for v in rng.normal(0.0, 0.15, size=3) * ext)
    rmax = max(math.hypot(sx * 0.5 * ext[0] + ox, sy * 0.5 * ext[1] + oy)
               for sx in (-1, 1) for sy in (-1, 1))
    sid = float(rmax * rng.uniform(1.3, 6.0))
    sdd = float(sid * rng.uniform(1.3, 2.2))
    mag = sdd / sid
    nu, nv = int(rng.integers(8, 65)), int(rng.integers(6, 61))
    # pixels sized so that the detector sees most of the volume's shadow
    du = float(mag * 2 * rmax / nu * rng.uniform(0.6, 1.4))
    dv = float(mag * (ext[2] + 2 * abs(oz)) / nv * rng.uniform(0.6, 1.6))
    nviews = int(rng.integers(3, 10))
    angles = sorted(float(a) for a in rng.uniform(0.0, 2 * math.pi, size=nviews))
    return dict(nx=nx, ny=ny, nz=nz, vx=vx, vy=vy, vz=vz, ox=ox, oy=oy, oz=oz, nu=nu, nv=nv,
                du=du, dv=dv, sid=sid, sdd=sdd, nviews=nviews, angles=angles,
                det_off_u=float(rng.normal(0.0, 2.0) * du),
                det_off_v=float(rng.normal(0.0, 2.0) * dv))


GEOMS = [random_geometry(np.random.default_rng(1000 + k)) for k in range(N_GEOMETRIES)]


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


@pytest.mark.parametrize("k", range(N_GEOMETRIES))
def test_siddon_pair_on_random_geometry(ct, k):
    cfg = GEOMS[k]
    og = oracle.OGeom(**cfg)
    g = ct.Geometry(**cfg)
    x = synth.random_field(g.vol_shape, seed=10 + k)
    y = synth.random_field(g.sino_shape, seed=50 + k)
    want_p = oracle.project(og, x.astype(np.float64))
    want_r = oracle.backproject(og, y.astype(np.float64))
    assert np.count_nonzero(want_p) > 0.05 * want_p.size, "the detector misses the volume"
    p = ct.project(g, torch.from_numpy(x).cuda())
    r = ct.backproject(g, torch.from_numpy(y).cuda())
    assert rel(p.cpu().numpy(), want_p) < TOL
    assert rel(r.cpu().numpy(), want_r) < TOL
    # the GPU pair is adjoint to FP32 rounding
    xd, yd = torch.from_numpy(x).cuda().double(), torch.from_numpy(y).cuda().double()
    lhs, rhs = float((p.double() * yd).sum()), float((xd * r.double()).sum())
    scale = float((p.double().abs() * yd.abs()).sum())
    assert abs(lhs - rhs) <= 2e-6 * scale
    assert abs(ct.count_nnz(g) - oracle.count_nnz(og)) <= 1e-3 * oracle.count_nnz(og)
    if k % 2 == 0:
        gd = ct.Geometry(**cfg, deterministic=True)
        assert rel(ct.backproject(gd, torch.from_numpy(y).cuda()).cpu().numpy(), want_r) < TOL
        assert torch.equal(ct.project(gd, torch.from_numpy(x).cuda()), p)


@pytest.mark.parametrize("kind", ["sf_tr", "sf_tt"])
@pytest.mark.parametrize("k", range(0, N_GEOMETRIES, 2))
def test_footprint_pair_on_random_geometry(ct, k, kind):
    cfg = GEOMS[k]
    og = oracle.OGeom(**cfg)
    g = ct.Geometry(**cfg, projector=kind, deterministic=(k % 4 == 0))
    x = np.abs(synth.random_field(g.vol_shape, seed=90 + k))
    y = synth.random_field(g.sino_shape, seed=95 + k)
    want_p = ofp.project(og, x.astype(np.float64), kind[3:])
    want_r = ofp.backproject(og, y.astype(np.float64), kind[3:])
    assert rel(ct.project(g, torch.from_numpy(x).cuda()).cpu().numpy(), want_p) < TOL
    assert rel(ct.backproject(g, torch.from_numpy(y).cuda()).cpu().numpy(), want_r) < TOL
