"""Mixed-precision storage (BF16 / FP16 volumes and sinograms, FP32 ray
sums, FP64 Krylov scalars).

* Typed outputs are the FP32 result rounded once to the storage type
  (bitwise), typed inputs keep the FP32 parity bar against the oracle applied
  to the same rounded values.
* Rounding an output of magnitude |y| to BF16 (8-bit significand) or FP16
  (11-bit) errs by at most 2^-9 |y| or 2^-12 |y|; the relative L2 error of a
  rounded sinogram is therefore below 2^-9 (BF16) and 2^-12 (FP16).
* CGLS with BF16 / FP16 Krylov vectors is measured against the FP32 run and
  the FP64 oracle; the bounds below are the measured errors with margin.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.solvers import cgls as ocgls

pytestmark = pytest.mark.gpu

CFG = dict(nx=37, ny=29, nz=21, vx=1.1, vy=0.9, vz=1.3, nu=71, nv=45, du=1.0, dv=1.2,
           sid=300.0, sdd=520.0, nviews=17)
RND = {torch.bfloat16: 2.0 ** -9, torch.float16: 2.0 ** -12}


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2110_13526_gb300 as m
    m.lib()
    oracle.build()
    return m


def rel(a, b):
    a = a.double().cpu().numpy() if torch.is_tensor(a) else np.asarray(a, dtype=np.float64)
    b = b.double().cpu().numpy() if torch.is_tensor(b) else np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a.ravel() - b.ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_typed_forward(ct, dt):
    g, og = ct.Geometry(**CFG), oracle.OGeom(**CFG)
    x = torch.from_numpy(synth.random_field(g.vol_shape, seed=30)).cuda()
    p32 = ct.project(g, x)
    # FP32 in, typed out: one rounding of the FP32 result
    pt = ct.project(g, x, out_dtype=dt)
    assert pt.dtype == dt and torch.equal(pt, p32.to(dt))
    want = oracle.project(og, x.cpu().double().numpy())
    assert rel(pt, want) < RND[dt]
    # typed in, FP32 out: same parity bar as FP32 on the rounded input
    xt = x.to(dt)
    p = ct.project(g, xt, out_dtype=torch.float32)
    assert rel(p, oracle.project(og, xt.double().cpu().numpy())) < 1e-5
    # typed in and out, alpha/beta epilogue
    y0 = torch.from_numpy(synth.random_field(g.sino_shape, seed=31)).cuda().to(dt)
    out = y0.clone()
    ct.project(g, xt, out=out, alpha=0.5, beta=-2.0)
    ref = (0.5 * ct.project(g, xt, out_dtype=torch.float32) - 2.0 * y0.float())
    assert rel(out, ref) < 2 * RND[dt]


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_typed_backward(ct, dt):
    g, og = ct.Geometry(**CFG), oracle.OGeom(**CFG)
    y = torch.from_numpy(synth.random_field(g.sino_shape, seed=32)).cuda()
    yt = y.to(dt)
    r = ct.backproject(g, yt, out_dtype=torch.float32)
    assert rel(r, oracle.backproject(og, yt.double().cpu().numpy())) < 1e-5
    # deterministic sums: typed output = FP32 result rounded once
    gd = ct.Geometry(**CFG, deterministic=True)
    r32 = ct.backproject(gd, y)
    rt = ct.backproject(gd, y, out_dtype=dt)
    assert rt.dtype == dt and torch.equal(rt, r32.to(dt))
    assert rel(rt, oracle.backproject(og, y.cpu().double().numpy())) < RND[dt]


@pytest.mark.parametrize("dt,tol_f32,tol_oracle", [("bf16", 3e-2, 3e-2), ("f16", 3e-3, 3e-3)])
def test_cgls_reduced_storage(ct, dt, tol_f32, tol_oracle):
    cfg = synth.CONFIGS["PR1"]
    og = oracle.OGeom(**cfg)
    x = synth.voxelize(synth.nested_phantom(64.0, seed=0), cfg)
    b = synth.gaussian_noise(oracle.project(og, x.astype(np.float64)), 0.01, seed=0)
    b32 = torch.from_numpy(b.astype(np.float32)).cuda()
    g = ct.Geometry(**cfg)
    x32, r32 = ct.cgls(g, b32, max_iter=20)
    xt, rt = ct.cgls(g, b32, max_iter=20, storage=dt)
    ref = ocgls(oracle.Operator(og), b.astype(np.float32).astype(np.float64), K=20)
    e32, eo = rel(xt, x32), rel(xt.cpu().numpy(), ref.x)
    print("storage %s: rel to FP32 run %.2e, to FP64 oracle %.2e; NB/NB0 %.4e vs %.4e"
          % (dt, e32, eo, rt.history[-1], r32.history[-1]))
    assert e32 < tol_f32 and eo < tol_oracle
    assert rt.history[-1] == pytest.approx(r32.history[-1], rel=10 * tol_f32)
    assert all(rt.history[k + 1] <= rt.history[k] * (1 + tol_f32) for k in range(19))


def test_p512_typed_forward_sampled_views(ct):
    """512^3 precision workload (0.5 mm voxels, 768x576 detector of 0.75 mm,
    720 views): BF16 and FP16 volumes against the oracle on 4 sampled views."""
    cfg = synth.CONFIGS["P512"]
    g = ct.Geometry(**cfg)
    views = [0, 180, 361, 545]
    og = oracle.OGeom(**cfg).subset(views)
    lo, hi = synth.box_of(cfg)
    x = torch.from_numpy(synth.voxelize(synth.random_ellipsoids(40, 2, lo, hi), cfg)).cuda()
    want = oracle.project(og, x.cpu().double().numpy())
    p32 = ct.project(g, x)[views]
    assert rel(p32, want) < 1e-5
    for dt in (torch.bfloat16, torch.float16):
        xt = x.to(dt)
        pt = ct.project(g, xt, out_dtype=dt)[views]
        # input rounding (relative 2^-9 / 2^-12 per voxel) plus output rounding
        assert rel(pt, want) < 2 * RND[dt]
