"""The bounds-checking build (CT_DEBUG_BOUNDS): every voxel and pixel index
the projector kernels touch is checked.  Small cases (8^3 and 16^3 volumes,
the parity geometries) through every projector path -- column-major and
ray-major walks, float and fixed-point backprojection, batched launches,
footprint projectors, the allocation-free projection, the solvers -- must
record no violation and still match the FP64 oracle.  It runs in a child
process because the library variant is chosen when the library loads."""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes
import numpy as np, torch
import paper_2110_13526_gb300 as ct
import oracle, synth
oracle.build()
assert ct.debug_bounds_build(), "the checking library was not loaded"
def rel(a, b):
    a = a.double().cpu().numpy().ravel(); b = np.ravel(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
cases = {
    "cube8": dict(nx=8, ny=8, nz=8, vx=1.0, vy=1.0, vz=1.0, nu=13, nv=11, du=1.0, dv=1.0,
                  sid=40.0, sdd=70.0, nviews=9),
    "ragged16": dict(nx=17, ny=15, nz=16, vx=1.1, vy=0.9, vz=1.3, nu=29, nv=37, du=1.0, dv=0.8,
                     sid=60.0, sdd=110.0, nviews=7, ox=1.5, oz=-2.0, det_off_u=0.7),
    "bigcone": dict(nx=16, ny=16, nz=40, vx=1.0, vy=1.0, vz=1.0, nu=24, nv=70, du=1.5, dv=2.5,
                    sid=30.0, sdd=60.0, nviews=5),
    "pairs": dict(nx=16, ny=16, nz=12, vx=1.0, vy=1.0, vz=1.0, nu=20, nv=90, du=0.5, dv=0.4,
                  sid=80.0, sdd=140.0, nviews=5),
    "source_inside": dict(nx=16, ny=16, nz=8, vx=2.0, vy=2.0, vz=1.0, nu=16, nv=12, du=2.0,
                          dv=1.5, sid=12.0, sdd=40.0, nviews=6),
    # steep rays advancing along z through a tall, narrow, off-centre volume
    # with a far-shifted detector (ray-major kernels, both setups)
    "steep": dict(nx=4, ny=5, nz=27, vx=1.37, vy=0.84, vz=1.31, ox=0.21, oy=-0.81, oz=7.27,
                  nu=54, nv=11, du=0.2, dv=8.54, sid=12.34, sdd=16.52, nviews=8,
                  det_off_u=-0.04, det_off_v=-28.28,
                  angles=[1.436, 2.112, 3.517, 3.806, 3.985, 5.232, 5.249, 6.111]),
}
for name, cfg in cases.items():
    g, og = ct.Geometry(**cfg), oracle.OGeom(**cfg)
    x = synth.random_field(g.vol_shape, seed=1)
    y = synth.random_field(g.sino_shape, seed=2)
    p = ct.project(g, torch.from_numpy(x).cuda()); ct.debug_status()
    assert rel(p, oracle.project(og, x.astype(np.float64))) < 1e-5, name
    r = ct.backproject(g, torch.from_numpy(y).cuda()); ct.debug_status()
    assert rel(r, oracle.backproject(og, y.astype(np.float64))) < 1e-5, name
    gd = ct.Geometry(**cfg, deterministic=True)
    ct.backproject(gd, torch.from_numpy(y).cuda()); ct.debug_status()
    xb = torch.from_numpy(synth.random_field((2,) + g.vol_shape, seed=3)).cuda()
    yb = ct.project_batch(g, xb); ct.backproject_batch(g, yb); ct.debug_status()
    ct.count_nnz(g); ct.project_norm2(g, torch.from_numpy(x).cuda()); ct.debug_status()
    xd = torch.from_numpy(x).cuda()
    sd = torch.empty(g.sino_shape, device="cuda")
    nd = torch.zeros((), dtype=torch.float64, device="cuda")
    assert ct.lib().ct_project_norm2_noalloc(g.handle, ctypes.c_void_p(xd.data_ptr()),
                                             ctypes.c_void_p(sd.data_ptr()), ctypes.c_float(1.0),
                                             ctypes.c_float(0.0), ctypes.c_void_p(nd.data_ptr()),
                                             None) == 0
    assert rel(sd, oracle.project(og, x.astype(np.float64))) < 1e-5, name
    ct.debug_status()
    b = torch.from_numpy(oracle.project(og, np.abs(x).astype(np.float64)).astype(np.float32)).cuda()
    for pc in ("none", "jacobi", "rowcol"):
        ct.cgls(g, b, max_iter=4, precond=pc); ct.debug_status()
        ct.lsqr(g, b, max_iter=4, precond=pc); ct.debug_status()
    ct.cgls(g, b, max_iter=4, tikhonov=0.1); ct.sirt(g, b, max_iter=3); ct.debug_status()
    bt = ct.Batch(); j = bt.add(g, b, max_iter=3)
    while not bt.done(j): bt.step()
    bt.result(j); bt.close(); ct.debug_status()
    if name != "source_inside":
        for proj in ("sf_tr", "sf_tt"):
            gs = ct.Geometry(**cfg, projector=proj)
            ct.project(gs, torch.from_numpy(x).cuda()); ct.backproject(gs, torch.from_numpy(y).cuda())
            ct.debug_status()
    print("checked", name, flush=True)
print("debug-bounds ok")
'''


def test_bounds_checking_build_records_no_violation():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2110_13526_gb300.build as B
    B.build(debug=True)
    env = dict(os.environ, CT_GB300_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", "import sys; sys.path.insert(0, %r)\n" % ROOT + CHILD],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug-bounds ok" in r.stdout
