"""ct_project_norm2_noalloc, the allocation-free entry point, against the
allocating ct_project_norm2, both called through the C ABI.

Callers that cannot let a library allocate device memory once they run (a
service that reserves HBM up front for its own pool, or a real-time pipeline
with no room for an allocator call) use the allocation-free variant.  It keeps
its FP64 partial sums in a fixed device array shared by every call, so this
test makes two calls in a row with different inputs and checks that each
matches the allocating entry point to the projector tolerance (1e-5
relative L2).  The file sorts last so a failure here stops a -x run only
after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5

# ragged tails, several CTAs per view, views advancing along x and along y
CFG = dict(nx=37, ny=29, nz=21, vx=1.1, vy=0.9, vz=1.3, nu=71, nv=45, du=1.0, dv=1.2,
           sid=300.0, sdd=520.0, nviews=17)


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2110_13526_gb300 as m
    m.lib()
    return m


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(L, name, g, vol, sino, alpha, beta, nrm):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = getattr(L, name)(g.handle, _p(vol), _p(sino), ctypes.c_float(alpha),
                          ctypes.c_float(beta), _p(nrm), stream)
    assert st == 0, L.ct_last_error()


def rel(a, b):
    a, b = a.double().cpu().numpy().ravel(), b.double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("projector", ["siddon", "sf_tt"])
def test_noalloc_matches_allocating_entry_point_twice(ct, projector):
    L = ct.lib()
    g = ct.Geometry(**CFG, projector=projector)
    for call, (seed, alpha, beta) in enumerate([(21, 1.0, 0.0), (22, -0.5, 1.5)]):
        vol = torch.from_numpy(synth.random_field(g.vol_shape, seed=seed)).cuda()
        start = torch.from_numpy(synth.random_field(g.sino_shape, seed=seed + 100)).cuda()
        s_ref, s_new = start.clone(), start.clone()
        n_ref = torch.zeros((), dtype=torch.float64, device="cuda")
        n_new = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        _call(L, "ct_project_norm2", g, vol, s_ref, alpha, beta, n_ref)
        _call(L, "ct_project_norm2_noalloc", g, vol, s_new, alpha, beta, n_new)
        torch.cuda.synchronize()
        assert rel(s_new, s_ref) < TOL, call
        assert abs(float(n_new) - float(n_ref)) <= TOL * float(n_ref), call
        assert float(n_new) == pytest.approx(float((s_new.double() ** 2).sum()), rel=1e-12)


def test_noalloc_grouped_views(ct):
    """nviews * ceil(nv/8) > 65535: the direct launch groups 2 views per grid
    slot (40001 views, 16 rows: G = ceil(40001 / 32767) = 2), and the last
    group is half empty.  Its idle CTAs must still write zero partials."""
    L = ct.lib()
    cfg = dict(nx=6, ny=5, nz=4, vx=1.0, vy=1.0, vz=1.0, nu=20, nv=16, du=0.7, dv=0.7,
               sid=40.0, sdd=70.0, nviews=40001)
    g = ct.Geometry(**cfg)
    for seed, alpha, beta in [(31, 1.0, 0.0), (32, 2.0, -1.0)]:
        vol = torch.from_numpy(synth.random_field(g.vol_shape, seed=seed)).cuda()
        start = torch.from_numpy(synth.random_field(g.sino_shape, seed=seed + 100)).cuda()
        s_ref, s_new = start.clone(), start.clone()
        n_ref = torch.zeros((), dtype=torch.float64, device="cuda")
        n_new = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        _call(L, "ct_project_norm2", g, vol, s_ref, alpha, beta, n_ref)
        _call(L, "ct_project_norm2_noalloc", g, vol, s_new, alpha, beta, n_new)
        torch.cuda.synchronize()
        assert rel(s_new, s_ref) < TOL
        assert abs(float(n_new) - float(n_ref)) <= TOL * float(n_ref)
        assert float(n_new) == pytest.approx(float((s_new.double() ** 2).sum()), rel=1e-12)


def test_noalloc_rejects_geometry_beyond_static_scratch(ct):
    L = ct.lib()
    # 8 * 8 * 4097 = 262 208 CTAs of 32 x 8 rays > 262 144 partial sums
    g = ct.Geometry(nx=4, ny=4, nz=4, vx=1, vy=1, vz=1, nu=256, nv=64, du=1, dv=1, sid=50,
                    sdd=80, nviews=4097)
    vol = torch.zeros(g.vol_shape, device="cuda")
    sino = torch.empty(g.sino_shape, device="cuda")
    nrm = torch.zeros((), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.ct_project_norm2_noalloc(g.handle, _p(vol), _p(sino), ctypes.c_float(1.0),
                                    ctypes.c_float(0.0), _p(nrm), stream)
    assert st == 1
    msg = L.ct_last_error()
    assert b"static scratch" in msg and b"262208" in msg


def test_noalloc_rejects_deterministic_footprint_geometry(ct):
    """A deterministic footprint geometry sums its projection in int64
    workspace, which the allocation-free entry point cannot take."""
    L = ct.lib()
    g = ct.Geometry(**CFG, projector="sf_tt", deterministic=True)
    vol = torch.zeros(g.vol_shape, device="cuda")
    sino = torch.empty(g.sino_shape, device="cuda")
    nrm = torch.zeros((), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.ct_project_norm2_noalloc(g.handle, _p(vol), _p(sino), ctypes.c_float(1.0),
                                    ctypes.c_float(0.0), _p(nrm), stream)
    assert st == 1 and b"int64" in L.ct_last_error()
