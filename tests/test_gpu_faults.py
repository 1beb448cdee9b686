"""Host-side failure handling and checkpoint/resume of the solvers.

No test here provokes a GPU fault: bad input is made on the host (NaN, Inf,
truncated or foreign state bytes) and the library must report it as a
status, with the device left usable.  CGLS checkpoint/resume (ct_cgls_state)
must continue a solve exactly: bitwise with a deterministic geometry, and
within the solver tolerance of the FP64 oracle in float mode.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.solvers import cgls as ocgls

pytestmark = pytest.mark.gpu

TOL_X = 1e-4
CFG = dict(nx=30, ny=26, nz=18, vx=1.0, vy=1.0, vz=1.2, nu=44, nv=28, du=1.0, dv=1.0,
           sid=250.0, sdd=400.0, nviews=24)


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2110_13526_gb300 as m
    m.lib()
    oracle.build()
    return m


@pytest.fixture(scope="module")
def data():
    og = oracle.OGeom(**CFG)
    ells = synth.random_ellipsoids(6, 5, *synth.box_of(CFG), axis_range=(3.0, 10.0))
    x = synth.voxelize(ells, CFG)
    b = synth.gaussian_noise(oracle.project(og, x.astype(np.float64)), 0.01, seed=1)
    return og, b.astype(np.float32)


def rel(a, b):
    a = a.double().cpu().numpy().ravel() if torch.is_tensor(a) else np.ravel(a)
    return float(np.linalg.norm(a - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("err_tol", [0.0, 1e-3])
def test_non_finite_b_is_reported(ct, data, err_tol):
    _, b = data
    g = ct.Geometry(**CFG)
    bad = torch.from_numpy(b).cuda()
    bad[3, 7, 11] = float("nan")
    for fn in (ct.cgls, ct.lsqr, ct.sirt):
        with pytest.raises(ct.CTError, match="CT_ERR_INVALID_ARG.*non-finite"):
            fn(g, bad, max_iter=5, err_tol=err_tol)
    bad[3, 7, 11] = float("inf")
    with pytest.raises(ct.CTError, match="non-finite"):
        ct.cgls(g, bad, max_iter=5, err_tol=err_tol)
    # the device is still usable afterwards
    x, rep = ct.cgls(g, torch.from_numpy(b).cuda(), max_iter=3)
    assert rep.iterations == 3 and torch.isfinite(x).all()


def test_non_finite_x0_is_reported(ct, data):
    _, b = data
    g = ct.Geometry(**CFG)
    x0 = torch.zeros(g.vol_shape, device="cuda")
    x0[5, 5, 5] = float("inf")
    with pytest.raises(ct.CTError, match="non-finite"):
        ct.cgls(g, torch.from_numpy(b).cuda(), x0=x0, max_iter=4)


def test_zero_b_gives_zero(ct):
    g = ct.Geometry(**CFG)
    zero = torch.zeros(g.sino_shape, device="cuda")
    for fn in (ct.cgls, ct.lsqr):
        x, rep = fn(g, zero, max_iter=4)
        assert float(x.abs().max()) == 0.0 and rep.nb0 == 0.0


@pytest.mark.parametrize("precond", ["none", "rowcol"])
def test_resume_is_bitwise_in_deterministic_mode(ct, data, precond):
    """10 updates in one call == 4, checkpoint to bytes, restore into a new
    state, 3 more, then 3 more: x and every history entry bitwise equal."""
    _, b = data
    g = ct.Geometry(**CFG, deterministic=True)
    bd = torch.from_numpy(b).cuda()
    x_ref, rep_ref = ct.cgls(g, bd, max_iter=10, precond=precond)
    s1 = ct.CglsState(g)
    x4, r4 = s1.run(bd, 4, precond=precond)
    assert s1.iterations == 4 and r4.iterations == 4
    blob = s1.to_bytes()
    s1.close()
    s2 = ct.CglsState(g)
    s2.from_bytes(blob)
    assert s2.iterations == 4
    x7, _ = s2.run(bd, 7, precond=precond)
    x10, r10 = s2.run(bd, 10, precond=precond)
    assert torch.equal(x10, x_ref)
    assert r10.iterations == 10 and r10.history == rep_ref.history
    # running a state again at its own count does nothing but return x
    x10b, _ = s2.run(bd, 10, precond=precond)
    assert torch.equal(x10b, x_ref)
    s2.close()


def test_resume_float_mode_matches_oracle(ct, data):
    og, b = data
    g = ct.Geometry(**CFG)
    bd = torch.from_numpy(b).cuda()
    s = ct.CglsState(g)
    s.run(bd, 5)
    x, rep = s.run(bd, 12)
    ref = ocgls(oracle.Operator(og), b.astype(np.float64), K=12)
    assert rep.iterations == 12
    assert rel(x, ref.x) < TOL_X
    np.testing.assert_allclose(rep.history, ref.history, rtol=TOL_X)
    s.close()


def test_state_import_rejects_bad_bytes(ct, data):
    _, b = data
    g = ct.Geometry(**CFG)
    s = ct.CglsState(g)
    s.run(torch.from_numpy(b).cuda(), 2)
    blob = s.to_bytes()
    with pytest.raises(ct.CTError, match="CT_ERR_INVALID_ARG"):
        s.from_bytes(blob[:-8])                       # truncated
    with pytest.raises(ct.CTError, match="CT_ERR_INVALID_ARG"):
        s.from_bytes(b"\0" * len(blob))               # not a state
    other = ct.CglsState(ct.Geometry(**dict(CFG, nz=17)))
    with pytest.raises(ct.CTError, match="sizes do not match"):
        other.from_bytes(blob)                        # another geometry size
    with pytest.raises(ct.CTError, match="max_iter"):
        s.run(torch.from_numpy(b).cuda(), 1)          # fewer updates than the state holds
    s.from_bytes(blob)                                # the state itself still restores
    assert s.iterations == 2
