"""GPU parity of ct_cgls / ct_lsqr with the FP64 oracle solvers.

Tolerance: iterates within 1e-4 relative L2 of the oracle after k iterations
(FP32 vectors, FP64 Krylov scalars)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.solvers import cgls as ocgls
from oracle.solvers import jacobi_weights, lsqr as olsqr, rowcol_weights
from oracle.solvers import sirt as osirt

pytestmark = pytest.mark.gpu

TOL_X = 1e-4


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


@pytest.fixture(scope="module")
def pr1():
    """PR1: 64^3 nested phantom, 90 views, b = A x + 1 % Gaussian noise."""
    cfg = synth.CONFIGS["PR1"]
    og = oracle.OGeom(**cfg)
    x = synth.voxelize(synth.nested_phantom(64.0, seed=0), cfg)
    b = synth.gaussian_noise(oracle.project(og, x.astype(np.float64)), 0.01, seed=0)
    return cfg, og, x, b.astype(np.float32)


SMALL = dict(nx=30, ny=26, nz=18, vx=1.0, vy=1.0, vz=1.2, nu=44, nv=28, du=1.0, dv=1.0,
             sid=250.0, sdd=400.0, nviews=24)


@pytest.fixture(scope="module")
def small():
    og = oracle.OGeom(**SMALL)
    ells = synth.random_ellipsoids(6, 5, *synth.box_of(SMALL), axis_range=(3.0, 10.0))
    x = synth.voxelize(ells, SMALL)
    b = synth.gaussian_noise(oracle.project(og, x.astype(np.float64)), 0.01, seed=1)
    return SMALL, og, x, b.astype(np.float32)


def test_cgls_pr1_k20(ct, pr1):
    cfg, og, _, b = pr1
    g = ct.Geometry(**cfg)
    x, rep = ct.cgls(g, torch.from_numpy(b).cuda(), max_iter=20)
    ref = ocgls(oracle.Operator(og), b.astype(np.float64), K=20)
    assert rep.iterations == 20
    assert rel(x.cpu().numpy(), ref.x) < TOL_X
    np.testing.assert_allclose(rep.history, ref.history, rtol=TOL_X)
    assert rep.nb0 == pytest.approx(ref.nb0, rel=1e-7)


def test_lsqr_pr1_k20(ct, pr1):
    cfg, og, _, b = pr1
    g = ct.Geometry(**cfg)
    x, rep = ct.lsqr(g, torch.from_numpy(b).cuda(), max_iter=20)
    ref = olsqr(oracle.Operator(og), b.astype(np.float64), K=20)
    assert rep.iterations == 20
    assert rel(x.cpu().numpy(), ref.x) < TOL_X
    np.testing.assert_allclose(rep.history, ref.history, rtol=TOL_X)


def test_operator_call_counts(ct, small):
    """Algorithm 1 saves a projection and a backprojection: K updates cost
    2K operator calls (one more A for a nonzero x0); LSQR costs 2K + 1."""
    cfg, _, _, b = small
    g = ct.Geometry(**cfg)
    bd = torch.from_numpy(b).cuda()
    for K in (1, 2, 5):
        _, r = ct.cgls(g, bd, max_iter=K)
        assert (r.n_forward, r.n_back) == (K, K)
        _, r = ct.cgls(g, bd, x0=torch.ones(g.vol_shape), max_iter=K)
        assert (r.n_forward, r.n_back) == (K + 1, K)
        _, r = ct.lsqr(g, bd, max_iter=K)
        assert (r.n_forward, r.n_back) == (K, K + 1)


def test_nonzero_x0_and_recompute(ct, small):
    cfg, og, _, b = small
    g = ct.Geometry(**cfg)
    x0 = synth.random_field(g.vol_shape, seed=3) * 0.1
    x, rep = ct.cgls(g, torch.from_numpy(b).cuda(), x0=torch.from_numpy(x0).cuda(), max_iter=8)
    ref = ocgls(oracle.Operator(og), b.astype(np.float64), x0=x0.astype(np.float64), K=8)
    assert rel(x.cpu().numpy(), ref.x) < TOL_X
    x, rep = ct.lsqr(g, torch.from_numpy(b).cuda(), x0=torch.from_numpy(x0).cuda(), max_iter=8)
    ref = olsqr(oracle.Operator(og), b.astype(np.float64), x0=x0.astype(np.float64), K=8)
    assert rel(x.cpu().numpy(), ref.x) < TOL_X
    x, rep = ct.cgls(g, torch.from_numpy(b).cuda(), max_iter=10, recompute_every=3)
    ref = ocgls(oracle.Operator(og), b.astype(np.float64), K=10, recompute_every=3)
    assert rel(x.cpu().numpy(), ref.x) < TOL_X
    assert rep.nb == pytest.approx(ref.nb, rel=1e-4)
    assert rep.n_forward == 10 + 3            # three recomputations at i = 3, 6, 9


def test_stopping_rule(ct, small):
    cfg, og, _, b = small
    g = ct.Geometry(**cfg)
    ref = ocgls(oracle.Operator(og), b.astype(np.float64), K=30)
    err = 0.5 * (ref.history[5] + ref.history[6])   # met at the 7th update
    _, rep = ct.cgls(g, torch.from_numpy(b).cuda(), max_iter=30, err_tol=err)
    assert rep.iterations == 7 and rep.nb / rep.nb0 <= err
    refl = olsqr(oracle.Operator(og), b.astype(np.float64), K=30, err=err)
    _, rep = ct.lsqr(g, torch.from_numpy(b).cuda(), max_iter=30, err_tol=err)
    assert rep.iterations == refl.iterations


def test_precond_weights_match_oracle(ct, small):
    cfg, og, _, _ = small
    g = ct.Geometry(**cfg)
    wj, _ = ct.precond_weights(g, "jacobi")
    assert rel(wj.cpu().numpy(), jacobi_weights(og)) < 1e-5
    wc, wr = ct.precond_weights(g, "rowcol")
    L, C = rowcol_weights(og)
    assert rel(wr.cpu().numpy(), L) < 1e-5
    assert rel(wc.cpu().numpy(), C) < 1e-5
    assert torch.isfinite(wj).all() and torch.isfinite(wr).all()
    # rays that miss the volume (wide detector) have no data: weight 0, no inf/NaN
    wide = dict(cfg, du=3.0, dv=3.0)
    gw = ct.Geometry(**wide)
    _, wr2 = ct.precond_weights(gw, "rowcol")
    L2, _ = rowcol_weights(oracle.OGeom(**wide))
    assert torch.isfinite(wr2).all() and (wr2 == 0).any()
    assert torch.equal(wr2 == 0, torch.from_numpy(L2 == 0).cuda())


@pytest.mark.parametrize("kind", ["jacobi", "rowcol"])
def test_preconditioned_solvers(ct, small, kind):
    cfg, og, _, b = small
    g = ct.Geometry(**cfg)
    if kind == "jacobi":
        left, right = None, jacobi_weights(og)
    else:
        left, right = rowcol_weights(og)
    for solver, osolver in ((ct.cgls, ocgls), (ct.lsqr, olsqr)):
        x, rep = solver(g, torch.from_numpy(b).cuda(), max_iter=10, precond=kind)
        ref = osolver(oracle.Operator(og), b.astype(np.float64), K=10, left=left, right=right)
        assert rel(x.cpu().numpy(), ref.x) < TOL_X
        np.testing.assert_allclose(rep.history, ref.history, rtol=TOL_X)


def test_timing_report_and_host_path(ct, small):
    cfg, _, _, b = small
    g = ct.Geometry(**cfg)
    xd, rd = ct.cgls(g, torch.from_numpy(b).cuda(), max_iter=4, timing=True)
    assert rd.ms_forward > 0 and rd.ms_back > 0
    xh, rh = ct.cgls(g, torch.from_numpy(b), max_iter=4)       # host tensors in and out
    assert xh.device.type == "cpu"
    assert rel(xh.numpy(), xd.cpu().numpy()) < 1e-5


@pytest.fixture(scope="module")
def b256_views():
    """The 256^3 workload (256^3 voxels of 1 mm, 384 x 288 detector of 1 mm
    pixels, SID 750 / SDD 1200, 40-ellipsoid phantom, seed 1) on 24 of its 360
    views, every 15 degrees: the same kernels and launch configuration as the
    full workload (column-major walk, one view per launch group, paired rows
    in A^T), with a view count that keeps the oracle's solves in seconds.
    b = A x_true by the oracle plus 1 % Gaussian noise."""
    full = synth.CONFIGS["B256"]
    cfg = dict(full, nviews=24, angles=[2.0 * np.pi * k / 24 for k in range(24)])
    og = oracle.OGeom(**cfg)
    x = synth.voxelize(synth.random_ellipsoids(40, 1, *synth.box_of(cfg)), cfg)
    b = synth.gaussian_noise(oracle.project(og, x.astype(np.float64)), 0.01, seed=6)
    return cfg, og, b.astype(np.float32)


@pytest.mark.parametrize("solver,precond", [("cgls", "none"), ("lsqr", "none"),
                                            ("cgls", "jacobi"), ("lsqr", "rowcol")])
def test_b256_solver_parity_k10(ct, b256_views, solver, precond):
    """CGLS (Algorithm 1) and LSQR iterates after 10 updates at the 256^3 size
    against the oracle's, within 1e-4, with and without preconditioning."""
    cfg, og, b = b256_views
    g = ct.Geometry(**cfg)
    left = right = None
    if precond == "jacobi":
        right = jacobi_weights(og)
    elif precond == "rowcol":
        left, right = rowcol_weights(og)
    run, oref = (ct.cgls, ocgls) if solver == "cgls" else (ct.lsqr, olsqr)
    x, rep = run(g, torch.from_numpy(b).cuda(), max_iter=10, precond=precond)
    ref = oref(oracle.Operator(og), b.astype(np.float64), K=10, left=left, right=right)
    assert rep.iterations == 10
    assert rel(x.cpu().numpy(), ref.x) < TOL_X
    np.testing.assert_allclose(rep.history, ref.history, rtol=TOL_X)


@pytest.mark.parametrize("precond", ["none", "rowcol"])
def test_deterministic_solvers_bitwise_and_parity(ct, small, precond):
    cfg, og, _, b = small
    g = ct.Geometry(**cfg, deterministic=True)
    bd = torch.from_numpy(b).cuda()
    for solver, osolver in ((ct.cgls, ocgls), (ct.lsqr, olsqr)):
        x1, r1 = solver(g, bd, max_iter=12, precond=precond)
        x2, r2 = solver(g, bd, max_iter=12, precond=precond)
        assert torch.equal(x1, x2) and r1.history == r2.history
        left, right = (None, None) if precond == "none" else rowcol_weights(og)
        ref = osolver(oracle.Operator(og), b.astype(np.float64), K=12, left=left, right=right)
        assert rel(x1.cpu().numpy(), ref.x) < TOL_X


@pytest.mark.parametrize("precond", ["none", "jacobi", "rowcol"])
def test_cgls_tikhonov(ct, small, precond):
    """Tikhonov-regularised CGLS (Software section): ||L (A x - b)||^2 +
    lam ||x||^2 against the oracle; lam = a tenth of the mean of diag(A^T A),
    large enough to change the result.  The unweighted case starts from a
    nonzero x0.  FP16 Krylov storage keeps its usual bound."""
    cfg, og, _, b = small
    g = ct.Geometry(**cfg)
    lam = 0.1 * float(oracle.backproject(og, np.ones(og.sino_shape), power=2).mean())
    left = right = None
    if precond == "jacobi":
        right = jacobi_weights(og)
    elif precond == "rowcol":
        left, right = rowcol_weights(og)
    x0 = synth.random_field(g.vol_shape, seed=7) * 0.05 if precond == "none" else None
    op, b64 = oracle.Operator(og), b.astype(np.float64)
    ref = ocgls(op, b64, x0=None if x0 is None else x0.astype(np.float64), K=12, left=left,
                right=right, tikhonov=lam)
    ref0 = ocgls(op, b64, x0=None if x0 is None else x0.astype(np.float64), K=12, left=left,
                 right=right)
    assert rel(ref.x, ref0.x) > 1e-2
    bd = torch.from_numpy(b).cuda()
    x0d = None if x0 is None else torch.from_numpy(x0).cuda()
    x, rep = ct.cgls(g, bd, x0=x0d, max_iter=12, precond=precond, tikhonov=lam)
    assert rel(x.cpu().numpy(), ref.x) < TOL_X
    np.testing.assert_allclose(rep.history, ref.history, rtol=TOL_X)
    xh, _ = ct.cgls(g, bd, x0=x0d, max_iter=12, precond=precond, tikhonov=lam, storage="f16")
    assert rel(xh.cpu().numpy(), ref.x) < 3e-3
    with pytest.raises(RuntimeError, match="CT_ERR_INVALID_ARG"):
        ct.cgls(g, bd, max_iter=2, tikhonov=-1.0)


@pytest.mark.parametrize("relax", [1.0, 1.5])
def test_sirt_psirt(ct, small, relax):
    """SIRT (relax 1) and the PSIRT reading (relax 1.5) against the oracle:
    iterates, the recomputed discrepancy history, operator calls (one A and
    one A^T per update, one more A for a nonzero x0) and the ERR stop."""
    cfg, og, _, b = small
    g = ct.Geometry(**cfg)
    op, b64 = oracle.Operator(og), b.astype(np.float64)
    bd = torch.from_numpy(b).cuda()
    ref = osirt(op, b64, K=8, lam=relax)
    x, rep = ct.sirt(g, bd, max_iter=8, relax=relax)
    assert rep.iterations == 8 and (rep.n_forward, rep.n_back) == (8, 8)
    assert rel(x.cpu().numpy(), ref.x) < TOL_X
    np.testing.assert_allclose(rep.history, ref.history, rtol=TOL_X)
    assert rep.nb0 == pytest.approx(ref.nb0, rel=1e-7)
    assert rep.nb == pytest.approx(ref.nb, rel=TOL_X)
    x0 = synth.random_field(g.vol_shape, seed=8) * 0.05
    ref = osirt(op, b64, K=5, lam=relax, x0=x0.astype(np.float64))
    x, rep = ct.sirt(g, bd, x0=torch.from_numpy(x0).cuda(), max_iter=5, relax=relax)
    assert (rep.n_forward, rep.n_back) == (6, 5)
    assert rel(x.cpu().numpy(), ref.x) < TOL_X
    full = osirt(op, b64, K=20, lam=relax)
    err = 0.5 * (full.history[9] + full.history[10])    # met at the 11th update
    _, rep = ct.sirt(g, bd, max_iter=20, err_tol=err, relax=relax)
    assert rep.iterations == 11 and rep.nb / rep.nb0 <= err
    for bad in (0.0, 2.0, -1.0):
        with pytest.raises(RuntimeError, match="CT_ERR_INVALID_ARG"):
            ct.sirt(g, bd, max_iter=2, relax=bad)


def test_cgls_beats_sirt_and_psirt_on_pr1(ct, pr1):
    """Results section: at equal numbers of projections and backprojections
    CGLS reaches a far smaller discrepancy than SIRT/PSIRT (GPU runs)."""
    cfg, _, _, b = pr1
    g = ct.Geometry(**cfg)
    bd = torch.from_numpy(b).cuda()
    _, rc = ct.cgls(g, bd, max_iter=20)
    _, rs = ct.sirt(g, bd, max_iter=20, relax=1.0)
    _, rp = ct.sirt(g, bd, max_iter=20, relax=1.5)
    assert rc.history[-1] < 0.5 * min(rs.history[-1], rp.history[-1])
    assert all(rs.history[k + 1] <= rs.history[k] * (1 + 1e-6) for k in range(19))


def test_graph_replay_equals_direct_launches(ct, small):
    """Without per-operator timing CGLS and LSQR capture one update as a CUDA
    graph and replay it; with timing they launch every kernel directly.  With
    fixed-point backprojection both give bitwise the same iterates, and the
    launch and operator-call counters count the replayed work like direct
    launches."""
    cfg, _, _, b = small
    g = ct.Geometry(**cfg, deterministic=True)
    bd = torch.from_numpy(b).cuda()
    for kw in (dict(), dict(precond="jacobi"), dict(tikhonov=0.05), dict(storage="bf16")):
        l0 = ct.kernel_launches()
        x1, r1 = ct.cgls(g, bd, max_iter=9, **kw)
        l1 = ct.kernel_launches()
        x2, r2 = ct.cgls(g, bd, max_iter=9, timing=True, **kw)
        l2 = ct.kernel_launches()
        assert torch.equal(x1, x2), kw
        assert r1.history == r2.history and r1.iterations == r2.iterations == 9
        assert l1 - l0 == l2 - l1 > 0
    for kw in (dict(), dict(precond="rowcol")):
        x1, r1 = ct.lsqr(g, bd, max_iter=9, **kw)
        x2, r2 = ct.lsqr(g, bd, max_iter=9, timing=True, **kw)
        assert torch.equal(x1, x2), kw
        assert r1.history == r2.history and (r1.n_forward, r1.n_back) == (r2.n_forward, r2.n_back)


@pytest.mark.parametrize("spread", [0.0, 40.0])
def test_streaming_norms_are_fp64_accurate(ct, small, spread):
    """NB0 = ||b|| comes from the streaming kernels' per-thread FP32-pair sums
    of squares and FP64 block sums: within 1e-12 of the FP64 norm, also for
    zeros and for terms far outside the FP32-pair range (|b| from 1e-20 to
    1e20, which the FP64 side path takes)."""
    cfg = small[0]
    g = ct.Geometry(**cfg)
    rng = np.random.default_rng(5)
    b = rng.uniform(0.0, 1000.0, g.sino_shape) * 10.0 ** rng.uniform(-spread / 2, spread / 2,
                                                                      g.sino_shape)
    b[rng.random(g.sino_shape) < 0.1] = 0.0
    b32 = b.astype(np.float32)
    _, rep = ct.cgls(g, torch.from_numpy(b32).cuda(), max_iter=1)
    want = float(np.sqrt(np.sum(b32.astype(np.float64) ** 2)))
    assert rep.nb0 == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("solver", ["cgls", "lsqr"])
def test_gradient_norm_history(ct, small, solver):
    """history_nr: ||A^T (b - A x_{k-1})|| at the iterate before each update,
    against the same norm of the FP64 oracle's iterates (CGLS computes it;
    LSQR carries the Paige-Saunders estimate, exact in exact arithmetic).
    Batched and resumed CGLS report the same values."""
    cfg, og, _, b = small
    g = ct.Geometry(**cfg)
    K = 10
    fn, ofn = (ct.cgls, ocgls) if solver == "cgls" else (ct.lsqr, olsqr)
    x, rep = fn(g, torch.from_numpy(b).cuda(), max_iter=K)
    op = oracle.Operator(og)
    ref = ofn(op, b.astype(np.float64), K=K, keep_iterates=True)
    prev = [np.zeros(og.vol_shape)] + list(ref.iterates[:-1])
    want = [float(np.linalg.norm(op.AT(b.astype(np.float64) - op.A(xk)))) for xk in prev]
    assert len(rep.history_nr) == K
    np.testing.assert_allclose(rep.history_nr, want, rtol=2e-3 if solver == "cgls" else 1e-2)
    assert want[-1] < 0.5 * want[0]          # the gradient shrinks
    if solver == "cgls":
        bt = ct.Batch()
        j = bt.add(g, torch.from_numpy(b).cuda(), max_iter=K)
        while not bt.done(j):
            bt.step()
        _, rb = bt.result(j)
        bt.close()
        np.testing.assert_allclose(rb.history_nr, rep.history_nr, rtol=1e-5)
        st = ct.CglsState(g)
        st.run(torch.from_numpy(b).cuda(), 4)
        blob = st.to_bytes()
        st.close()
        st2 = ct.CglsState(g)
        st2.from_bytes(blob)
        _, rr = st2.run(torch.from_numpy(b).cuda(), K)
        st2.close()
        np.testing.assert_allclose(rr.history_nr, rep.history_nr, rtol=1e-5)
