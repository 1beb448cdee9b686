"""Differentiation through the hand-written projector pair (autograd.Function).

* loss ||A x - b||^2 on the differentiation workload shape (batch of 8 128^3
  volumes, 192x144 detector, 180 views): central finite differences
  (h = 1e-3) on 64 random voxels, and the FP64 oracle gradient 2 A^T (A x - b);
* the unrolled, checkpointed CGLS: its forward equals ct_cgls, and its
  gradient with respect to b passes a finite-difference check.

Finite differences of FP32 projections carry ~1e-3 relative rounding noise
(the two perturbed projections differ only along the rays through the voxel,
by 2h a_ij against sums of a few hundred FP32 terms), hence rtol 2e-2 there.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DIFF = dict(nx=128, ny=128, nz=128, vx=1.0, vy=1.0, vz=1.0, nu=192, nv=144, du=1.6, dv=1.6,
            sid=750.0, sdd=1200.0, nviews=180)


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2110_13526_gb300 as m
    m.lib()
    oracle.build()
    return m


@pytest.fixture(scope="module")
def batch(ct):
    g = ct.Geometry(**DIFF)
    lo, hi = synth.box_of(DIFF)
    xs = [synth.voxelize(synth.random_ellipsoids(20, 100 + i, lo, hi, axis_scale=0.5), DIFF)
          for i in range(8)]
    x_true = torch.from_numpy(np.stack(xs)).cuda()
    from paper_2110_13526_gb300.autograd import A
    with torch.no_grad():
        b = A(g, x_true) + 0.01 * torch.randn(8, *g.sino_shape, device="cuda",
                                              generator=torch.Generator("cuda").manual_seed(4))
    x = x_true + 0.05 * torch.randn(x_true.shape, device="cuda",
                                    generator=torch.Generator("cuda").manual_seed(5))
    return g, x, b


def loss_fn(g, x, b):
    from paper_2110_13526_gb300.autograd import A
    r = A(g, x) - b
    return (r.double() ** 2).sum()


def test_batched_apply_matches_single(ct, batch):
    from paper_2110_13526_gb300.autograd import A, AT
    g, x, b = batch
    y = A(g, x)
    assert torch.equal(y[3], ct.project(g, x[3].contiguous()))
    z = AT(g, b)
    # float-atomic sums: the order of the additions into a voxel varies from
    # launch to launch, so two launches agree to FP32 rounding, not bitwise
    z1 = ct.backproject(g, b[5].contiguous())
    assert ((z[5] - z1).norm() / z1.norm()).item() < 1e-6
    # with fixed-point sums they agree bitwise
    gd = ct.Geometry(**DIFF, deterministic=True)
    assert torch.equal(AT(gd, b)[5], ct.backproject(gd, b[5].contiguous()))


def test_batch_is_one_projector_launch(ct, batch):
    """The 8 items of a batch take one projector launch per operator (plus a
    layout transpose per item for A and a combine per item for A^T)."""
    from paper_2110_13526_gb300.autograd import A, AT
    g, x, b = batch
    torch.cuda.synchronize()
    l0 = ct.kernel_launches()
    A(g, x)
    torch.cuda.synchronize()
    assert ct.kernel_launches() - l0 == 8 + 1
    l0 = ct.kernel_launches()
    AT(g, b)
    torch.cuda.synchronize()
    assert ct.kernel_launches() - l0 == 1 + 8


def test_batch_entry_points_alpha_beta_and_fallback(ct):
    """alpha/beta epilogues of the batched entry points, and geometries that
    run item by item (rays advancing along z: ray-major kernels)."""
    for cfg in (dict(nx=20, ny=18, nz=14, vx=1.0, vy=1.0, vz=1.0, nu=30, nv=40, du=1.0, dv=1.0,
                     sid=120.0, sdd=200.0, nviews=7),
                dict(nx=16, ny=16, nz=40, vx=1.0, vy=1.0, vz=1.0, nu=24, nv=70, du=1.5, dv=2.5,
                     sid=30.0, sdd=60.0, nviews=5)):
        g = ct.Geometry(**cfg)
        x = torch.from_numpy(synth.random_field((3,) + g.vol_shape, seed=50)).cuda()
        y0 = torch.from_numpy(synth.random_field((3,) + g.sino_shape, seed=51)).cuda()
        out = y0.clone()
        ct.project_batch(g, x, out=out, alpha=-0.5, beta=2.0)
        for i in range(3):
            want = ct.project(g, x[i].contiguous(), out=y0[i].clone(), alpha=-0.5, beta=2.0)
            assert torch.equal(out[i], want)
        v0 = torch.from_numpy(synth.random_field((3,) + g.vol_shape, seed=52)).cuda()
        vout = v0.clone()
        ct.backproject_batch(g, y0, out=vout, alpha=0.25, beta=-1.0)
        for i in range(3):
            want = ct.backproject(g, y0[i].contiguous(), out=v0[i].clone(), alpha=0.25, beta=-1.0)
            assert ((vout[i] - want).norm() / want.norm()).item() < 1e-6


def test_finite_differences_64_voxels(ct, batch):
    g, x, b = batch
    xg = x.clone().requires_grad_(True)
    loss_fn(g, xg, b).backward()
    grad = xg.grad
    rng = np.random.default_rng(6)
    flat = grad.reshape(-1)
    # voxels inside the field of view (nonzero gradient), random batch items
    cand = torch.nonzero(flat.abs() > 1e-3 * flat.abs().max()).flatten().cpu().numpy()
    picks = rng.choice(cand, size=64, replace=False)
    h = 1e-3
    fd, ad = [], []
    with torch.no_grad():
        for j in picks:
            xp = x.clone().reshape(-1)
            xp[j] += h
            lp = loss_fn(g, xp.reshape(x.shape), b).item()
            xp[j] -= 2 * h
            lm = loss_fn(g, xp.reshape(x.shape), b).item()
            fd.append((lp - lm) / (2 * h))
            ad.append(flat[j].item())
    fd, ad = np.array(fd), np.array(ad)
    assert np.linalg.norm(fd - ad) / np.linalg.norm(ad) < 2e-2
    assert np.all(np.abs(fd - ad) <= 2e-2 * np.abs(ad) + 1e-3 * np.abs(ad).max())


def test_gradient_matches_fp64_oracle(ct, batch):
    """d/dx ||A x - b||^2 = 2 A^T (A x - b), item 0 against the FP64 oracle."""
    g, x, b = batch
    xg = x.clone().requires_grad_(True)
    loss_fn(g, xg, b).backward()
    og = oracle.OGeom(**DIFF)
    x0 = x[0].cpu().double().numpy()
    r = oracle.project(og, x0) - b[0].cpu().double().numpy()
    want = 2.0 * oracle.backproject(og, r)
    got = xg.grad[0].cpu().double().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5


def test_unrolled_cgls_forward_and_gradient(ct):
    from paper_2110_13526_gb300.autograd import unrolled_cgls
    cfg = dict(nx=24, ny=20, nz=16, vx=1.0, vy=1.0, vz=1.0, nu=36, nv=24, du=1.0, dv=1.0,
               sid=200.0, sdd=320.0, nviews=20)
    g = ct.Geometry(**cfg)
    lo, hi = synth.box_of(cfg)
    xt = torch.from_numpy(synth.voxelize(synth.random_ellipsoids(5, 7, lo, hi,
                                                                 axis_range=(3.0, 8.0)), cfg)).cuda()
    b = ct.project(g, xt)
    x_lib, _ = ct.cgls(g, b, max_iter=10)
    bb = b.clone().requires_grad_(True)
    x_ad = unrolled_cgls(g, bb, K=10)
    rel = (x_ad.detach() - x_lib).norm() / x_lib.norm()
    assert rel.item() < 1e-4
    w = torch.from_numpy(synth.random_field(g.vol_shape, seed=8)).cuda()
    (x_ad * w).sum().backward()
    grad = bb.grad.reshape(-1)
    rng = np.random.default_rng(9)
    idx = rng.choice(np.nonzero(b.reshape(-1).cpu().numpy() > 0.1)[0], size=16, replace=False)
    h = 1e-2
    with torch.no_grad():
        for j in idx:
            bp = b.clone().reshape(-1)
            bp[j] += h
            fp = (unrolled_cgls(g, bp.reshape(b.shape), K=10).double() * w).sum().item()
            bp[j] -= 2 * h
            fm = (unrolled_cgls(g, bp.reshape(b.shape), K=10).double() * w).sum().item()
            fd = (fp - fm) / (2 * h)
            assert fd == pytest.approx(grad[j].item(), rel=5e-2, abs=5e-3 * grad.abs().max().item())
