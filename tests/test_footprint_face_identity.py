"""The identity behind the footprint backprojection's shared z faces (CPU, FP64).

For a column of voxels, face f (the bottom of voxel f) projects onto the
detector's v axis as the interval [lo_f, hi_f]; both ends grow with z.  The
unit ramp of face f rises linearly from 0 at lo_f to 1 at hi_f and stays 1
above.  Where hi_k <= lo_{k+1}, voxel k's axial footprint (the unit
trapezoid lo_k, hi_k, lo_{k+1}, hi_{k+1}) equals ramp_k - ramp_{k+1}.
Hence, for any row weights su(l) on the detector rows 0..nv-1, with cells
[l - 1/2, l + 1/2]:

    sum_l trap_k(l) su(l) = W_k - W_{k+1} + sum_{l = b_k + 1}^{b_{k+1}} su(l),

where W_f sums the ramp's integral over the cells a_f..b_f that its rise
touches (a_f, b_f the cells holding lo_f and hi_f, clipped to the detector)
and the last term adds the rows wholly above ramp k and not yet above ramp
k + 1.  The kernel computes each W_f once for the two voxels sharing face f.
Checked on random columns, with rows cut off at both detector edges and
with step faces (lo = hi, the TR footprint).
"""
import math

import numpy as np


def _piece(a, b, lo, hi):
    """Integral over [a, b] of the unit ramp lo -> hi (1 above hi)."""
    r = 0.0
    x1, x2 = max(a, lo), min(b, hi)
    if x2 > x1:
        r += (x2 - x1) * (x2 + x1 - 2 * lo) / (2 * (hi - lo))
    x1 = max(a, hi)
    if b > x1:
        r += b - x1
    return r


def _trap_cell(t, a, b):
    """Integral over [a, b] of the unit trapezoid t0 <= t1 <= t2 <= t3."""
    t0, t1, t2, t3 = t
    r = 0.0
    x1, x2 = max(a, t0), min(b, t1)
    if x2 > x1:
        r += (x2 - x1) * (x2 + x1 - 2 * t0) / (2 * (t1 - t0))
    x1, x2 = max(a, t1), min(b, t2)
    if x2 > x1:
        r += x2 - x1
    x1, x2 = max(a, t2), min(b, t3)
    if x2 > x1:
        r += (x2 - x1) * (2 * t3 - x1 - x2) / (2 * (t3 - t2))
    return r


def _column(rng, nfaces, nv, step):
    """Monotone faces whose neighbouring ramps do not overlap."""
    lo = np.empty(nfaces)
    hi = np.empty(nfaces)
    v = rng.uniform(-4.0, 2.0)
    for f in range(nfaces):
        lo[f] = v
        hi[f] = v if step else v + rng.uniform(0.0, 0.9)
        v = hi[f] + rng.uniform(0.05, 2.5)        # the gap keeps hi_k <= lo_{k+1}
    return lo, hi


def test_face_ramp_form_equals_the_trapezoid_sums():
    rng = np.random.default_rng(11)
    worst = 0.0
    for trial in range(400):
        nv = int(rng.integers(1, 40))
        nfaces = int(rng.integers(2, 18))
        step = trial % 4 == 0
        lo, hi = _column(rng, nfaces, nv, step)
        su = rng.standard_normal(nv)
        a = [max(0, math.floor(x + 0.5)) for x in lo]
        b = [min(max(math.floor(x + 0.5), -1), nv - 1) for x in hi]
        W = [sum(_piece(l - 0.5, l + 0.5, lo[f], hi[f]) * su[l] for l in range(a[f], b[f] + 1))
             for f in range(nfaces)]
        for k in range(nfaces - 1):
            assert hi[k] <= lo[k + 1]
            t = (lo[k], hi[k], lo[k + 1], hi[k + 1])
            want = sum(_trap_cell(t, l - 0.5, l + 0.5) * su[l] for l in range(nv))
            got = W[k] - W[k + 1] + sum(su[l] for l in range(max(b[k] + 1, 0), b[k + 1] + 1))
            scale = float(np.abs(su).sum()) + 1e-300
            worst = max(worst, abs(got - want) / scale)
    assert worst < 1e-12


def test_overlapping_ramps_are_not_the_ramp_difference():
    # where hi_k > lo_{k+1} the difference of the two ramps is no longer the
    # unit trapezoid: the kernel then integrates the voxel's own trapezoid
    lo = (0.0, 0.5)
    hi = (1.5, 3.0)
    t = (lo[0], lo[1], hi[0], hi[1])          # sorted breakpoints of the voxel
    for l in range(-1, 5):
        trap = _trap_cell(t, l - 0.5, l + 0.5)
        diff = _piece(l - 0.5, l + 0.5, lo[0], hi[0]) - _piece(l - 0.5, l + 0.5, lo[1], hi[1])
        if l in (0, 1, 2):
            assert abs(trap - diff) > 1e-3
