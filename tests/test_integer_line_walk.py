"""The integer-line crossing rule of the Siddon slab walks (CPU).

A ray's lateral coordinate in voxel units is held as an integer line in
Q.32 fixed point, X(k) = X0 +- k dX at the start of slab k (dX >= 0 the
step per slab); grid planes sit at the multiples of 2^32.  The walks keep
phi, the distance modulo 2^32 from X(k) to the next plane ahead (a plane at
X(k) itself counts, at distance 0), and step it by phi -= dX.  The rule they
rely on: slab k crosses a plane iff phi < dX (the borrow of the
subtraction), at the fraction phi / dX of the slab, and the index of the
voxel the slab starts in moves by one exactly then.  A plane exactly at the
start of a slab is crossed in that slab, at fraction 0; one exactly at its
end belongs to the next slab.  Every step is an exact integer operation, so
nothing drifts: after any number of slabs phi equals the distance computed
afresh from X0 +- k dX.  Checked against exact rational arithmetic on
random lines in both directions, with dX = 0, lines starting on a plane and
steps close to 2^32.
"""
from fractions import Fraction

import numpy as np

M = 1 << 32


def _walk(X0, dX, up, nslabs):
    """The walks' recurrence: (crossing, fraction, voxel index, phi) per slab."""
    phi = (-X0) % M if up else X0 % M
    idx = (X0 - 1) >> 32 if up else X0 >> 32      # a start on a plane: the voxel behind it
    out = []
    for _ in range(nslabs):
        cross = phi < dX
        out.append((cross, Fraction(phi, dX) if cross else None, idx, phi))
        phi = (phi - dX) % M
        if cross:
            idx += 1 if up else -1
    return out


def _exact(X0, dX, up, k):
    """The same quantities from the line itself, in exact arithmetic."""
    s = 1 if up else -1
    a, b = X0 + s * k * dX, X0 + s * (k + 1) * dX
    if up:
        p = a + (-a) % M            # first plane at or above the start
        cross = a <= p < b
        idx = (a - 1) // M
    else:
        p = a - a % M               # first plane at or below the start
        cross = b < p <= a
        idx = a // M
    frac = Fraction(abs(p - a), dX) if cross else None
    return cross, frac, idx, abs(p - a)


def test_crossing_rule_matches_exact_lines():
    rng = np.random.default_rng(5)
    cases = [(0, 0), (0, 1), (M, M - 1), (5 * M, M - 1), (123, 0), (-7 * M + 3, 2 ** 31),
             (M - 1, 1), (M - 1, 2), (-M, 3), (1, M - 1)]
    for _ in range(300):
        cases.append((int(rng.integers(-(1 << 40), 1 << 40)), int(rng.integers(0, M))))
    crossings = 0
    for X0, dX in cases:
        for up in (True, False):
            for k, (cross, frac, idx, phi) in enumerate(_walk(X0, dX, up, 40)):
                ecross, efrac, eidx, ephi = _exact(X0, dX, up, k)
                assert phi == ephi, (X0, dX, up, k)         # no drift after k steps
                assert cross == ecross, (X0, dX, up, k)
                assert idx == eidx, (X0, dX, up, k)
                if cross:
                    crossings += 1
                    assert frac == efrac and 0 <= frac < 1
    assert crossings > 1000


def test_line_starting_on_a_plane():
    # the first slab crosses that plane at fraction 0: the ray starts in the
    # voxel behind the plane with a zero-length segment, then moves on
    for up in (True, False):
        cross, frac, idx, phi = _walk(3 * M, M - 1, up, 1)[0]
        assert cross and frac == 0 and phi == 0
        assert idx == (2 if up else 3)
