"""FP64 NumPy oracle of the Krylov solvers (test infrastructure only).

Everything here calls the operator through an object with ``A(x)`` and
``AT(y)`` (``oracle.Operator`` for the Siddon oracle, or a dense-matrix
operator in the tiny tests), so each solver reads line by line against the
algorithm it follows.

* ``cgls``  -- Algorithm 1 (CGLS with delayed residual computation), with the
  direction update read as d_x = r_x + beta d_x (the printed line has the two
  terms the other way round, which breaks conjugacy; ``literal_update=True``
  runs the printed form, only to show that it is wrong).  Optional diagonal
  preconditioning: the algorithm is run unchanged on L A W with right-hand
  side L b (left weights L on rays, right weights W on voxels), x = x0 + W y.
  ``tikhonov = lam > 0`` (Software section: Tikhonov regularisation) runs
  the same steps on the stacked system [L A; sqrt(lam) I] x ~ [L b; 0], that
  is it minimises ||L (A x - b)||^2 + lam ||x||^2 (with x = x0 + W y the
  regulariser acts on x itself).  Written out: the gradient is
  r = W (A^T L e - lam x), NP2 = ||L A z||^2 + lam ||z||^2 for the x-space
  direction z = W d, and NB stays the data discrepancy ||L (b - A x)||, so the
  stopping test keeps its meaning.
* ``lsqr``  -- Paige & Saunders (1982) LSQR, cited in Materials and Methods,
  in its standard published form, on the same preconditioned operator.
* ``sirt`` / ``psirt`` -- the classical comparison methods of the Software
  and Results sections.  The paper gives no formula: SIRT is
  x += lam C^-1 A^T R^-1 (b - A x) with R = A 1 and C = A^T 1 (row and column
  sums), lam = 1.  PSIRT (Gregor & Benson 2008) is read as the same update
  over-relaxed with lam = 2 / (1 + eps), inside the (0, 2) interval where the
  iteration converges because the spectrum of C^-1 A^T R^-1 A lies in [0, 1].
  The paper gives no eps; eps = 1/3 (lam = 1.5) is this oracle's choice.
  Steps close to 2 barely damp the eigenvalue-1 mode (the constant vector is
  an eigenvector with eigenvalue exactly 1), so they converge slower than
  SIRT, contradicting the Discussion's ordering (SIRT slower than PSIRT).
  The Discussion also says PSIRT keeps no column-sum vector; the variant that
  drops C for one scalar step lam / sigma_max (sigma_max the largest
  eigenvalue of A^T R^-1 A, power iteration) is ``variant="scalar"``.  It too
  converges slower than SIRT.  PSIRT against the paper's own numbers: parity
  unpinned (its fixed point, the weighted normal equations, is pinned).
* ``inv_sqrt_guarded`` / ``jacobi_weights`` / ``rowcol_weights`` -- the
  preconditioners of the Software and Discussion sections (Jacobi = diagonal
  of A^T A; row/column sums), with tiny sums (cone boundary) mapped to 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np


def _nrm(a) -> float:
    return float(np.sqrt(np.sum(np.asarray(a, dtype=np.float64) ** 2)))


@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    nb: float
    nb0: float
    history: List[float] = field(default_factory=list)   # NB / NB0 after each x update
    iterates: List[np.ndarray] = field(default_factory=list)


def inv_sqrt_guarded(v, rel: float = 1e-6):
    """1/sqrt(v) where v > rel * max(v), else 0 (no data there: cone boundary)."""
    v = np.asarray(v, dtype=np.float64)
    m = float(v.max()) if v.size else 0.0
    out = np.zeros_like(v)
    ok = v > rel * m
    out[ok] = 1.0 / np.sqrt(v[ok])
    return out


def jacobi_weights(g, threads=None):
    """W = diag(A^T A)^(-1/2): the Jacobi preconditioner of the Discussion section."""
    from . import backproject
    ones = np.ones(g.sino_shape)
    return inv_sqrt_guarded(backproject(g, ones, threads, power=2))


def rowcol_weights(g, threads=None):
    """(L, W) = (R^(-1/2), C^(-1/2)), R = A 1 row sums, C = A^T 1 column sums."""
    from . import backproject, project
    R = project(g, np.ones(g.vol_shape), threads)
    C = backproject(g, np.ones(g.sino_shape), threads)
    return inv_sqrt_guarded(R), inv_sqrt_guarded(C)


def cgls(op, b, x0=None, K: int = 20, err: float = 0.0, left=None, right=None,
         literal_update: bool = False, recompute_every: int = 0,
         keep_iterates: bool = False, tikhonov: float = 0.0) -> SolveResult:
    """Algorithm 1, CGLS with delayed residual computation.

    Returns x, the iteration count i (number of x updates, the first one
    before the loop), NB (final discrepancy norm) and NB/NB0 after each update.
    With ``left``/``right`` the same steps run on L A W (see module doc).
    ``recompute_every = k > 0`` replaces the updated discrepancy by b - A x
    every k updates (the reorthogonalisation the Discussion describes).
    ``tikhonov = lam`` adds lam ||x||^2 to the objective (module doc).
    """
    lam = float(tikhonov)
    if lam < 0:
        raise ValueError("tikhonov must be >= 0")
    b = np.asarray(b, dtype=np.float64)
    Lw = None if left is None else np.asarray(left, dtype=np.float64).reshape(b.shape)

    def lmul(y):
        return y if Lw is None else Lw * y

    def A(z):
        return lmul(op.A(z))

    def AT_w(e):
        g = op.AT(lmul(e))
        return g if right is None else np.asarray(right).reshape(g.shape) * g

    def wmul(r):
        return r if right is None else np.asarray(right).reshape(r.shape) * r

    NB0 = _nrm(lmul(b))                                   # NB0 = ||b||
    x0a = None if x0 is None else np.asarray(x0, dtype=np.float64)
    if x0a is None or not np.any(x0a):
        e = lmul(b).copy()                                # p_b = A x0 = 0 (call skipped)
    else:
        e = lmul(b) - A(x0a)                              # p_b = A x ; e_b = b - p_b
    x = np.zeros(op.g.vol_shape) if x0a is None else x0a.reshape(op.g.vol_shape).copy()  # x = x0
    r = AT_w(e) - lam * wmul(x)                           # r_x = A^T e_b (- lam W x)
    d = r.copy()                                          # d_x = r_x
    z = wmul(d)                                           # direction in x-space, W d
    NR2_old = float(np.sum(r * r))                        # NR2_old = ||r_x||^2
    p = A(z)                                              # p_b = A d_x
    NP2 = float(np.sum(p * p)) + lam * float(np.sum(z * z))  # NP2 = ||p_b||^2 (+ lam ||z||^2)
    alpha = NR2_old / NP2 if NP2 > 0 else 0.0             # alpha = NR2_old / NP2
    x = x + alpha * z                                     # x = x + alpha d_x
    e = e - alpha * p                                     # e_b = e_b - alpha p_b
    NB = _nrm(e)                                          # NB = ||e_b||
    i = 1
    res = SolveResult(x=x, iterations=1, nb=NB, nb0=NB0, history=[NB / NB0 if NB0 else 0.0])
    if keep_iterates:
        res.iterates.append(x.copy())
    while (NB / NB0 > err if NB0 > 0 else False) and i < K:
        r = AT_w(e) - lam * wmul(x)                       # r_x = A^T e_b (- lam W x)
        NR2_now = float(np.sum(r * r))                    # NR2_now = ||r_x||^2
        beta = NR2_now / NR2_old if NR2_old > 0 else 0.0  # beta = NR2_now / NR2_old
        if literal_update:
            d = d + beta * r                              # the printed line, for the pin only
        else:
            d = r + beta * d                              # d_x = r_x + beta d_x
        z = wmul(d)
        NR2_old = NR2_now                                 # NR2_old = NR2_now
        p = A(z)                                          # p_b = A d_x
        NP2 = float(np.sum(p * p)) + lam * float(np.sum(z * z))  # NP2 (+ lam ||z||^2)
        alpha = NR2_old / NP2 if NP2 > 0 else 0.0         # alpha = NR2_old / NP2
        x = x + alpha * z                                 # x = x + alpha d_x
        e = e - alpha * p                                 # e_b = e_b - alpha p_b
        i += 1                                            # i = i + 1
        if recompute_every > 0 and i % recompute_every == 0:
            e = lmul(b) - A(x)                            # discrepancy from the solution
        NB = _nrm(e)                                      # NB = ||e_b||
        res.history.append(NB / NB0)
        if keep_iterates:
            res.iterates.append(x.copy())
    res.x, res.iterations, res.nb = x, i, NB
    return res


def lsqr(op, b, x0=None, K: int = 20, err: float = 0.0, left=None, right=None,
         keep_iterates: bool = False) -> SolveResult:
    """LSQR (Paige & Saunders 1982) on L A W, x = x0 + W y.

    NB is the recurrence estimate phibar of ||L (b - A x)||; history holds
    phibar / ||L b|| after each iteration.
    """
    b = np.asarray(b, dtype=np.float64)
    Lw = None if left is None else np.asarray(left, dtype=np.float64).reshape(b.shape)

    def lmul(y):
        return y if Lw is None else Lw * y

    def Aop(y):
        z = y if right is None else np.asarray(right).reshape(y.shape) * y
        return lmul(op.A(z))

    def ATop(u):
        g = op.AT(lmul(u))
        return g if right is None else np.asarray(right).reshape(g.shape) * g

    NB0 = _nrm(lmul(b))
    if x0 is not None and np.any(x0):
        x0 = np.asarray(x0, dtype=np.float64)
        u = lmul(b) - lmul(op.A(x0))                      # beta_1 u_1 = b - A x0
    else:
        x0 = None
        u = lmul(b).copy()
    beta = _nrm(u)
    u = u / beta if beta > 0 else u
    v = ATop(u)                                           # alpha_1 v_1 = A^T u_1
    alpha = _nrm(v)
    v = v / alpha if alpha > 0 else v
    w = v.copy()
    phibar, rhobar = beta, alpha
    y = np.zeros_like(v)
    res = SolveResult(x=None, iterations=0, nb=phibar, nb0=NB0)

    def x_of(yv):
        dx = yv if right is None else np.asarray(right).reshape(yv.shape) * yv
        return dx if x0 is None else x0 + dx

    i = 0
    while i < K and (phibar / NB0 > err if NB0 > 0 else False):
        u = Aop(v) - alpha * u                            # beta u = A v - alpha u
        beta = _nrm(u)
        u = u / beta if beta > 0 else u
        v = ATop(u) - beta * v                            # alpha v = A^T u - beta v
        alpha = _nrm(v)
        v = v / alpha if alpha > 0 else v
        rho = float(np.hypot(rhobar, beta))               # rho = sqrt(rhobar^2 + beta^2)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        y = y + (phi / rho) * w                           # x += (phi / rho) w
        w = v - (theta / rho) * w                         # w = v - (theta / rho) w
        i += 1
        res.history.append(phibar / NB0)
        if keep_iterates:
            res.iterates.append(x_of(y))
    res.x, res.iterations, res.nb = x_of(y), i, phibar
    return res


def sirt(op, b, K: int = 20, lam: float = 1.0, R=None, C=None, x0=None,
         rel_guard: float = 1e-6) -> SolveResult:
    """SIRT: x += lam C^-1 A^T R^-1 (b - A x), R = A 1, C = A^T 1 (guarded)."""
    b = np.asarray(b, dtype=np.float64)
    if R is None:
        R = op.A(np.ones(op.g.vol_shape))
    if C is None:
        C = op.AT(np.ones(op.g.sino_shape))
    Rinv = np.where(R > rel_guard * R.max(), 1.0 / np.where(R > 0, R, 1.0), 0.0)
    Cinv = np.where(C > rel_guard * C.max(), 1.0 / np.where(C > 0, C, 1.0), 0.0)
    return _landweber(op, b, K, lambda g: lam * Cinv * g, Rinv, x0)


def psirt(op, b, K: int = 20, lam: float = 1.5, R=None, C=None, x0=None,
          variant: str = "relaxed", n_power: int = 30, seed: int = 0,
          rel_guard: float = 1e-6) -> SolveResult:
    """PSIRT reading (see module doc).

    ``variant="relaxed"``: x += lam C^-1 A^T R^-1 (b - A x), lam = 2 / (1 + 1/3).
    ``variant="scalar"``:  x += (lam / sigma_max) A^T R^-1 (b - A x), no C,
    sigma_max = largest eigenvalue of A^T R^-1 A by ``n_power`` power steps.
    """
    if variant == "relaxed":
        return sirt(op, b, K=K, lam=lam, R=R, C=C, x0=x0, rel_guard=rel_guard)
    if variant != "scalar":
        raise ValueError("variant must be 'relaxed' or 'scalar'")
    b = np.asarray(b, dtype=np.float64)
    if R is None:
        R = op.A(np.ones(op.g.vol_shape))
    Rinv = np.where(R > rel_guard * R.max(), 1.0 / np.where(R > 0, R, 1.0), 0.0)
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(op.g.vol_shape)
    q /= _nrm(q)
    sigma = 0.0
    for _ in range(n_power):
        q2 = op.AT(Rinv * op.A(q))
        sigma = _nrm(q2)
        q = q2 / sigma
    step = lam / sigma
    return _landweber(op, b, K, lambda g: step * g, Rinv, x0)


def _landweber(op, b, K, precond: Callable, Rinv, x0) -> SolveResult:
    NB0 = _nrm(b)
    x = np.zeros(op.g.vol_shape) if x0 is None else np.array(x0, dtype=np.float64)
    e = b - op.A(x) if np.any(x) else b.copy()
    res = SolveResult(x=x, iterations=0, nb=_nrm(e), nb0=NB0)
    for k in range(K):
        x = x + precond(op.AT(Rinv * e))
        e = b - op.A(x)
        res.history.append(_nrm(e) / NB0)
    res.x, res.iterations, res.nb = x, K, _nrm(e)
    return res


class DenseOperator:
    """A given as an explicit matrix (tiny tests); vectors keep their shapes."""

    def __init__(self, M, vol_shape, sino_shape):
        self.M = np.asarray(M, dtype=np.float64)
        self.vol_shape, self.sino_shape = tuple(vol_shape), tuple(sino_shape)
        self.n_forward = self.n_back = 0

        class _G:
            pass
        self.g = _G()
        self.g.vol_shape, self.g.sino_shape = self.vol_shape, self.sino_shape

    def A(self, x):
        self.n_forward += 1
        return (self.M @ np.asarray(x).ravel()).reshape(self.sino_shape)

    def AT(self, y):
        self.n_back += 1
        return (self.M.T @ np.asarray(y).ravel()).reshape(self.vol_shape)

    @property
    def calls(self):
        return self.n_forward + self.n_back
