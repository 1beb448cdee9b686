"""Python binding of the GB300 (sm_103a) cone-beam CT library (``include/ct.h``).

Argument marshalling only: every step of the operator and of the solvers runs
in the CUDA library ``_build/libct_gb300.so``; PyTorch supplies device
memory and streams.  There is no CPU fallback: without the built library, or
without a CUDA device, every call raises.

    import paper_2110_13526_gb300 as ct
    g = ct.Geometry(nx=256, ny=256, nz=256, vx=1, vy=1, vz=1, nu=384, nv=288,
                    du=1, dv=1, sid=750, sdd=1200, nviews=360)
    sino = ct.project(g, vol)                 # A x      (vol: cuda float32 [nz, ny, nx])
    back = ct.backproject(g, sino)            # A^T b
    x, rep = ct.cgls(g, b, max_iter=50)       # Algorithm 1 (CGLS)
    x, rep = ct.lsqr(g, b, max_iter=50)       # LSQR

CPU tensors passed to ``cgls`` / ``lsqr`` / ``project`` / ``backproject`` are
copied to the device and the result is copied back (the end-to-end path).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# CT_GB300_DEBUG_BOUNDS=1 loads the bounds-checking build (see ct_debug_status).
LIB_PATH = os.path.join(_PKG, "_build", "libct_gb300_debug.so"
                        if os.environ.get("CT_GB300_DEBUG_BOUNDS") == "1" else "libct_gb300.so")

CT_OK = 0
CT_PRECOND_NONE, CT_PRECOND_JACOBI, CT_PRECOND_ROWCOL = 0, 1, 2
# ct_projector: Siddon pixel-centre rays, separable footprints (TR, TT)
PROJECTORS = {"siddon": 0, "sf_tr": 1, "sf_tt": 2}
_PRECOND = {"none": 0, None: 0, "jacobi": 1, "rowcol": 2, 0: 0, 1: 1, 2: 2}
_STATUS = {0: "CT_OK", 1: "CT_ERR_INVALID_ARG", 2: "CT_ERR_CUDA", 3: "CT_ERR_OOM",
           4: "CT_ERR_TIMEOUT", 5: "CT_ERR_INTERNAL"}

# Every symbol include/ct.h declares (checked by the CPU tests).
EXPORTS = ("ct_geometry_create", "ct_geometry_destroy", "ct_geometry_sizes", "ct_project",
           "ct_backproject", "ct_project_norm2", "ct_count_nnz", "ct_precond_weights",
           "ct_cgls", "ct_lsqr", "ct_last_error", "ct_version", "ct_kernel_launches",
           "ct_project_norm2_noalloc", "ct_geometry_set_deterministic", "ct_project_ex",
           "ct_backproject_ex", "ct_sirt", "ct_geometry_set_projector", "ct_batch_create",
           "ct_batch_destroy", "ct_batch_add_cgls", "ct_batch_step", "ct_batch_poll",
           "ct_batch_remove", "ct_project_batch", "ct_backproject_batch",
           "ct_cgls_state_create", "ct_cgls_state_destroy", "ct_cgls_state_iterations",
           "ct_cgls_state_export", "ct_cgls_state_import", "ct_cgls_resume",
           "ct_debug_status", "ct_debug_bounds_build")


class CTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("vz", ctypes.c_double),
                ("off_x", ctypes.c_double), ("off_y", ctypes.c_double),
                ("off_z", ctypes.c_double),
                ("nu", ctypes.c_int32), ("nv", ctypes.c_int32),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("det_off_u", ctypes.c_double), ("det_off_v", ctypes.c_double),
                ("sid", ctypes.c_double), ("sdd", ctypes.c_double),
                ("nviews", ctypes.c_int32),
                ("angles_rad", ctypes.POINTER(ctypes.c_double))]


class SirtOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("err_tol", ctypes.c_double),
                ("relax", ctypes.c_double), ("timing", ctypes.c_int32)]


class SolverOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("err_tol", ctypes.c_double),
                ("precond", ctypes.c_int32), ("tikhonov_lambda", ctypes.c_double),
                ("recompute_every", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("storage", ctypes.c_int32)]


class _Report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("nb0", ctypes.c_double),
                ("nb", ctypes.c_double), ("history_nb", ctypes.POINTER(ctypes.c_double)),
                ("history_cap", ctypes.c_int32), ("n_forward", ctypes.c_int32),
                ("n_back", ctypes.c_int32), ("ms_forward", ctypes.c_double),
                ("ms_back", ctypes.c_double), ("history_nr", ctypes.POINTER(ctypes.c_double))]


@dataclass
class SolveReport:
    iterations: int
    nb0: float
    nb: float
    history: list          # NB / NB0 after each x update
    n_forward: int
    n_back: int
    ms_forward: float
    ms_back: float
    # ||A^T e_b|| at the iterate before each update (CGLS: NR, computed; LSQR:
    # the Paige-Saunders estimate); empty for SIRT
    history_nr: list = field(default_factory=list)


def _new_report(cap: int):
    """A ct_solver_report with host history arrays of cap entries."""
    cap = max(int(cap), 1)
    hist, hist_nr = (ctypes.c_double * cap)(), (ctypes.c_double * cap)()
    dp = ctypes.POINTER(ctypes.c_double)
    rep = _Report(0, 0.0, 0.0, ctypes.cast(hist, dp), cap, 0, 0, 0.0, 0.0,
                  ctypes.cast(hist_nr, dp))
    return rep, hist, hist_nr


def _solve_report(rep, hist, hist_nr, with_nr: bool = True) -> "SolveReport":
    k = rep.iterations
    return SolveReport(k, rep.nb0, rep.nb, list(hist[:k]), rep.n_forward, rep.n_back,
                       rep.ms_forward, rep.ms_back, list(hist_nr[:k]) if with_nr else [])


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is not built; run __graft_entry__.build() or "
                               "python -m paper_2110_13526_gb300.build" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, vp = ctypes.POINTER, ctypes.c_void_p
        sig = {
            "ct_geometry_create": ([P(_Desc), P(vp)], ctypes.c_int),
            "ct_geometry_destroy": ([vp], None),
            "ct_geometry_sizes": ([vp, P(ctypes.c_int64), P(ctypes.c_int64)], ctypes.c_int),
            "ct_project": ([vp, vp, vp, ctypes.c_float, ctypes.c_float, vp], ctypes.c_int),
            "ct_backproject": ([vp, vp, vp, ctypes.c_float, ctypes.c_float, vp], ctypes.c_int),
            "ct_project_batch": ([vp, vp, vp, ctypes.c_int32, ctypes.c_float, ctypes.c_float, vp],
                                 ctypes.c_int),
            "ct_cgls_state_create": ([vp, P(vp)], ctypes.c_int),
            "ct_debug_status": ([], ctypes.c_int),
            "ct_debug_bounds_build": ([], ctypes.c_int32),
            "ct_cgls_state_destroy": ([vp], None),
            "ct_cgls_state_iterations": ([vp, P(ctypes.c_int32)], ctypes.c_int),
            "ct_cgls_state_export": ([vp, vp, ctypes.c_int64, P(ctypes.c_int64)], ctypes.c_int),
            "ct_cgls_state_import": ([vp, vp, ctypes.c_int64], ctypes.c_int),
            "ct_cgls_resume": ([vp, vp, vp, P(SolverOpts), P(_Report), vp, vp], ctypes.c_int),
            "ct_backproject_batch": ([vp, vp, vp, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                      vp], ctypes.c_int),
            "ct_project_norm2": ([vp, vp, vp, ctypes.c_float, ctypes.c_float, vp, vp],
                                 ctypes.c_int),
            "ct_project_norm2_noalloc": ([vp, vp, vp, ctypes.c_float, ctypes.c_float, vp, vp],
                                         ctypes.c_int),
            "ct_count_nnz": ([vp, P(ctypes.c_int64), vp], ctypes.c_int),
            "ct_precond_weights": ([vp, ctypes.c_int32, vp, vp, vp], ctypes.c_int),
            "ct_cgls": ([vp, vp, vp, P(SolverOpts), P(_Report), vp], ctypes.c_int),
            "ct_lsqr": ([vp, vp, vp, P(SolverOpts), P(_Report), vp], ctypes.c_int),
            "ct_sirt": ([vp, vp, vp, P(SirtOpts), P(_Report), vp], ctypes.c_int),
            "ct_geometry_set_projector": ([vp, ctypes.c_int32], ctypes.c_int),
            "ct_last_error": ([], ctypes.c_char_p),
            "ct_version": ([], ctypes.c_char_p),
            "ct_kernel_launches": ([], ctypes.c_int64),
            "ct_geometry_set_deterministic": ([vp, ctypes.c_int32], ctypes.c_int),
            "ct_project_ex": ([vp, vp, ctypes.c_int32, vp, ctypes.c_int32, ctypes.c_float,
                               ctypes.c_float, vp], ctypes.c_int),
            "ct_backproject_ex": ([vp, vp, ctypes.c_int32, vp, ctypes.c_int32, ctypes.c_float,
                                   ctypes.c_float, vp], ctypes.c_int),
            "ct_batch_create": ([vp, P(vp)], ctypes.c_int),
            "ct_batch_destroy": ([vp], ctypes.c_int),
            "ct_batch_add_cgls": ([vp, vp, vp, vp, P(SolverOpts), P(ctypes.c_int32)],
                                  ctypes.c_int),
            "ct_batch_step": ([vp, P(ctypes.c_int32)], ctypes.c_int),
            "ct_batch_poll": ([vp, ctypes.c_int32, P(ctypes.c_int32), P(_Report)],
                              ctypes.c_int),
            "ct_batch_remove": ([vp, ctypes.c_int32], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status: int):
    if status != CT_OK:
        raise CTError(status, lib().ct_last_error().decode("utf-8", "replace"))


def version() -> str:
    return lib().ct_version().decode()


def debug_status() -> None:
    """Raise CTError (CT_ERR_INTERNAL) if the bounds-checking build recorded an
    index out of range since the last call (waits for the current device)."""
    _check(lib().ct_debug_status())


def debug_bounds_build() -> bool:
    return bool(lib().ct_debug_bounds_build())


def kernel_launches() -> int:
    """Kernels this library has launched in this process so far."""
    return int(lib().ct_kernel_launches())


class Geometry:
    """Circular cone-beam scan geometry on the current CUDA device (ct_geometry).

    Lengths in mm.  ``angles`` (radians) defaults to 2 pi k / nviews.
    Volume tensors are float32 [nz, ny, nx]; sinograms float32 [nviews, nv, nu].
    ``projector``: "siddon" (pixel-centre rays), "sf_tr" or "sf_tt" (separable
    footprints averaged over detector cells; ct_geometry_set_projector).
    """

    def __init__(self, nx, ny, nz, vx, vy, vz, nu, nv, du, dv, sid, sdd, nviews,
                 ox=0.0, oy=0.0, oz=0.0, det_off_u=0.0, det_off_v=0.0,
                 angles: Optional[Sequence[float]] = None, device=None,
                 deterministic: bool = False, projector: str = "siddon"):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.nu, self.nv, self.nviews = int(nu), int(nv), int(nviews)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        ang = None
        if angles is not None:
            arr = (ctypes.c_double * int(nviews))(*[float(a) for a in angles])
            ang = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        d = _Desc(self.nx, self.ny, self.nz, float(vx), float(vy), float(vz), float(ox),
                  float(oy), float(oz), self.nu, self.nv, float(du), float(dv),
                  float(det_off_u), float(det_off_v), float(sid), float(sdd), self.nviews, ang)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().ct_geometry_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.deterministic = bool(deterministic)
        if projector not in PROJECTORS:
            raise ValueError("projector must be one of %s" % sorted(PROJECTORS))
        self.projector = projector
        if PROJECTORS[projector] != 0:
            _check(lib().ct_geometry_set_projector(h, PROJECTORS[projector]))
        if deterministic:
            _check(lib().ct_geometry_set_deterministic(h, 1))

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("geometry is closed")
        return self._h

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.nviews, self.nv, self.nu)

    def sizes(self):
        n, m = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ct_geometry_sizes(self.handle, ctypes.byref(n), ctypes.byref(m)))
        return n.value, m.value

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().ct_geometry_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# storage element types (ct_dtype)
DTYPES = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}
_DTYPE_NAMES = {"f32": torch.float32, "float32": torch.float32, "bf16": torch.bfloat16,
                "bfloat16": torch.bfloat16, "f16": torch.float16, "float16": torch.float16}


def _torch_dtype(d):
    if d is None or isinstance(d, torch.dtype):
        return d
    return _DTYPE_NAMES[d]


def _dev(t: torch.Tensor, shape, name: str, device, typed: bool = False) -> torch.Tensor:
    if t.dtype != torch.float32 and not (typed and t.dtype in DTYPES):
        raise TypeError("%s must be float32%s" % (name, " / bfloat16 / float16" if typed else ""))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_cuda:
        t = t.pin_memory().to(device, non_blocking=True) if t.device.type == "cpu" else t.to(device)
    if t.device != device:
        raise ValueError("%s is on %s, geometry on %s" % (name, t.device, device))
    return t.contiguous()


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def project(g: Geometry, vol: torch.Tensor, out: Optional[torch.Tensor] = None,
            alpha: float = 1.0, beta: float = 0.0, stream=None, out_dtype=None) -> torch.Tensor:
    """out = alpha * A vol + beta * out (ct_project; ct_project_ex for BF16/FP16
    storage).  out_dtype (default: vol's dtype) types a new output."""
    host = not vol.is_cuda
    v = _dev(vol, g.vol_shape, "vol", g.device, typed=True)
    if out is None:
        od = _torch_dtype(out_dtype) or v.dtype
        o = torch.empty(g.sino_shape, dtype=od, device=g.device)
    else:
        o = _dev(out, g.sino_shape, "out", g.device, typed=True)
    if v.dtype == torch.float32 and o.dtype == torch.float32:
        _check(lib().ct_project(g.handle, _ptr(v), _ptr(o), float(alpha), float(beta),
                                _stream(stream)))
    else:
        _check(lib().ct_project_ex(g.handle, _ptr(v), DTYPES[v.dtype], _ptr(o), DTYPES[o.dtype],
                                   float(alpha), float(beta), _stream(stream)))
    if out is not None and o.data_ptr() != out.data_ptr():
        out.copy_(o)
        return out
    return o.cpu() if host else o


def project_norm2(g: Geometry, vol: torch.Tensor, out: Optional[torch.Tensor] = None,
                  alpha: float = 1.0, beta: float = 0.0, stream=None):
    """(out, ||out||^2 as a 0-d cuda float64 tensor) (ct_project_norm2)."""
    v = _dev(vol, g.vol_shape, "vol", g.device)
    o = (torch.empty(g.sino_shape, dtype=torch.float32, device=g.device) if out is None
         else _dev(out, g.sino_shape, "out", g.device))
    nrm = torch.empty((), dtype=torch.float64, device=g.device)
    _check(lib().ct_project_norm2(g.handle, _ptr(v), _ptr(o), float(alpha), float(beta),
                                  _ptr(nrm), _stream(stream)))
    if out is not None and o.data_ptr() != out.data_ptr():
        out.copy_(o)
        o = out
    return o, nrm


def backproject(g: Geometry, sino: torch.Tensor, out: Optional[torch.Tensor] = None,
                alpha: float = 1.0, beta: float = 0.0, stream=None,
                out_dtype=None) -> torch.Tensor:
    """out = alpha * A^T sino + beta * out (ct_backproject; ct_backproject_ex for
    BF16/FP16 storage).  out_dtype (default: sino's dtype) types a new output."""
    host = not sino.is_cuda
    s = _dev(sino, g.sino_shape, "sino", g.device, typed=True)
    if out is None:
        od = _torch_dtype(out_dtype) or s.dtype
        o = torch.empty(g.vol_shape, dtype=od, device=g.device)
    else:
        o = _dev(out, g.vol_shape, "out", g.device, typed=True)
    if s.dtype == torch.float32 and o.dtype == torch.float32:
        _check(lib().ct_backproject(g.handle, _ptr(s), _ptr(o), float(alpha), float(beta),
                                    _stream(stream)))
    else:
        _check(lib().ct_backproject_ex(g.handle, _ptr(s), DTYPES[s.dtype], _ptr(o),
                                       DTYPES[o.dtype], float(alpha), float(beta),
                                       _stream(stream)))
    if out is not None and o.data_ptr() != out.data_ptr():
        out.copy_(o)
        return out
    return o.cpu() if host else o


def _batched(fn, g: Geometry, t: torch.Tensor, in_shape, out_shape, name, alpha, beta, out,
             stream):
    if tuple(t.shape[-3:]) != tuple(in_shape):
        raise ValueError("%s: expected trailing shape %s, got %s"
                         % (name, tuple(in_shape), tuple(t.shape)))
    lead = tuple(t.shape[:-3])
    host = not t.is_cuda
    x = t.reshape((-1,) + tuple(in_shape))
    if x.dtype != torch.float32:
        raise ValueError("%s: FP32 only" % name)
    nb = x.shape[0]
    # out is checked before anything moves to the device
    if out is not None and (out.dtype != torch.float32 or not out.is_cuda
                            or not out.is_contiguous()
                            or out.numel() != nb * out_shape[0] * out_shape[1] * out_shape[2]):
        raise ValueError("%s: out must be a contiguous FP32 cuda tensor of %d items"
                         % (name, nb))
    x = x.to(g.device).contiguous()
    if out is None:
        o = torch.empty((nb,) + tuple(out_shape), dtype=torch.float32, device=g.device)
    else:
        o = out
    _check(fn(g.handle, _ptr(x), _ptr(o), int(nb), float(alpha), float(beta), _stream(stream)))
    if out is not None:
        return out
    o = o.reshape(lead + tuple(out_shape))
    return o.cpu() if host else o


def project_batch(g: Geometry, vols: torch.Tensor, out: Optional[torch.Tensor] = None,
                  alpha: float = 1.0, beta: float = 0.0, stream=None) -> torch.Tensor:
    """A applied to every item of vols [..., nz, ny, nx] (ct_project_batch:
    one projector launch over all items for column-major Siddon geometries)."""
    return _batched(lib().ct_project_batch, g, vols, g.vol_shape, g.sino_shape,
                    "project_batch", alpha, beta, out, stream)


def backproject_batch(g: Geometry, sinos: torch.Tensor, out: Optional[torch.Tensor] = None,
                      alpha: float = 1.0, beta: float = 0.0, stream=None) -> torch.Tensor:
    """A^T applied to every item of sinos [..., nviews, nv, nu]
    (ct_backproject_batch)."""
    return _batched(lib().ct_backproject_batch, g, sinos, g.sino_shape, g.vol_shape,
                    "backproject_batch", alpha, beta, out, stream)


def count_nnz(g: Geometry, stream=None) -> int:
    """Nonzeros of A: (ray, voxel) pairs with positive length (ct_count_nnz)."""
    n = ctypes.c_int64()
    _check(lib().ct_count_nnz(g.handle, ctypes.byref(n), _stream(stream)))
    return n.value


def precond_weights(g: Geometry, kind, stream=None):
    """(vol_w, sino_w or None) of CT_PRECOND_JACOBI / CT_PRECOND_ROWCOL."""
    k = _PRECOND[kind]
    vw = torch.empty(g.vol_shape, dtype=torch.float32, device=g.device)
    sw = torch.empty(g.sino_shape, dtype=torch.float32, device=g.device) if k == 2 else None
    _check(lib().ct_precond_weights(g.handle, k, _ptr(vw), _ptr(sw), _stream(stream)))
    return vw, sw


def _solve(fn, g: Geometry, b, x0, max_iter, err_tol, precond, recompute_every, timing,
           stream, storage="f32", tikhonov=0.0):
    host = not b.is_cuda
    bd = _dev(b, g.sino_shape, "b", g.device)
    if x0 is None:
        x = torch.zeros(g.vol_shape, dtype=torch.float32, device=g.device)
    else:
        x = _dev(x0, g.vol_shape, "x0", g.device).clone()
    opts = SolverOpts(int(max_iter), float(err_tol), _PRECOND[precond], float(tikhonov),
                      int(recompute_every), 1 if timing else 0,
                      DTYPES[_torch_dtype(storage)])
    rep, hist, hist_nr = _new_report(max_iter)
    _check(fn(g.handle, _ptr(bd), _ptr(x), ctypes.byref(opts), ctypes.byref(rep),
              _stream(stream)))
    return (x.cpu() if host else x), _solve_report(rep, hist, hist_nr)


def cgls(g: Geometry, b: torch.Tensor, x0: Optional[torch.Tensor] = None, max_iter: int = 20,
         err_tol: float = 0.0, precond="none", recompute_every: int = 0, timing: bool = False,
         stream=None, storage="f32", tikhonov: float = 0.0):
    """CGLS with delayed residual computation (Algorithm 1) -> (x, SolveReport).

    storage ("f32", "bf16", "f16") types the Krylov vectors d_x, e_b, p_b; x,
    the backprojection sums and the FP64 scalars keep their precision.
    tikhonov = lam >= 0 minimises ||L (A x - b)||^2 + lam ||x||^2 (NB stays
    the data discrepancy)."""
    return _solve(lib().ct_cgls, g, b, x0, max_iter, err_tol, precond, recompute_every, timing,
                  stream, storage, tikhonov)


class Batch:
    """Several CGLS solves advanced in lock step (ct_batch): every ``step()``
    performs one x update of each active job, with the projectors of all
    column-major Siddon jobs in one batched launch per operator.  Jobs join
    with ``add`` between steps and leave when their stopping rule fires.

    All work runs on ``stream`` (default: the current stream at creation).
    One host thread at a time."""

    def __init__(self, stream=None):
        self._stream = torch.cuda.current_stream() if stream is None else stream
        self._device = self._stream.device
        h = ctypes.c_void_p()
        with torch.cuda.device(self._device):
            _check(lib().ct_batch_create(ctypes.c_void_p(self._stream.cuda_stream),
                                         ctypes.byref(h)))
        self._h = h
        self._jobs = {}   # id -> (geometry, b, x, host, max_iter)

    def add(self, g: Geometry, b: torch.Tensor, x0: Optional[torch.Tensor] = None,
            max_iter: int = 20, err_tol: float = 0.0, precond="none",
            tikhonov: float = 0.0) -> int:
        """Admit a CGLS job (initialisation and first update run now); returns its id."""
        host = not b.is_cuda
        with torch.cuda.device(self._device), torch.cuda.stream(self._stream):
            bd = _dev(b, g.sino_shape, "b", g.device)
            if x0 is None:
                x = torch.zeros(g.vol_shape, dtype=torch.float32, device=g.device)
            else:
                x = _dev(x0, g.vol_shape, "x0", g.device).clone()
        opts = SolverOpts(int(max_iter), float(err_tol), _PRECOND[precond], float(tikhonov),
                          0, 0, 0)
        jid = ctypes.c_int32(0)
        _check(lib().ct_batch_add_cgls(self.handle, g.handle, _ptr(bd), _ptr(x),
                                       ctypes.byref(opts), ctypes.byref(jid)))
        self._jobs[jid.value] = (g, bd, x, host, int(max_iter))
        return jid.value

    def step(self) -> int:
        """One update of every active job; returns the number still active."""
        n = ctypes.c_int32(0)
        _check(lib().ct_batch_step(self.handle, ctypes.byref(n)))
        return n.value

    def done(self, job: int) -> bool:
        d = ctypes.c_int32(0)
        _check(lib().ct_batch_poll(self.handle, int(job), ctypes.byref(d), None))
        return bool(d.value)

    def result(self, job: int, remove: bool = True):
        """(x, SolveReport) of a finished job (None while it runs); by default
        the job then leaves the batch."""
        _, _, x, host, k = self._jobs[job]
        rep, hist, hist_nr = _new_report(k)
        d = ctypes.c_int32(0)
        _check(lib().ct_batch_poll(self.handle, int(job), ctypes.byref(d), ctypes.byref(rep)))
        if not d.value:
            return None
        r = _solve_report(rep, hist, hist_nr)
        if remove:
            self.remove(job)
        return (x.cpu() if host else x), r

    def remove(self, job: int):
        _check(lib().ct_batch_remove(self.handle, int(job)))
        self._jobs.pop(job, None)

    def cancel(self, job: int) -> torch.Tensor:
        """Stop a job between steps, finished or not: it leaves the batch with
        its pending update applied; returns its x (the iterate after its last
        update)."""
        _, _, x, host, _ = self._jobs[job]
        self.remove(job)
        return x.cpu() if host else x

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("batch is closed")
        return self._h

    def active(self) -> int:
        return sum(not self.done(j) for j in self._jobs)

    def close(self):
        if self._h is not None:
            _check(lib().ct_batch_destroy(self._h))
            self._h = None
            self._jobs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sirt(g: Geometry, b: torch.Tensor, x0: Optional[torch.Tensor] = None, max_iter: int = 20,
         err_tol: float = 0.0, relax: float = 1.0, timing: bool = False, stream=None):
    """SIRT (relax = 1) or PSIRT (relax = 1.5) -> (x, SolveReport) (ct_sirt):
    x += relax C^-1 A^T R^-1 (b - A x); NB = ||b - A x|| of the returned x."""
    host = not b.is_cuda
    bd = _dev(b, g.sino_shape, "b", g.device)
    if x0 is None:
        x = torch.zeros(g.vol_shape, dtype=torch.float32, device=g.device)
    else:
        x = _dev(x0, g.vol_shape, "x0", g.device).clone()
    opts = SirtOpts(int(max_iter), float(err_tol), float(relax), 1 if timing else 0)
    rep, hist, hist_nr = _new_report(max_iter)
    _check(lib().ct_sirt(g.handle, _ptr(bd), _ptr(x), ctypes.byref(opts), ctypes.byref(rep),
                         _stream(stream)))
    return (x.cpu() if host else x), _solve_report(rep, hist, hist_nr, with_nr=False)


class CglsState:
    """A resumable CGLS solve (ct_cgls_state): run(), then run() again with a
    larger max_iter continues it; to_bytes() / from_bytes() checkpoint it to
    host memory (or a file) and back."""

    def __init__(self, g: Geometry):
        self.g = g
        h = ctypes.c_void_p()
        with torch.cuda.device(g.device):
            _check(lib().ct_cgls_state_create(g.handle, ctypes.byref(h)))
        self._h = h

    @property
    def iterations(self) -> int:
        n = ctypes.c_int32()
        _check(lib().ct_cgls_state_iterations(self._h, ctypes.byref(n)))
        return n.value

    def run(self, b: torch.Tensor, max_iter: int, x0: Optional[torch.Tensor] = None,
            err_tol: float = 0.0, precond="none", tikhonov: float = 0.0, stream=None):
        """CGLS until max_iter updates in total (or the stopping rule);
        returns (x, SolveReport over all updates)."""
        g = self.g
        host = not b.is_cuda
        bd = _dev(b, g.sino_shape, "b", g.device)
        x = (torch.zeros(g.vol_shape, dtype=torch.float32, device=g.device) if x0 is None
             else _dev(x0, g.vol_shape, "x0", g.device).clone())
        opts = SolverOpts(int(max_iter), float(err_tol), _PRECOND[precond], float(tikhonov), 0, 0,
                          DTYPES[torch.float32])
        rep, hist, hist_nr = _new_report(max_iter)
        _check(lib().ct_cgls_resume(g.handle, _ptr(bd), _ptr(x), ctypes.byref(opts),
                                    ctypes.byref(rep), self._h, _stream(stream)))
        return (x.cpu() if host else x), _solve_report(rep, hist, hist_nr)

    def to_bytes(self) -> bytes:
        n = ctypes.c_int64()
        _check(lib().ct_cgls_state_export(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().ct_cgls_state_export(self._h, buf, n.value, ctypes.byref(n)))
        return buf.raw

    def from_bytes(self, data: bytes) -> None:
        _check(lib().ct_cgls_state_import(self._h, data, len(data)))

    def close(self):
        if self._h:
            lib().ct_cgls_state_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lsqr(g: Geometry, b: torch.Tensor, x0: Optional[torch.Tensor] = None, max_iter: int = 20,
         err_tol: float = 0.0, precond="none", timing: bool = False, stream=None):
    """LSQR (Paige & Saunders 1982) -> (x, SolveReport); NB is the phi_bar estimate."""
    return _solve(lib().ct_lsqr, g, b, x0, max_iter, err_tol, precond, 0, timing, stream)
