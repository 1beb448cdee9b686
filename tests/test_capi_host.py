"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every symbol include/ct.h declares.  No compute call is made (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2110_13526_gb300 import build
    return build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ct_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("ct_geometry_create", "ct_project", "ct_backproject", "ct_cgls", "ct_lsqr"):
        assert want in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    for name in declared_functions():
        assert hasattr(lib, name), name
    import paper_2110_13526_gb300 as ct
    assert sorted(ct.EXPORTS) == declared_functions()


def test_version_and_error_without_gpu(built_lib):
    import paper_2110_13526_gb300 as ct
    assert ct.version().startswith("ct-gb300")
    L = ct.lib()
    # argument validation happens before any CUDA call
    st = L.ct_geometry_create(None, None)
    assert st == 1 and b"non-NULL" in L.ct_last_error()
    opts = ct.SolverOpts(0, 0.0, 0, 0.0, 0, 0)
    assert L.ct_cgls(None, None, None, ctypes.byref(opts), None, None) == 1
    assert L.ct_project(None, None, None, 1.0, 0.0, None) == 1


def test_bad_geometry_rejected_before_cuda(built_lib):
    import paper_2110_13526_gb300 as ct
    L = ct.lib()
    d = ct._Desc(0, 8, 8, 1, 1, 1, 0, 0, 0, 8, 8, 1, 1, 0, 0, 750, 1200, 4, None)
    h = ctypes.c_void_p()
    assert L.ct_geometry_create(ctypes.byref(d), ctypes.byref(h)) == 1
    d = ct._Desc(8, 8, 8, 1, 1, 1, 0, 0, 0, 8, 8, 1, 1, 0, 0, 1200, 750, 4, None)
    assert L.ct_geometry_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"sid" in L.ct_last_error()
    d = ct._Desc(8, 8, 8, -1, 1, 1, 0, 0, 0, 8, 8, 1, 1, 0, 0, 750, 1200, 4, None)
    assert L.ct_geometry_create(ctypes.byref(d), ctypes.byref(h)) == 1
    # grid limits: nv <= 65535 * 8, nviews and nz <= 65535
    d = ct._Desc(8, 8, 8, 1, 1, 1, 0, 0, 0, 8, 65535 * 8 + 1, 1, 1, 0, 0, 750, 1200, 4, None)
    assert L.ct_geometry_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"nv" in L.ct_last_error()
    d = ct._Desc(8, 8, 8, 1, 1, 1, 0, 0, 0, 8, 8, 1, 1, 0, 0, 750, 1200, 65536, None)
    assert L.ct_geometry_create(ctypes.byref(d), ctypes.byref(h)) == 1
    # the walks' integer lines: nx and ny <= 65535 as well
    d = ct._Desc(65536, 2, 2, 1, 1, 1, 0, 0, 0, 8, 8, 1, 1, 0, 0, 750, 1200, 4, None)
    assert L.ct_geometry_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"nx, ny, nz" in L.ct_last_error()


def test_solver_options_rejected_before_cuda(built_lib):
    import paper_2110_13526_gb300 as ct
    L = ct.lib()
    so = ct.SirtOpts(5, 0.0, 1.0, 0)
    assert L.ct_sirt(None, None, None, ctypes.byref(so), None, None) == 1
    assert b"geometry" in L.ct_last_error()


def test_batch_arguments_rejected_before_cuda(built_lib):
    """ct_batch_*: NULL handles and outputs are argument errors (status 1)
    with a message; destroying NULL is a no-op."""
    import paper_2110_13526_gb300 as ct
    L = ct.lib()
    n = ctypes.c_int32()
    assert L.ct_batch_create(None, None) == 1
    assert L.ct_batch_step(None, ctypes.byref(n)) == 1
    assert b"batch" in L.ct_last_error()
    assert L.ct_batch_poll(None, 1, ctypes.byref(n), None) == 1
    assert L.ct_batch_remove(None, 1) == 1
    assert L.ct_batch_add_cgls(None, None, None, None, None, ctypes.byref(n)) == 1
    assert L.ct_batch_destroy(None) == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2110_13526_gb300 as ct
    monkeypatch.setattr(ct, "_lib", None)
    monkeypatch.setattr(ct, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        ct.lib()
