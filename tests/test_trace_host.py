"""NVTX ranges of the C ABI (tracing), checked without a GPU: an NVTX
injection library (tests/nvtx/nvtx_probe.c, built here with gcc) records
every range the library opens.  Each compute entry point opens a range named
after itself for the whole call, also when it returns an error early, so
calls with a NULL geometry (rejected before any CUDA work) exercise them."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

CHILD = r'''
import ctypes, sys
sys.path.insert(0, %r)
import paper_2110_13526_gb300 as ct
L = ct.lib()
n = ctypes.c_void_p()
assert L.ct_project(None, None, None, ctypes.c_float(1), ctypes.c_float(0), None) == 1
assert L.ct_backproject(None, None, None, ctypes.c_float(1), ctypes.c_float(0), None) == 1
assert L.ct_project_norm2(None, None, None, ctypes.c_float(1), ctypes.c_float(0), None, None) == 1
assert L.ct_cgls(None, None, None, None, None, None) == 1
assert L.ct_lsqr(None, None, None, None, None, None) == 1
assert L.ct_count_nnz(None, None, None) == 1
print("calls done")
'''


def test_entry_points_open_named_ranges(tmp_path):
    if shutil.which("gcc") is None or not os.path.exists(os.path.join(CUDA_INC, "nvtx3")):
        pytest.skip("needs gcc and the CUDA nvtx3 headers")
    import paper_2110_13526_gb300.build as B
    B.build(debug=False)
    so = str(tmp_path / "libnvtx_probe.so")
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-I" + CUDA_INC,
                    os.path.join(ROOT, "tests", "nvtx", "nvtx_probe.c"), "-o", so], check=True)
    log = str(tmp_path / "ranges.log")
    env = dict(os.environ, NVTX_INJECTION64_PATH=so, CT_NVTX_LOG=log)
    r = subprocess.run([sys.executable, "-c", CHILD % ROOT], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0 and "calls done" in r.stdout, r.stdout + r.stderr
    lines = open(log).read().split("\n")
    pushes = [ln[5:] for ln in lines if ln.startswith("push ")]
    assert pushes == ["ct_project", "ct_backproject", "ct_project_norm2", "ct_cgls", "ct_lsqr",
                      "ct_count_nnz"]
    assert sum(ln == "pop" for ln in lines) == len(pushes)
