"""The Python binding's argument checks on the CPU: a tensor of the wrong
dtype or shape is refused with TypeError / ValueError before the library is
called, so a mistaken `out` can never be handed to a kernel as a buffer of
the wrong size."""
import pytest
import torch

import paper_2110_13526_gb300 as ct


class _Geom:
    vol_shape = (4, 5, 6)
    sino_shape = (3, 7, 8)
    device = torch.device("cuda", 0)
    handle = None


@pytest.fixture
def no_lib(monkeypatch):
    def _lib():
        raise AssertionError("the library must not be called")
    monkeypatch.setattr(ct, "lib", _lib)
    return _Geom()


def _vol(dtype=torch.float32, shape=_Geom.vol_shape):
    return torch.zeros(shape, dtype=dtype)


def _sino(dtype=torch.float32, shape=_Geom.sino_shape):
    return torch.zeros(shape, dtype=dtype)


@pytest.mark.parametrize("fn", [ct.project, ct.project_norm2])
def test_forward_rejects_bad_volume(no_lib, fn):
    g = no_lib
    with pytest.raises(TypeError, match="vol must be float32"):
        fn(g, _vol(torch.float64))
    with pytest.raises(ValueError, match=r"vol must have shape \(4, 5, 6\)"):
        fn(g, _vol(shape=(4, 6, 5)))


def test_backward_rejects_bad_sinogram(no_lib):
    g = no_lib
    with pytest.raises(TypeError, match="sino must be float32"):
        ct.backproject(g, _sino(torch.int32))
    with pytest.raises(ValueError, match=r"sino must have shape \(3, 7, 8\)"):
        ct.backproject(g, _sino(shape=(3, 8, 7)))


def test_typed_storage_only_where_allowed(no_lib):
    g = no_lib
    # project_norm2 and the solvers take FP32 only; the typed entry points
    # also take BF16 / FP16, nothing else
    with pytest.raises(TypeError, match="vol must be float32$"):
        ct.project_norm2(g, _vol(torch.bfloat16))
    with pytest.raises(TypeError, match="float32 / bfloat16 / float16"):
        ct.project(g, _vol(torch.float64))


def test_batched_rejects_bad_items(no_lib):
    g = no_lib
    with pytest.raises(ValueError, match="expected trailing shape"):
        ct._batched(None, g, torch.zeros(2, 4, 5, 7), g.vol_shape, g.sino_shape,
                    "project_batch", 1.0, 0.0, None, None)
    with pytest.raises(ValueError, match="FP32 only"):
        ct._batched(None, g, torch.zeros(2, 4, 5, 6, dtype=torch.float64), g.vol_shape,
                    g.sino_shape, "project_batch", 1.0, 0.0, None, None)
    bad_out = torch.zeros(2, 3, 7, 8)      # a host tensor: refused before any launch
    with pytest.raises(ValueError, match="out must be a contiguous FP32 cuda tensor"):
        ct._batched(None, g, torch.zeros(2, 4, 5, 6), g.vol_shape, g.sino_shape,
                    "project_batch", 1.0, 0.0, bad_out, None)


def test_solvers_reject_bad_right_hand_side(no_lib):
    g = no_lib
    with pytest.raises(ValueError, match=r"b must have shape \(3, 7, 8\)"):
        ct._solve(None, g, _sino(shape=(3, 7, 9)), None, 5, 0.0, "none", 0, False, None)
    with pytest.raises(TypeError, match="b must be float32"):
        ct._solve(None, g, _sino(torch.float16), None, 5, 0.0, "none", 0, False, None)
