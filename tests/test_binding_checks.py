"""The Python binding checks every buffer it hands to the C ABI as a raw
pointer (the library reads or writes exactly the documented number of
values there) and refuses a wrong dtype, layout or size with the library's
own argument error, DG_ERR_ARG, before any library call.  CPU-side: these
checks run before the library is loaded."""
import numpy as np
import pytest

from paper_2404_12703_gb300 import dg
from paper_2404_12703_gb300 import workloads as W


def _arg_error(fn, *a, **kw):
    with pytest.raises(dg.DgError) as e:
        fn(*a, **kw)
    assert e.value.code == dg.DG_ERR_ARG
    return str(e.value)


def test_host_arrays():
    a = np.zeros(10)
    assert dg._host_buf(a, 10, "U") is a
    _arg_error(dg._host_buf, a, 11, "U")
    _arg_error(dg._host_buf, a.astype(np.float32), 10, "U")
    _arg_error(dg._host_buf, np.zeros((10, 2))[:, 0], 10, "U")      # strided view


def test_mesh_arrays():
    m = W.box_mesh(3, (3, 3, 3))
    dg._mesh_arrays(m["xyz"], m["corner_vid"], 3)
    assert "xyz" in _arg_error(dg._mesh_arrays, m["xyz"], m["corner_vid"], 4)
    assert "corner_vid" in _arg_error(dg._mesh_arrays, m["xyz"], m["corner_vid"][:-1], 3)
    dg._mesh_arrays(m["xyz"][:0], m["corner_vid"][:0], 3)            # empty: the library refuses it


def test_device_buffers_must_be_cuda_tensors():
    torch = pytest.importorskip("torch")
    t = torch.zeros(12, dtype=torch.float64)                          # a host tensor
    assert "CUDA" in _arg_error(dg._device_buf, t, 12, "U")
    _arg_error(dg._device_buf, np.zeros(12), 12, "U")
    _arg_error(dg.convert_check, t)
    J = torch.zeros((2, 64), dtype=torch.float64)
    _arg_error(dg.kinetic_noalloc, 3, torch.zeros((2, 64, 5), dtype=torch.float64), J)
    _arg_error(dg.kinetic_noalloc, 9, None, J)
