"""Host-side argument marshalling of the Python binding (no GPU): arrays are converted to the
C types the ABI declares, and a value that would wrap in the conversion is rejected instead of
turning into another valid index or residue code."""
import numpy as np
import pytest

from paper_1908_10574_gb300 import Context


def test_host_conversion_keeps_values():
    x = Context._host(np.array([[1, 2], [3, 4]], dtype=np.int64), np.int32, (-1, 2))
    assert x.dtype == np.int32 and x.flags.c_contiguous and x.tolist() == [[1, 2], [3, 4]]
    y = Context._host(np.arange(20, dtype=np.int64)[::2], np.uint8)
    assert y.dtype == np.uint8 and y.flags.c_contiguous and y.tolist() == list(range(0, 20, 2))
    z = Context._host([0, 3, 9], np.int64)
    assert z.dtype == np.int64 and z.tolist() == [0, 3, 9]
    assert Context._host(np.zeros(0, np.int64), np.uint8).size == 0
    m = Context._host(np.eye(20, dtype=np.int32) * 5 - 1, np.int8, (400,))
    assert m.dtype == np.int8 and m.shape == (400,)
    for labels in (np.array([0.0, 1.0, 0.5]), np.array([True, False]), [0, 1]):
        f = Context._host(labels, np.float32)          # float targets: plain conversion
        assert f.dtype == np.float32 and f.tolist() == np.asarray(labels, np.float32).tolist()


@pytest.mark.parametrize("arr,dtype", [
    (np.array([0, (1 << 32) + 5], dtype=np.int64), np.int32),     # would wrap to 5
    (np.array([-1 - (1 << 31)], dtype=np.int64), np.int32),
    (np.array([3, 259], dtype=np.int64), np.uint8),               # would wrap to residue 3
    (np.array([-1], dtype=np.int32), np.uint8),
    (np.array([200], dtype=np.int32), np.int8),                   # matrix entry out of int8
    (np.array([1.5]), np.int32),
])
def test_host_conversion_rejects_wrapping(arr, dtype):
    with pytest.raises(ValueError):
        Context._host(arr, dtype)
