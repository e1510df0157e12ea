"""CPU checks of the binding's array checks (_need, _need_host): the
conditions under which an array reaches the library. A stand-in object
plays a device tensor (is_cuda, dtype, shape, device, is_contiguous), so no
GPU is needed; the GPU tests (test_gpu_arguments.py) call the binding."""
import numpy as np
import pytest
import torch

from paper_2107_08145_b300 import _need, _need_host


class FakeDeviceTensor:
    def __init__(self, shape, dtype=torch.float32, index=0, contiguous=True, is_cuda=True):
        self.shape = torch.Size(shape)
        self.dtype = dtype
        self.device = torch.device("cuda", index)
        self.is_cuda = is_cuda
        self._c = contiguous

    def is_contiguous(self):
        return self._c


DEV = torch.device("cuda", 0)


def test_need_accepts_the_exact_array():
    t = FakeDeviceTensor((2, 3, 4))
    assert _need("x", t, (2, 3, 4), torch.float32, DEV) is t
    assert _need("x", t, (2, 3, 4), torch.float32, DEV, contiguous=True) is t
    # a strided input is accepted (the binding copies it); a strided output is not
    s = FakeDeviceTensor((2, 3, 4), contiguous=False)
    assert _need("x", s, (2, 3, 4), torch.float32, DEV) is s
    with pytest.raises(ValueError, match="contiguous"):
        _need("out", s, (2, 3, 4), torch.float32, DEV, contiguous=True)


@pytest.mark.parametrize("bad", [
    FakeDeviceTensor((2, 3, 5)),                      # one element short per row
    FakeDeviceTensor((2, 3, 4), dtype=torch.float64),  # the other precision
    FakeDeviceTensor((2, 3, 4), index=1),              # another GPU
    FakeDeviceTensor((2, 3, 4), is_cuda=False),        # host memory
    torch.zeros((2, 3, 4)),                            # a host tensor
    np.zeros((2, 3, 4), np.float32),                   # not a tensor
    None,
])
def test_need_refuses(bad):
    with pytest.raises(ValueError, match="x must be"):
        _need("x", bad, (2, 3, 4), torch.float32, DEV)


def test_need_host():
    a = np.zeros((3, 4))
    assert _need_host("a", a, (3, 4), np.float64, writable=True) is a
    for bad in (np.zeros((3, 5)), np.zeros((3, 4), np.float32), np.zeros((3, 8))[:, ::2], [[0.0] * 4] * 3):
        with pytest.raises(ValueError, match="a must be"):
            _need_host("a", bad, (3, 4), np.float64)
    ro = np.zeros((3, 4))
    ro.flags.writeable = False
    assert _need_host("a", ro, (3, 4), np.float64) is ro  # inputs may be read-only
    with pytest.raises(ValueError, match="writable"):
        _need_host("a", ro, (3, 4), np.float64, writable=True)
