"""Test helpers: move numpy arrays to and from CUDA tensors bit for bit."""
import numpy as np

_VIEW = {np.dtype(np.uint32): np.int32, np.dtype(np.uint16): np.int16,
         np.dtype(np.uint64): np.int64, np.dtype(np.float32): np.float32,
         np.dtype(np.int64): np.int64, np.dtype(np.int32): np.int32,
         np.dtype(np.float64): np.float64}


def dev(a):
    """numpy -> contiguous CUDA tensor with identical bits (unsigned as signed)."""
    import torch
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(_VIEW[a.dtype]).copy()).cuda()


def host(t, dtype):
    """CUDA tensor -> numpy array reinterpreted as `dtype`."""
    return t.detach().cpu().contiguous().numpy().view(dtype)


def bits_equal(a, b):
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    if a.dtype.itemsize != b.dtype.itemsize or a.shape != b.shape:
        return False
    u = {4: np.uint32, 8: np.uint64, 2: np.uint16}[a.dtype.itemsize]
    return np.array_equal(a.view(u), b.view(u))
