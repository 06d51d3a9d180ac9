"""Array namespace for the oracle (test infrastructure only).

numpy arrays are computed with numpy.  torch tensors (CPU, float64) are
computed with the same operations from torch, so that running the unchanged
oracle code on tensors that require gradients gives, through autograd, the
exact discrete adjoint of the oracle's step.
"""
import numpy as np


class _TorchNS:
    def __init__(self):
        import torch
        self.t = torch

    def asarray(self, x):
        if isinstance(x, self.t.Tensor):
            return x
        return self.t.as_tensor(np.asarray(x), dtype=self.t.float64)

    def einsum(self, sub, *ops):
        return self.t.einsum(sub, *[self.asarray(o) for o in ops])

    def roll(self, x, shift, axis):
        return self.t.roll(x, shift, dims=axis)

    def maximum(self, a, b):
        return self.t.maximum(a, b)

    def abs(self, x):
        return self.t.abs(x)

    def sqrt(self, x):
        return self.t.sqrt(x)

    def stack(self, xs, axis=0):
        return self.t.stack(list(xs), dim=axis)

    def zeros_like(self, x):
        return self.t.zeros_like(x)

    def ones_like(self, x):
        return self.t.ones_like(x)

    def max(self, x):
        return self.t.max(x)


class _NumpyNS:
    asarray = staticmethod(np.asarray)
    einsum = staticmethod(np.einsum)
    maximum = staticmethod(np.maximum)
    abs = staticmethod(np.abs)
    sqrt = staticmethod(np.sqrt)
    stack = staticmethod(np.stack)
    zeros_like = staticmethod(np.zeros_like)
    ones_like = staticmethod(np.ones_like)
    max = staticmethod(np.max)

    @staticmethod
    def roll(x, shift, axis):
        return np.roll(x, shift, axis=axis)


_NP = _NumpyNS()
_TORCH = None


def xp_of(*arrays):
    global _TORCH
    for a in arrays:
        if type(a).__module__.split(".")[0] == "torch":
            if _TORCH is None:
                _TORCH = _TorchNS()
            return _TORCH
    return _NP
