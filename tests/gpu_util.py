"""Helpers shared by the GPU tests (device buffers via torch)."""
import numpy as np
import torch

from paper_2106_07616_gb300 import rbffd

_ctx = None


def ctx():
    global _ctx
    if _ctx is None:
        from paper_2106_07616_gb300 import _build
        _build.build()
        _ctx = rbffd.Context(0)
    return _ctx


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to("cuda:0")


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
