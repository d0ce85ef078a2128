"""Helpers shared by the GPU parity tests (device transfer of seeded inputs)."""
import numpy as np


def to_dev(a, dtype=None):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype == np.uint16:
        a = a.view(np.int16)
    t = torch.from_numpy(a)
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def to_host(t, dtype=None):
    a = t.detach().cpu().numpy()
    return a.view(dtype) if dtype is not None else a


def hist_tolerance_ok(gpu, ref, ref_abs, rel=1e-5, atol=1e-12):
    """|gpu - ref| <= rel * (sum of |g| of the rows in the bin) elementwise."""
    return np.all(np.abs(gpu - ref) <= rel * ref_abs + atol)
