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


def hist_tolerance_ok(gpu, ref, ref_abs, rel=1e-5, atol=1e-12, slack=0.0):
    """|gpu - ref| <= rel * (sum of |g| of the rows in the bin) + slack elementwise."""
    return np.all(np.abs(gpu - ref) <= rel * ref_abs + slack + atol)


FIXED_ROWS_PER_CTA = 4096   # rows per CTA of the fixed-point histogram kernel's default tiling


def fixed_point_row_error(v64, rows_per_cta=FIXED_ROWS_PER_CTA):
    """Largest rounding error of one row's value in the fixed-point histogram kernel (the
    default, tiles.kernel 7): a CTA of at most rows_per_cta rows takes the scale 2^e with
    1.001 * S < 2^(30-e) <= 2 * 1.001 * S, S the sum of |v| over its rows, and rounds
    v 2^e to floor(v 2^e + u) with a dither u in [0, 1), so the error is below
    2^-e <= 2.002 * S * 2^-30."""
    v = np.abs(np.asarray(v64, np.float64))
    S = min(v.sum(), rows_per_cta * v.max(initial=0.0))
    return 2.002 * S * 2.0 ** -30


def fixed_point_slack(count, g64, h64, chain=2, rows_per_cta=FIXED_ROWS_PER_CTA):
    """Rounding slack of fixed-point histogram cells. count[..., 2]: rows of each cell, or for
    a level below the root the root's rows of the bin: a sibling by subtraction carries its
    parent's rounding, and along a chain of subtractions the directly built children are
    disjoint subsets of the root's rows, so chain = 2 bounds every level."""
    err = np.array([fixed_point_row_error(g64, rows_per_cta), fixed_point_row_error(h64, rows_per_cta)])
    return chain * np.asarray(count, np.float64) * err
