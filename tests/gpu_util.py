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


def lockstep_check(res, sp_gpu, pred_gpu, lv_gpu=None, pred_atol=1e-4, lv_rtol=1e-4, lv_atol=1e-7, where=""):
    """Compare a GPU boosting run with the oracle run that followed its splits
    (oracle.fit(..., follow=sp_gpu)): no level may have a GPU split that scores below
    the oracle's best by more than the near-tie margin (followed == -1); every split is
    then identical, leaf values agree (if given) and the predictions after the last tree
    are within pred_atol. Returns a small report dict."""
    fl = res["followed"]
    bad = np.argwhere(fl < 0)
    assert bad.size == 0, f"{where}: GPU split outside the near-tie margin at (tree, level) {bad[:8].tolist()}"
    f_ref, k_ref = res["split_f"], res["split_k"]
    assert np.array_equal(sp_gpu["feature"][:f_ref.shape[0]], f_ref), where
    used = f_ref >= 0
    assert np.array_equal(sp_gpu["border"][:f_ref.shape[0]][used], k_ref[used]), where
    rep = {"levels": int(fl.size), "near_ties_followed": int((fl == 1).sum())}
    if lv_gpu is not None:
        lv_ref = res["leaf_values"]
        lv = np.asarray(lv_gpu)[:lv_ref.shape[0]]
        assert np.allclose(lv, lv_ref, rtol=lv_rtol, atol=lv_atol), \
            (where, float(np.max(np.abs(lv - lv_ref) / (np.abs(lv_ref) + lv_atol / lv_rtol))))
        rep["leaf_value_max_rel"] = float(np.max(np.abs(lv - lv_ref) / np.maximum(np.abs(lv_ref), 1e-300)))
    err = np.abs(np.asarray(pred_gpu, np.float64) - res["pred"])
    rep["pred_max_abs"] = float(err.max(initial=0.0))
    assert rep["pred_max_abs"] <= pred_atol, (where, rep)
    return rep


def hist_cell_report(hist, ref, ref_abs, direct_leaves, copied_feature=-1, rel=1e-5, atol=1e-12):
    """Per-cell error of a level's GPU histogram against the FP64 oracle, relative to the
    sum of |g| (|h|) over the cell's own rows. Cells built directly from rows (leaves in
    direct_leaves; at every level except the root the feature of the parent's split is
    copied from the parent instead) must meet rel; the others (siblings obtained by
    subtraction, copied cells) carry their ancestors' rounding and are only reported.
    Returns (worst direct ratio, worst other ratio), ratio = |gpu - fp64| / own sum, over
    cells that have rows."""
    err = np.abs(hist - ref)
    denom = np.maximum(ref_abs, 1e-300)
    # cells without rows of their own (own sum 0) have no relative error to report; a
    # subtracted one may hold rounding residue, which the caller bounds by the root's rows
    ratio = np.where((err <= atol) | (ref_abs == 0), 0.0, err / denom)
    direct = np.zeros(hist.shape[:2], bool)
    direct[list(direct_leaves)] = True
    if copied_feature >= 0:
        direct[:, copied_feature] = False
    d_ratio = ratio[direct]
    o_ratio = ratio[~direct]
    worst_d = float(d_ratio.max(initial=0.0))
    worst_o = float(o_ratio.max(initial=0.0))
    assert np.all(err[direct] <= rel * ref_abs[direct] + atol), ("direct cells", worst_d)
    return worst_d, worst_o


def direct_children(leaf, d):
    """Leaves of level d (d >= 1) that the level builder histograms from their rows: of
    the children p (bin <= k) and p + 2^(d-1) (bin > k) of every parent p, the one with
    fewer rows, ties to p. The root (d = 0) is always direct."""
    if d == 0:
        return [0]
    half = 1 << (d - 1)
    cnt = np.bincount(np.asarray(leaf, np.int64), minlength=2 * half)
    return [p if cnt[p] <= cnt[p + half] else p + half for p in range(half)]
