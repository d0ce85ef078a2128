"""Pins of the oracle's histogram, split search, leaf index, leaf values and
boosting loop (Sections 3 and 4) against closed forms, library routines and
exhaustive enumeration from raw rows."""
import itertools

import numpy as np
import pytest

import oracle
from conftest import golden_directives, golden_rows
from paper_1810_11363_gb300 import synth


def _case(seed=0, n=2000, F=6, F_pad=16, max_bins=33, depth=3):
    bins, nb, g, h, forced = synth.random_level_case(seed, n, F, F_pad, max_bins, depth)
    return bins, nb, g.astype(np.float64), h.astype(np.float64), forced


def test_histogram_counts_equal_bincount():
    bins, nb, g, h, _ = _case()
    n, F = bins.shape[0], nb.shape[0]
    rng = np.random.default_rng(1)
    leaf = rng.integers(0, 4, n).astype(np.uint16)
    mb = int(nb.max()) + 1
    hist = oracle.histogram(bins, F, np.ones(n), np.ones(n), leaf, 4, mb)
    for l in range(4):
        for f in range(F):
            want = np.bincount(bins[leaf == l, f], minlength=mb)
            assert np.array_equal(hist[l, f, :, 0], want)
            assert np.array_equal(hist[l, f, :, 1], want)


def test_histogram_conservation():
    bins, nb, g, h, _ = _case(seed=2)
    n, F = bins.shape[0], nb.shape[0]
    leaf = np.random.default_rng(3).integers(0, 8, n).astype(np.uint16)
    mb = int(nb.max()) + 1
    hist = oracle.histogram(bins, F, g, h, leaf, 8, mb)
    tot = oracle.leaf_totals(g, h, leaf, 8)
    for f in range(F):
        assert np.allclose(hist[:, f].sum(axis=1), tot, rtol=1e-12, atol=1e-9)
    assert np.allclose(hist.sum(axis=(0, 2))[0], [g.sum(), h.sum()], rtol=1e-12)
    # the leaf totals match a direct numpy reduction
    assert np.allclose(tot[:, 0], np.bincount(leaf, weights=g, minlength=8), rtol=1e-12, atol=1e-12)


def _raw_score(bins, g, h, leaf, n_leaves, f, k, l2):
    """Score of candidate (f, k) from raw rows: for every leaf, sum g and h of the
    rows sent left (bin <= k) and right (bin > k), then G^2/(H+l2) per side."""
    s = 0.0
    for l in range(n_leaves):
        m = leaf == l
        right = bins[:, f] > k
        for side in (m & ~right, m & right):
            G, H = g[side].sum(), h[side].sum()
            s += 0.0 if H + l2 == 0 else G * G / (H + l2)
    return s


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("l2", [0.0, 3.0])
def test_split_search_matches_exhaustive_enumeration(seed, l2):
    # <= 12 rows: at every level enumerate every (f, k) and score it from the raw
    # rows, with no histogram; the oracle must pick the same split and score.
    rng = np.random.default_rng(seed)
    n, F, depth = 12, 3, 3
    nb = np.array([3, 1, 5], np.int32)
    bins = np.zeros((n, 16), np.uint8)
    for f in range(F):
        bins[:, f] = rng.integers(0, nb[f] + 1, n)
    y = rng.normal(size=n).astype(np.float32)
    res = oracle.fit(bins, F, nb, y, "rmse", depth, 1, 1.0, l2)
    g = -y.astype(np.float64)                   # RMSE gradient at pred 0
    h = np.ones(n)
    leaf = np.zeros(n, np.int64)
    for d in range(depth):
        cands = [(f, k) for f in range(F) for k in range(nb[f])]
        scores = [_raw_score(bins, g, h, leaf, 1 << d, f, k, l2) for f, k in cands]
        best = max(range(len(cands)), key=lambda i: (scores[i], -cands[i][0], -cands[i][1]))
        srt = sorted(scores, reverse=True)
        if srt[0] - srt[1] > 1e-9 * abs(srt[0]):
            assert (res["split_f"][0, d], res["split_k"][0, d]) == cands[best]
        assert res["score"][0, d] == pytest.approx(srt[0], rel=1e-12)
        assert res["second"][0, d] == pytest.approx(srt[1], rel=1e-12)
        f, k = int(res["split_f"][0, d]), int(res["split_k"][0, d])
        leaf += (bins[:, f] > k).astype(np.int64) << d


def test_depth1_rmse_is_the_least_squares_mean_split():
    # lambda = 0, RMSE from pred 0: the best split minimises the summed squared
    # error around the two side means, and the leaf values are those means.
    rng = np.random.default_rng(7)
    n, F = 400, 4
    nb = np.array([10, 7, 3, 12], np.int32)
    bins = np.zeros((n, 16), np.uint8)
    for f in range(F):
        bins[:, f] = rng.integers(0, nb[f] + 1, n)
    y = (bins[:, 1] > 3) * 2.0 + rng.normal(0, 0.5, n)
    y = y.astype(np.float32)
    res = oracle.fit(bins, F, nb, y, "rmse", 1, 1, 1.0, 0.0)
    best, best_sse = None, np.inf
    for f in range(F):
        for k in range(nb[f]):
            r = bins[:, f] > k
            sse = np.var(y[~r]) * (~r).sum() + np.var(y[r]) * r.sum()
            if sse < best_sse - 1e-9:
                best, best_sse = (f, k), sse
    assert (res["split_f"][0, 0], res["split_k"][0, 0]) == best
    f, k = best
    r = bins[:, f] > k
    assert res["leaf_values"][0, 0] == pytest.approx(np.mean(y[~r].astype(np.float64)), rel=1e-12)
    assert res["leaf_values"][0, 1] == pytest.approx(np.mean(y[r].astype(np.float64)), rel=1e-12)
    pred_want = np.where(r, y[r].astype(np.float64).mean(), y[~r].astype(np.float64).mean())
    assert np.allclose(res["pred"], pred_want, rtol=1e-12)


def test_logloss_leaf_values_closed_form_from_zero():
    # From pred 0, g = 1/2 - y and h = 1/4, so v = -sum(1/2 - y) / (n_leaf/4 + l2).
    rng = np.random.default_rng(8)
    n, F, l2 = 1000, 3, 3.0
    nb = np.array([5, 5, 5], np.int32)
    bins = rng.integers(0, 6, size=(n, 16)).astype(np.uint8)
    bins[:, F:] = 0
    y = (rng.random(n) < 0.3).astype(np.float32)
    res = oracle.fit(bins, F, nb, y, "logloss", 2, 1, 1.0, l2)
    leaf = oracle.tree_leaf_index(bins, res["split_f"][0], res["split_k"][0])
    for l in range(4):
        m = leaf == l
        want = -np.sum(0.5 - y[m].astype(np.float64)) / (m.sum() / 4.0 + l2)
        assert res["leaf_values"][0, l] == pytest.approx(want, rel=1e-12, abs=1e-15)


def test_pure_leaves_reach_zero_loss():
    # y is a function of three binary features with weights 4, 2, 1: a depth-3
    # tree with lr 1 and l2 0 makes every leaf pure, so RMSE drops to 0.
    rng = np.random.default_rng(9)
    n = 512
    bits = rng.integers(0, 2, size=(n, 3))
    bins = np.zeros((n, 16), np.uint8)
    bins[:, :3] = bits
    bins[:, 3] = rng.integers(0, 2, n)          # a noise feature
    y = (4 * bits[:, 0] + 2 * bits[:, 1] + bits[:, 2]).astype(np.float32)
    res = oracle.fit(bins, 4, np.array([1, 1, 1, 1], np.int32), y, "rmse", 3, 1, 1.0, 0.0)
    assert res["losses"][0] == pytest.approx(0.0, abs=1e-12)
    assert sorted(res["split_f"][0].tolist()) == [0, 1, 2]


def test_leaf_index_encoding_hand_worked():
    splits = golden_directives("leaf_index_example.txt", "S")
    feats = [int(s[1]) for s in splits]
    borders = [int(s[2]) for s in splits]
    rows = golden_rows("leaf_index_example.txt")
    bins = np.zeros((len(rows), 16), np.uint8)
    for i, r in enumerate(rows):
        bins[i, :3] = [int(v) for v in r[:3]]
    want = [int(r[3]) for r in rows]
    assert oracle.tree_leaf_index(bins, feats, borders).tolist() == want
    leaf = np.zeros(len(rows), np.uint16)
    for d, (f, k) in enumerate(zip(feats, borders)):
        leaf = oracle.update_leaf(bins, f, k, d, leaf)
    assert leaf.tolist() == want


def test_apply_reproduces_build_leaf_indices():
    bins, nb, g, h, _ = _case(seed=4, n=3000, depth=4)
    y = np.random.default_rng(4).normal(size=bins.shape[0]).astype(np.float32)
    res = oracle.fit(bins, nb.shape[0], nb, y, "rmse", 4, 3, 0.1, 3.0)
    pred = np.zeros(bins.shape[0])
    for t in range(3):
        leaf = oracle.tree_leaf_index(bins, res["split_f"][t], res["split_k"][t])
        pred = oracle.apply_leaf_values(leaf, res["leaf_values"][t], 0.1, pred)
    assert np.allclose(pred, res["pred"], rtol=0, atol=1e-12)


def test_no_candidate_leaves_rows_in_place():
    n = 50
    bins = np.zeros((n, 16), np.uint8)
    y = np.random.default_rng(0).normal(size=n).astype(np.float32)
    res = oracle.fit(bins, 2, np.array([0, 0], np.int32), y, "rmse", 2, 1, 1.0, 0.0)
    assert res["split_f"][0].tolist() == [-1, -1]
    assert res["leaf_values"][0, 0] == pytest.approx(float(np.mean(y.astype(np.float64))), rel=1e-12)
    assert np.all(res["leaf_values"][0, 1:] == 0)


def test_boosting_decreases_training_loss():
    w = synth.rmse_10k(n=3000)
    prep = oracle.preprocess(w, 16)
    res = oracle.fit(prep["bins"], w.n_features, prep["n_borders"], w.y, w.loss, w.depth, 10,
                     w.lr, w.l2)
    assert np.all(np.diff(res["losses"]) < 0)


def test_split_score_ties_go_to_smallest_feature_then_border():
    # Two identical features: every score ties, the first feature must win.
    n = 64
    rng = np.random.default_rng(1)
    col = rng.integers(0, 4, n)
    bins = np.zeros((n, 16), np.uint8)
    bins[:, 0] = col
    bins[:, 1] = col
    y = rng.normal(size=n).astype(np.float32)
    res = oracle.fit(bins, 2, np.array([3, 3], np.int32), y, "rmse", 1, 1, 1.0, 3.0)
    assert res["split_f"][0, 0] == 0
    assert res["second"][0, 0] == res["score"][0, 0]


def _fit_case(seed=4, n=3000, F=5, max_bins=17, depth=3, trees=4):
    rng = np.random.default_rng(seed)
    bins = rng.integers(0, max_bins, size=(n, 16)).astype(np.uint8)
    bins[:, F:] = 0
    nb = np.full(F, max_bins - 1, np.int32)
    y = (rng.random(n) < 1 / (1 + np.exp(-(bins[:, 0] / 8.0 - 1 + (bins[:, 2] > 9))))).astype(np.float32)
    return bins, nb, y, depth, trees


def test_following_its_own_splits_changes_nothing():
    bins, nb, y, D, T = _fit_case()
    a = oracle.fit(bins, nb.size, nb, y, "logloss", D, T, 0.1, 3.0)
    b = oracle.fit(bins, nb.size, nb, y, "logloss", D, T, 0.1, 3.0, follow=(a["split_f"], a["split_k"]))
    assert np.all(b["followed"] == 0)
    assert np.array_equal(a["pred"], b["pred"])
    assert np.array_equal(a["leaf_values"], b["leaf_values"])


def test_a_duplicate_column_is_an_exact_tie_that_the_lock_step_follows():
    """Feature 5 is a copy of feature 0, so every split on one scores exactly like the
    same split on the other: the oracle takes the smaller feature, and told to follow the
    copy it does so (flag 1) and reaches the same predictions (the rows go the same way)."""
    bins, nb, y, D, T = _fit_case()
    bins[:, 5] = bins[:, 0]
    nb = np.append(nb, nb[0]).astype(np.int32)
    a = oracle.fit(bins, 6, nb, y, "logloss", D, T, 0.1, 3.0)
    assert np.any(a["split_f"] == 0)
    ff = np.where(a["split_f"] == 0, 5, a["split_f"])
    b = oracle.fit(bins, 6, nb, y, "logloss", D, T, 0.1, 3.0, follow=(ff, a["split_k"]))
    assert np.array_equal(b["split_f"], ff)
    assert np.array_equal(b["followed"], (a["split_f"] == 0).astype(np.int32))
    assert np.array_equal(a["score"], b["score"])
    assert np.array_equal(a["pred"], b["pred"])


def test_a_clearly_worse_split_is_flagged_and_not_followed():
    bins, nb, y, D, T = _fit_case()
    a = oracle.fit(bins, nb.size, nb, y, "logloss", D, T, 0.1, 3.0)
    ff = a["split_f"].copy()
    fk = a["split_k"].copy()
    fk[1, 0] = 0 if fk[1, 0] != 0 else 1            # the root split of tree 1 moved to another border
    b = oracle.fit(bins, nb.size, nb, y, "logloss", D, T, 0.1, 3.0, follow=(ff, fk))
    assert b["followed"][1, 0] == -1
    assert np.all(np.delete(b["followed"].ravel(), D) == 0)
    assert np.array_equal(a["pred"], b["pred"])


def test_a_followed_split_drives_the_leaves_and_values():
    """With a margin that admits any split, the followed structure is taken at every
    level, and the predictions equal the leaf values of that structure computed from
    the definitions (leaf index, FP64 totals, Newton step) tree by tree."""
    bins, nb, y, D, T = _fit_case(trees=3)
    rng = np.random.default_rng(7)
    ff = rng.integers(0, nb.size, size=(T, D)).astype(np.int32)
    fk = rng.integers(0, nb[0], size=(T, D)).astype(np.int32)
    b = oracle.fit(bins, nb.size, nb, y, "logloss", D, T, 0.1, 3.0, follow=(ff, fk), follow_tol=1e9)
    assert np.array_equal(b["split_f"], ff) and np.array_equal(b["split_k"], fk)
    assert np.all(b["followed"] >= 0)
    pred = np.zeros(y.size)
    for t in range(T):
        g, h = oracle.gradients("logloss", y, pred)
        leaf = oracle.tree_leaf_index(bins, ff[t], fk[t])
        v = oracle.leaf_values(oracle.leaf_totals(g, h, leaf, 1 << D), 3.0)
        assert np.allclose(b["leaf_values"][t], v, rtol=1e-13, atol=0)
        pred = pred + 0.1 * v[leaf]
    assert np.allclose(b["pred"], pred, rtol=1e-13, atol=1e-15)
