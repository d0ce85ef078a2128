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
