"""Pins of the ordered-boosting oracle (Section 3 "Fighting Gradient Bias", Algorithm 1
with the log-scale supporting models M'_i) against what the mathematics fixes:

- the size bound of the supporting values (fewer than 4n per permutation);
- at the first tree every model value is 0, so the ordered gradients are the plain
  ones and the first tree is classic boosting's first tree;
- with one feature of two bins the structure is forced, and for RMSE without L2 each
  Newton step moves a model's value a fraction lr of the way to the mean label of its
  leaf over its own training positions: closed form m (1 - (1 - lr)^T);
- the split score of the second tree recomputed by hand from the rule "position k
  takes its gradient from M'_{floor(log2 k)}, position 0 from the start value";
- M'_i never sees a label at a position >= 2^i (Algorithm 1's defining property);
- each permutation's categorical columns hold that permutation's ordered TS.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_11363_gb300 import synth


def test_sup_size_and_offsets():
    for n, want in [(1, 1), (2, 2), (3, 5), (4, 6), (5, 11), (8, 14), (9, 23)]:
        # i = 0..floor(log2(n-1)), model i holds min(2^(i+1), n) values
        I = int(math.floor(math.log2(n - 1))) if n > 1 else 0
        assert sum(min(2 ** (i + 1), n) for i in range(I + 1)) == want
        assert oracle.ordered_sup_size(n) == want
        off = oracle.ordered_sup_offsets(n)
        assert off[0] == 0 and off[-1] == want and len(off) == I + 2
    for n in [2, 17, 1000, 1 << 20, (1 << 20) + 1, 10_000_000]:
        assert oracle.ordered_sup_size(n) < 4 * n          # the section's bound


def _random_case(seed, n, F, s, max_bin, loss):
    rng = np.random.default_rng(seed)
    bins = np.zeros((s, n, 32), np.uint8)
    base = rng.integers(0, max_bin + 1, size=(n, F))
    for q in range(s):
        bins[q, :, :F] = base
        bins[q, :, F - 1] = rng.integers(0, max_bin + 1, size=n)   # a column that differs per permutation
    nb = np.full(F, max_bin, np.int32)
    y = ((rng.random(n) < 0.4).astype(np.float32) if loss == "logloss"
         else rng.normal(0.5, 2.0, n).astype(np.float32))
    perms = np.stack([oracle.make_permutation(seed + q, n) for q in range(s)])
    return bins, nb, y, perms


@pytest.mark.parametrize("loss", ["logloss", "rmse"])
@pytest.mark.parametrize("s", [1, 3])
def test_first_tree_is_the_classic_first_tree(loss, s):
    bins, nb, y, perms = _random_case(7 + s, 600, 5, s, 6, loss)
    o = oracle.fit_ordered(bins, 5, nb, y, loss, 3, 1, 0.1, 2.0, perms)
    c = oracle.fit(bins[0], 5, nb, y, loss, 3, 1, 0.1, 2.0)
    assert np.array_equal(o["split_f"], c["split_f"]) and np.array_equal(o["split_k"], c["split_k"])
    assert np.array_equal(o["score"], c["score"])
    assert np.array_equal(o["leaf_values"], c["leaf_values"])
    assert np.array_equal(o["pred"], c["pred"])


def _forced_case(seed, n, s, depth):
    """One feature with two bins (one border): every level must split on (0, 0). The
    bin differs per permutation, as a categorical column's would."""
    rng = np.random.default_rng(seed)
    bins = np.zeros((s, n, 32), np.uint8)
    bins[:, :, 0] = rng.integers(0, 2, size=(s, n))
    perms = np.stack([oracle.make_permutation(seed * 31 + q, n) for q in range(s)])
    return bins, np.array([1], np.int32), perms, depth


def _leaf(bin_col, depth):
    # every level splits on (0, 0): leaf bit d is the bin for every d
    return bin_col.astype(np.int64) * ((1 << depth) - 1)


@pytest.mark.parametrize("depth", [1, 2])
@pytest.mark.parametrize("n", [1, 2, 3, 37, 1000])
def test_rmse_supporting_models_closed_form(n, depth):
    s, T, lr = 2, 5, 0.3
    bins, nb, perms, _ = _forced_case(n + depth, n, s, depth)
    y = np.random.default_rng(n).normal(1.0, 3.0, n).astype(np.float32)
    o = oracle.fit_ordered(bins, 1, nb, y, "rmse", depth, T, lr, 0.0, perms)
    assert np.all(o["split_f"] == 0) and np.all(o["split_k"] == 0)
    frac = 1.0 - (1.0 - lr) ** T
    off = oracle.ordered_sup_offsets(n)
    tol = 2e-6 * np.abs(y).max()          # gradients are stored in FP32 after the first tree
    for q in range(s):
        leaf_pos = _leaf(bins[q, perms[q], 0], depth)     # leaf by position of sigma_q
        y_pos = y[perms[q]].astype(np.float64)
        for i in range(len(off) - 1):
            train, held = min(1 << i, n), min(2 << i, n)
            want = np.zeros(held)
            for l in np.unique(leaf_pos[:held]):
                m = leaf_pos[:train] == l
                if m.any():                                  # an empty leaf gets -0/(0+0) := 0
                    want[leaf_pos[:held] == l] = y_pos[:train][m].mean() * frac
            got = o["sup"][q, off[i]:off[i] + held]
            assert np.allclose(got, want, rtol=0, atol=tol), (q, i)
    # the final model: the same law over all rows, leaves on permutation 0's bins
    leaf0 = _leaf(bins[0, :, 0], depth)
    want = np.zeros(n)
    for l in np.unique(leaf0):
        want[leaf0 == l] = y[leaf0 == l].astype(np.float64).mean() * frac
    assert np.allclose(o["pred"], want, rtol=0, atol=tol)


def test_second_tree_score_uses_the_log_scale_model_of_each_position():
    n, s, lr, l2 = 300, 2, 0.5, 0.7
    bins, nb, perms, depth = _forced_case(5, n, s, 1)
    y = np.random.default_rng(1).normal(0.0, 1.0, n).astype(np.float32)
    o = oracle.fit_ordered(bins, 1, nb, y, "rmse", depth, 2, lr, l2, perms)
    # tree 1 takes permutation 1. After tree 0 (all values 0, g = -y, h = 1), model i of
    # permutation 1 holds lr * S_l / (c_l + l2) for its positions, S_l and c_l over its
    # training positions p < 2^i in leaf l (leaves on permutation 1's bins).
    b_pos = bins[1, perms[1], 0].astype(np.int64)
    y_pos = y[perms[1]].astype(np.float64)
    a = np.zeros(n)
    for k in range(1, n):
        i = int(math.floor(math.log2(k)))
        m = b_pos[:1 << i] == b_pos[k]
        a[k] = lr * (y_pos[:1 << i][m].sum() / (m.sum() + l2))
    g = (a - y_pos).astype(np.float32).astype(np.float64)
    want = sum(g[b_pos == b].sum() ** 2 / ((b_pos == b).sum() + l2) for b in (0, 1))
    assert o["score"][1, 0] == pytest.approx(want, rel=1e-12)
    # the same score with every position on model floor(log2 k) + 1 (a plausible slip)
    # differs, so the check above can tell the two apart
    a2 = np.zeros(n)
    for k in range(1, n):
        i = min(int(math.floor(math.log2(k))) + 1, int(math.floor(math.log2(n - 1))))
        m = b_pos[:1 << i] == b_pos[k]
        a2[k] = lr * (y_pos[:1 << i][m].sum() / (m.sum() + l2))
    g2 = (a2 - y_pos).astype(np.float32).astype(np.float64)
    other = sum(g2[b_pos == b].sum() ** 2 / ((b_pos == b).sum() + l2) for b in (0, 1))
    assert abs(other - want) > 1e-6 * want


@pytest.mark.parametrize("i_cut", [0, 3, 6, 8])
def test_model_i_never_sees_labels_from_position_2_to_the_i_on(i_cut):
    n, s, T = 1000, 2, 4
    bins, nb, perms, depth = _forced_case(11, n, s, 2)
    y = (np.random.default_rng(2).random(n) < 0.5).astype(np.float32)
    base = oracle.fit_ordered(bins, 1, nb, y, "logloss", depth, T, 0.2, 1.0, perms)
    off = oracle.ordered_sup_offsets(n)
    for q in range(s):
        y2 = y.copy()
        late = perms[q][1 << i_cut:]
        y2[late] = 1.0 - y2[late]                   # flip every label at positions >= 2^i_cut of sigma_q
        o = oracle.fit_ordered(bins, 1, nb, y2, "logloss", depth, T, 0.2, 1.0, perms)
        for i in range(i_cut + 1):
            a, b = off[i], off[i + 1]
            assert np.array_equal(o["sup"][q, a:b], base["sup"][q, a:b]), (q, i)
        # ... while the next model, trained on those positions, does change
        a, b = off[i_cut + 1], off[i_cut + 2]
        assert not np.array_equal(o["sup"][q, a:b], base["sup"][q, a:b])


def test_degenerate_one_and_two_rows():
    for n in (1, 2):
        bins, nb, perms, depth = _forced_case(3, n, 2, 1)
        y = np.array([1.0, 0.0][:n], np.float32)
        o = oracle.fit_ordered(bins, 1, nb, y, "logloss", depth, 3, 0.5, 1.0, perms)
        assert o["sup"].shape == (2, n)
        assert np.all(np.isfinite(o["sup"])) and np.all(np.isfinite(o["pred"]))
        # model 0 is trained on position 0 alone: its value there moves toward that label
        for q in range(2):
            first = y[perms[q][0]]
            assert (o["sup"][q, 0] > 0) == (first == 1.0)


def test_preprocess_ordered_gives_each_permutation_its_own_ts():
    w = synth.rmse_10k(n=3000)
    F_pad = 32
    res = oracle.preprocess_ordered(w, F_pad, 3)
    base = oracle.preprocess(w, F_pad)
    assert np.array_equal(res["perms"][0], base["perm"]) and np.array_equal(res["bins_all"][0], base["bins"])
    Ff = w.n_float
    for q in range(1, 3):
        assert np.array_equal(res["perms"][q], oracle.make_permutation(w.seed + q, w.n))
        assert np.array_equal(res["bins_all"][q][:, :Ff], base["bins"][:, :Ff])
        for c in range(w.n_cat):
            ts = oracle.ordered_ts(w.cat[c], w.y, res["perms"][q], base["prior"], w.a)[0]
            col = oracle.quantize(ts[None, :], base["borders"][Ff + c:Ff + c + 1], base["n_borders"][Ff + c:Ff + c + 1],
                                  1)[:, 0]
            assert np.array_equal(res["bins_all"][q][:, Ff + c], col)
        assert not np.array_equal(res["bins_all"][q][:, Ff:w.n_features], base["bins"][:, Ff:w.n_features])
