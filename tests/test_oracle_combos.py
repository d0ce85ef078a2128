"""Pins of the feature-combination oracle (Section 2 "Feature combinations") against
what the definitions fix, independent of the hash that names a combination's values:

- Eq. 1 depends only on which rows share a value, so a combination whose values split the
  rows exactly like a known column has that column's ordered TS, bit for bit: a column
  joined with a function of itself, with a constant column, and with a two-valued split
  (the product of the column and the bit, built by hand);
- without categorical columns, or with max_complexity 1, boosting is classic boosting;
- the first level of every tree takes no combination;
- an interaction that no single column carries (the label depends on c1 XOR c2 only) is
  found by the combination of the two columns at the second level.
"""
import numpy as np
import pytest

import oracle


def _ts(ids, y, perm, P, a=1.0):
    return oracle.ordered_ts(ids, y, perm, P, a)[0]


def _case(seed, n):
    rng = np.random.default_rng(seed)
    c1 = rng.integers(0, 50, n).astype(np.uint32) * 7919 + 13
    y = (rng.random(n) < 0.3).astype(np.float32)
    perm = oracle.make_permutation(seed, n)
    return rng, c1, y, perm


@pytest.mark.parametrize("n", [1, 7, 2000])
def test_combination_with_a_function_of_itself_has_the_columns_ts(n):
    rng, c1, y, perm = _case(1, n)
    c2 = (c1 // 3 + 5).astype(np.uint32)            # a function of c1: no new split of the rows
    cat = np.stack([c1, c2])
    bins = np.zeros((n, 32), np.uint8)
    P = 0.3
    ids = oracle.combo_ids([(0, 0, 0), (0, 1, 0)], cat, bins)
    assert np.array_equal(_ts(ids, y, perm, P).view(np.uint32), _ts(c1, y, perm, P).view(np.uint32))


def test_combination_with_a_constant_column_has_the_columns_ts():
    n = 3000
    rng, c1, y, perm = _case(2, n)
    cat = np.stack([np.full(n, 42, np.uint32), c1])
    bins = np.zeros((n, 32), np.uint8)
    ids = oracle.combo_ids([(0, 0, 0), (0, 1, 0)], cat, bins)
    assert np.array_equal(_ts(ids, y, perm, 0.3).view(np.uint32), _ts(c1, y, perm, 0.3).view(np.uint32))


@pytest.mark.parametrize("k", [0, 2, 5])
def test_combination_with_a_split_is_the_product_of_column_and_bit(k):
    n = 4000
    rng, c1, y, perm = _case(3, n)
    bins = np.zeros((n, 32), np.uint8)
    bins[:, 4] = rng.integers(0, 8, n)
    cat = c1[None, :]
    ids = oracle.combo_ids([(0, 0, 0), (1, 4, k)], cat, bins)
    bit = (bins[:, 4] > k).astype(np.uint32)
    product = np.unique(c1, return_inverse=True)[1].astype(np.uint32) * 2 + bit
    assert np.array_equal(_ts(ids, y, perm, 0.3).view(np.uint32), _ts(product, y, perm, 0.3).view(np.uint32))
    # ... and differs from the column's own TS (the bit does split the rows)
    assert not np.array_equal(_ts(ids, y, perm, 0.3), _ts(c1, y, perm, 0.3))


def _workload(seed, n, n_float, C, interaction=False):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n_float, n)).astype(np.float32)
    cat = rng.integers(0, 4, size=(C, n)).astype(np.uint32) * 1000003 + 17
    if interaction:
        z = ((cat[0] // 1000003) % 2) ^ ((cat[1] // 1000003) % 2)
        y = (rng.random(n) < np.where(z == 1, 0.9, 0.1)).astype(np.float32)
    else:
        y = (rng.random(n) < 1.0 / (1.0 + np.exp(-x[0] if n_float else 0.0))).astype(np.float32)
    perm = oracle.make_permutation(seed, n)
    P = oracle.prior(y, "binary")
    ts = np.stack([_ts(cat[c], y, perm, P) for c in range(C)]) if C else np.zeros((0, n), np.float32)
    cols = np.concatenate([x, ts]) if C else x
    borders, nb = oracle.select_borders(cols, 15)
    bins = oracle.quantize(cols, borders, nb, 32)
    return bins, nb, cat, y, perm, P


def test_without_combinations_it_is_classic_boosting():
    bins, nb, cat, y, perm, P = _workload(4, 3000, 5, 0)
    c = oracle.fit(bins, 5, nb, y, "logloss", 4, 3, 0.1, 3.0)
    o = oracle.fit_combos(bins, 5, 5, nb, cat, y, "logloss", 4, 3, 0.1, 3.0, perm, P, 1.0, 15)
    for key in ("split_f", "split_k", "leaf_values", "pred"):
        assert np.array_equal(o[key], c[key]), key
    bins, nb, cat, y, perm, P = _workload(5, 3000, 4, 3)
    c = oracle.fit(bins, 7, nb, y, "logloss", 4, 3, 0.1, 3.0)
    o = oracle.fit_combos(bins, 7, 4, nb, cat, y, "logloss", 4, 3, 0.1, 3.0, perm, P, 1.0, 15, max_complexity=1)
    for key in ("split_f", "split_k", "leaf_values", "pred"):
        assert np.array_equal(o[key], c[key]), key
    assert np.all(o["combo_items"] == -1)


def test_interaction_is_found_by_the_combination_at_the_second_level():
    bins, nb, cat, y, perm, P = _workload(6, 6000, 0, 3, interaction=True)
    o = oracle.fit_combos(bins, 3, 0, nb, cat, y, "logloss", 3, 2, 0.3, 1.0, perm, P, 1.0, 15)
    F = 3
    assert np.all(o["split_f"][:, 0] < F)                    # no combination at the first level
    # the first split takes one of the two interacting columns (their TS leak a little of
    # the label through the prior's noise); at level 1 it is joined with its partner
    assert o["split_f"][0, 0] in (0, 1)
    assert o["split_f"][0, 1] == F
    items = [tuple(it) for it in o["combo_items"][0, 1] if it[0] >= 0]
    assert items == [(0, 0, 0), (0, 1, 0)]
    assert o["combo_nb"][0, 1] >= 1
    # the combination makes the training loss fall far below what single columns allow
    c = oracle.fit(bins, 3, nb, y, "logloss", 3, 2, 0.3, 1.0)
    assert o["losses"][-1] < c["losses"][-1] - 0.05


def test_combinations_respect_max_complexity():
    bins, nb, cat, y, perm, P = _workload(7, 3000, 3, 4)
    for mc in (2, 3):
        o = oracle.fit_combos(bins, 7, 3, nb, cat, y, "logloss", 5, 3, 0.1, 3.0, perm, P, 1.0, 15, max_complexity=mc)
        used = (o["combo_items"][..., 0] >= 0).sum(axis=-1)
        assert used.max() <= mc
        assert np.all(o["split_f"][:, 0] < 7)
        is_combo = o["split_f"] >= 7
        assert np.array_equal(is_combo, used > 0)


def _sign_interaction(seed, n=6000):
    """P(y) = sigmoid(2 x0 + 1.5 s(c) sign(x0)), s(c) = +-1 by the parity of the category:
    the categorical column has no effect of its own, only joined with the split on x0."""
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(2, n)).astype(np.float32)
    cat = rng.integers(0, 4, size=(1, n)).astype(np.uint32) * 1000003 + 17
    par = ((cat[0] // 1000003) % 2) * 2.0 - 1.0
    z = np.clip(2 * x[0] + 1.5 * par * np.sign(x[0]), -30, 30)
    y = (rng.random(n) < 1 / (1 + np.exp(-z))).astype(np.float32)
    perm = oracle.make_permutation(seed, n)
    P = oracle.prior(y, "binary")
    cols = np.concatenate([x, _ts(cat[0], y, perm, P)[None]])
    borders, nb = oracle.select_borders(cols, 15)
    return oracle.quantize(cols, borders, nb, 32), nb, cat, y, perm, P


def test_a_split_in_the_tree_joins_combinations_as_a_two_valued_column():
    bins, nb, cat, y, perm, P = _sign_interaction(1)
    o = oracle.fit_combos(bins, 3, 2, nb, cat, y, "logloss", 3, 3, 0.3, 1.0, perm, P, 1.0, 15)
    combos = [(t, d) for t in range(3) for d in range(3) if o["split_f"][t, d] >= 3]
    assert combos
    for t, d in combos:
        items = [tuple(int(v) for v in it) for it in o["combo_items"][t, d] if it[0] >= 0]
        # the only categorical column joined with a float split taken earlier in the tree
        earlier = {(1, int(o["split_f"][t, e]), int(o["split_k"][t, e])) for e in range(d) if o["split_f"][t, e] < 2}
        assert len(items) == 2 and items[0] == (0, 0, 0) and items[1] in earlier


def test_a_combination_that_ties_an_ordinary_split_loses_the_tie():
    """c2 is a function of c1, so the only candidate {c1, c2} has c1's TS, borders and
    scores exactly: it can never beat c1's column strictly, and no combination is taken."""
    n = 5000
    rng = np.random.default_rng(8)
    c1 = rng.integers(0, 12, n).astype(np.uint32)
    c2 = (c1 % 3).astype(np.uint32) + 100
    y = (rng.random(n) < 0.2 + 0.05 * (c1 % 7)).astype(np.float32)
    perm = oracle.make_permutation(8, n)
    P = oracle.prior(y, "binary")
    cat = np.stack([c1, c2])
    cols = np.stack([_ts(c1, y, perm, P), _ts(c2, y, perm, P)])
    borders, nb = oracle.select_borders(cols, 15)
    bins = oracle.quantize(cols, borders, nb, 32)
    o = oracle.fit_combos(bins, 2, 0, nb, cat, y, "logloss", 4, 3, 0.3, 1.0, perm, P, 1.0, 15)
    assert np.all(o["split_f"] < 2)
    c = oracle.fit(bins, 2, nb, y, "logloss", 4, 3, 0.3, 1.0)
    assert np.array_equal(o["split_f"], c["split_f"]) and np.array_equal(o["pred"], c["pred"])


def test_max_complexity_caps_the_interaction_case():
    bins, nb, cat, y, perm, P = _workload(6, 6000, 0, 3, interaction=True)
    o4 = oracle.fit_combos(bins, 3, 0, nb, cat, y, "logloss", 3, 2, 0.3, 1.0, perm, P, 1.0, 15)
    assert (o4["combo_items"][..., 0] >= 0).sum(axis=-1).max() == 3    # {c0, c1, c2} at level 2
    o2 = oracle.fit_combos(bins, 3, 0, nb, cat, y, "logloss", 3, 2, 0.3, 1.0, perm, P, 1.0, 15, max_complexity=2)
    assert (o2["combo_items"][..., 0] >= 0).sum(axis=-1).max() == 2
