"""Pins of the oracle's permutation, prior and ordered target statistic (Eq. 1)
against values and properties fixed by the paper and by mathematics."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import golden_rows


def test_splitmix64_published_vectors():
    # Published first outputs of SplitMix64 seeded with 0.
    for idx, hexval in golden_rows("splitmix64_seed0.txt"):
        assert oracle.splitmix64(0, int(idx)) == int(hexval, 16)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 3), (1000, 0), (4097, 12345)])
def test_permutation_is_bijection_sorted_by_key(n, seed):
    perm = oracle.make_permutation(seed, n)
    assert np.array_equal(np.sort(perm), np.arange(n, dtype=np.uint32))
    keys = np.array([oracle.splitmix64(seed, int(i)) for i in perm], dtype=np.uint64)
    assert np.all(keys[1:] >= keys[:-1])


def test_permutation_depends_on_seed():
    assert not np.array_equal(oracle.make_permutation(0, 100), oracle.make_permutation(1, 100))


def test_prior_binary_is_positive_rate():
    y = np.array([1, 0, 1, 1, 0, 0, 0, 1, 1, 1], np.float32)
    assert oracle.prior(y, "binary") == 6 / 10


def test_prior_real_is_mean():
    y = np.array([1.5, -2.0, 4.25, 0.25], np.float32)
    assert oracle.prior(y, "real") == pytest.approx(1.0, abs=0)


def test_ts_hand_worked_example():
    rows = golden_rows("ts_worked_example.txt")
    ids = {"A": 7, "B": 11}
    cat = np.array([ids[r[0]] for r in rows], np.uint32)
    y = np.array([float(r[1]) for r in rows], np.float32)
    perm = np.arange(len(rows), dtype=np.uint32)          # rows already in permutation order
    ts, cnt, s = oracle.ordered_ts(cat, y, perm, 0.6, 1.0)
    for i, r in enumerate(rows):
        exact = Fraction(int(r[2]), int(r[3]))
        assert abs(float(ts[i]) - float(exact)) <= 1e-7 * float(exact)
    assert cnt.tolist() == [0, 0, 1, 2, 1]
    assert s.tolist() == [0.0, 0.0, 1.0, 1.0, 0.0]


def test_ts_hand_worked_example_under_a_permutation():
    # The same example with rows stored out of order: sigma lists them.
    rows = golden_rows("ts_worked_example.txt")
    ids = {"A": 7, "B": 11}
    order = [3, 0, 4, 1, 2]                      # storage slot of the p-th row in sigma
    n = len(rows)
    cat = np.zeros(n, np.uint32)
    y = np.zeros(n, np.float32)
    for p, slot in enumerate(order):
        cat[slot] = ids[rows[p][0]]
        y[slot] = float(rows[p][1])
    ts, _, _ = oracle.ordered_ts(cat, y, np.array(order, np.uint32), 0.6, 1.0)
    for p, slot in enumerate(order):
        exact = Fraction(int(rows[p][2]), int(rows[p][3]))
        assert abs(float(ts[slot]) - float(exact)) <= 1e-7 * float(exact)


@pytest.mark.parametrize("a", [1.0, 2.0, 4.0])
def test_ts_first_occurrence_is_prior_exactly(a):
    rng = np.random.default_rng(5)
    n = 3000
    cat = rng.integers(0, 50, n).astype(np.uint32)
    y = (rng.random(n) < 0.3).astype(np.float32)
    perm = oracle.make_permutation(9, n)
    P = oracle.prior(y, "binary")
    ts, cnt, _ = oracle.ordered_ts(cat, y, perm, P, a)
    first = cnt == 0
    assert first.sum() == len(np.unique(cat))
    assert np.all(ts[first] == np.float32(P))


@pytest.mark.parametrize("kind", ["binary", "real"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ts_matches_quadratic_brute_force(kind, seed):
    rng = np.random.default_rng(seed)
    n = 64
    cat = rng.integers(0, 6, n).astype(np.uint32) * 1000003
    y = ((rng.random(n) < 0.5).astype(np.float32) if kind == "binary"
         else rng.normal(0, 2, n).astype(np.float32))
    perm = oracle.make_permutation(seed, n)
    P = oracle.prior(y, kind)
    ts, _, _ = oracle.ordered_ts(cat, y, perm, P, 1.0)
    ref = oracle.ordered_ts_quadratic(cat, y, perm, P, 1.0)
    assert np.array_equal(ts.view(np.uint32), ref.view(np.uint32))


def test_ts_single_category_closed_form():
    # One category: position p (0-based) sees every earlier row, so
    # TS_p = (#positives among the first p rows + a*P) / (p + a).
    rng = np.random.default_rng(3)
    n, a, P = 500, 1.0, 0.25
    y = (rng.random(n) < 0.4).astype(np.float32)
    perm = oracle.make_permutation(1, n)
    ts, _, _ = oracle.ordered_ts(np.full(n, 42, np.uint32), y, perm, P, a)
    ys = y[perm].astype(np.int64)
    pos_before = np.concatenate([[0], np.cumsum(ys)[:-1]])
    want = np.array([float(Fraction(int(k)) + Fraction(1, 4)) / (p + 1) for p, k in enumerate(pos_before)])
    got = ts[perm].astype(np.float64)
    assert np.all(np.abs(got - want) <= 1e-7 * np.abs(want) + 1e-12)


def test_ts_all_distinct_categories_give_prior():
    n = 257
    y = np.linspace(-3, 3, n).astype(np.float32)
    perm = oracle.make_permutation(4, n)
    P = oracle.prior(y, "real")
    ts, cnt, _ = oracle.ordered_ts(np.arange(n, dtype=np.uint32) * 7919, y, perm, P, 1.0)
    assert np.all(cnt == 0)
    assert np.all(ts == np.float32(P))


def test_ts_binary_stays_in_unit_interval_and_counts_are_exact():
    rng = np.random.default_rng(11)
    n = 5000
    cat = rng.integers(0, 30, n).astype(np.uint32)
    y = (rng.random(n) < 0.2).astype(np.float32)
    perm = oracle.make_permutation(2, n)
    ts, cnt, s = oracle.ordered_ts(cat, y, perm, oracle.prior(y, "binary"), 1.0)
    assert ts.min() >= 0 and ts.max() <= 1
    # count before = rank of the row among its category in sigma
    pos = np.empty(n, np.int64)
    pos[perm] = np.arange(n)
    for c in np.unique(cat)[:5]:
        rows = np.nonzero(cat == c)[0]
        rows = rows[np.argsort(pos[rows])]
        assert cnt[rows].tolist() == list(range(len(rows)))
        assert s[rows].tolist() == np.concatenate([[0], np.cumsum(y[rows])[:-1]]).tolist()
