"""Pins of the oracle's inference steps: the full-data target statistic of new rows and
the model value of a row (Section 4 "Fast scorer"), against hand-worked examples, the
training path's own predictions and the ordered statistic of an appended row."""
import numpy as np
import pytest

import oracle
from conftest import golden_directives, golden_rows
from paper_1810_11363_gb300 import synth


def test_predict_worked_example():
    trees = golden_directives("predict_worked_example.txt", "T")
    T, D = len(trees), 2
    sf = np.array([[int(t[1]), int(t[3])] for t in trees], np.int32)
    sk = np.array([[int(t[2]), int(t[4])] for t in trees], np.int32)
    lv = np.array([[float(v) for v in t[5:9]] for t in trees], np.float64)
    rows = golden_rows("predict_worked_example.txt")
    bins = np.zeros((len(rows), 32), np.uint8)
    for i, r in enumerate(rows):
        bins[i, :3] = [int(v) for v in r[:3]]
    expect = np.array([float(r[3]) for r in rows])
    assert sf.shape == (T, D)
    assert np.array_equal(oracle.predict(bins, sf, sk, lv, 0.5), expect)


def test_predict_reproduces_the_training_predictions():
    """The model value recomputed from the stored trees (leaf from all splits at once)
    equals the prediction the boosting loop built tree by tree (leaf updated level by
    level), bit for bit: both add lr * v in tree order in FP64."""
    for loss, w, trees in (("rmse", synth.rmse_10k(n=3000), 6), ("logloss", synth.logloss_1m(n=4000, trees=5), 5)):
        prep = oracle.preprocess(w, 32 * ((w.n_features + 31) // 32))
        res = oracle.fit(prep["bins"], w.n_features, prep["n_borders"], w.y, loss, w.depth, trees, w.lr, w.l2)
        pred = oracle.predict(prep["bins"], res["split_f"], res["split_k"], res["leaf_values"], w.lr)
        assert np.array_equal(pred, res["pred"]), loss


def test_ts_full_worked_example():
    train = np.array([int(v) for v in golden_directives("ts_full_worked_example.txt", "TRAIN")[0]], np.uint32)
    label = np.array([float(v) for v in golden_directives("ts_full_worked_example.txt", "LABEL")[0]], np.float32)
    rows = golden_rows("ts_full_worked_example.txt")
    new = np.array([int(r[0]) for r in rows], np.uint32)
    expect = np.array([np.float32(float(r[1]) / float(r[2])) for r in rows], np.float32)
    got = oracle.ts_full(train, label, 0.6, 1.0, new)
    assert np.array_equal(got, expect)


@pytest.mark.parametrize("a", [1.0, 2.0, 4.0])
def test_ts_full_unseen_category_is_the_prior(a):
    rng = np.random.default_rng(3)
    cat = rng.integers(0, 20, 500).astype(np.uint32)
    y = (rng.random(500) < 0.3).astype(np.float32)
    P = oracle.prior(y, "binary")
    got = oracle.ts_full(cat, y, P, a, np.array([1000, 2000], np.uint32))
    assert np.all(got == np.float32(P))


@pytest.mark.parametrize("label", ["binary", "real"])
def test_ts_full_equals_ordered_ts_of_an_appended_row(label):
    """A new row's full-data statistic is what Eq. 1 gives a row placed after every
    training row in the permutation; computed here with the ordered-TS walk."""
    rng = np.random.default_rng(11)
    n = 800
    cat = synth.zipf_ids(rng, 40, 1.1, n).astype(np.uint32)
    y = ((rng.random(n) < 0.4).astype(np.float32) if label == "binary"
         else rng.standard_t(3, n).astype(np.float32))
    P = oracle.prior(y, label)
    perm = oracle.make_permutation(5, n)
    new = np.concatenate([cat[rng.integers(0, n, 30)], np.array([0xdeadbeef], np.uint32)])
    got = oracle.ts_full(cat, y, P, 1.0, new)
    for i, c in enumerate(new):
        cat2 = np.concatenate([cat, [c]]).astype(np.uint32)
        y2 = np.concatenate([y, [0.0]]).astype(np.float32)
        perm2 = np.concatenate([perm, [n]]).astype(np.uint32)
        ts2, _, _ = oracle.ordered_ts(cat2, y2, perm2, P, 1.0)
        if label == "binary":
            assert got[i] == ts2[n], i
        else:   # label sums in permutation order against row order
            assert abs(float(got[i]) - float(ts2[n])) <= 1e-12 * (np.abs(y).sum() + abs(P)) + np.spacing(abs(ts2[n]))
