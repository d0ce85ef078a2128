"""GPU parity of the inference path against the oracle: full-data target statistics of
new rows (cbg_ts_table + cbg_ts_apply) and the model value (cbg_predict), with the
training rows' predictions reproduced bit for bit from the stored trees."""
import numpy as np
import pytest

import oracle
from gpu_util import to_dev, to_host
from paper_1810_11363_gb300 import cbg, synth, train

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = cbg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("label", ["binary", "real"])
@pytest.mark.parametrize("n,K", [(1, 1), (5000, 3), (20000, 5000), (70000, 60000)])
def test_ts_table_and_apply_match_oracle(ctx, label, n, K):
    rng = np.random.default_rng(n + K)
    cat = synth.zipf_ids(rng, K, 1.1, n).astype(np.uint32)
    y = ((rng.random(n) < 0.35).astype(np.float32) if label == "binary"
         else rng.standard_t(3, n).astype(np.float32))
    P = oracle.prior(y, label)
    # new rows: seen ids, and ids absent from the training rows
    new = np.concatenate([cat[rng.integers(0, n, 3000)], rng.integers(0, 2**32, 500, dtype=np.uint64).astype(np.uint32),
                          np.array([0, 0xffffffff], np.uint32)])
    tables = train.ts_tables(ctx, to_dev(cat[None, :]), to_dev(y), label)
    t = tables[0]
    got = to_host(train.ts_apply(ctx, tables, to_dev(new[None, :]), P, 1.0))[0]
    cbg.cbg_sync(ctx)
    uniq = np.unique(cat)
    U = int(to_host(t.n_unique)[0])
    assert U == uniq.size
    assert np.array_equal(to_host(t.ids)[:U].view(np.uint32), uniq)
    counts = np.bincount(np.searchsorted(uniq, cat), minlength=U)
    assert np.array_equal(to_host(t.cnts)[:U].view(np.uint32), counts)
    ref = oracle.ts_full(cat, y, P, 1.0, new)
    if label == "binary":
        assert np.array_equal(got, ref)
    else:   # FP64 segmented sums against row-order sums
        sabs = np.zeros(U)
        np.add.at(sabs, np.searchsorted(uniq, cat), np.abs(y.astype(np.float64)))
        idx = np.searchsorted(uniq, new)
        seen = (idx < U) & (uniq[np.minimum(idx, U - 1)] == new)
        bound = np.where(seen, 1e-12 * (sabs[np.minimum(idx, U - 1)] + abs(P)), 0.0) + np.spacing(np.abs(ref))
        assert np.all(np.abs(got.astype(np.float64) - ref.astype(np.float64)) <= bound)


def test_ts_apply_of_no_rows_is_a_no_op(ctx):
    import torch
    tables = train.ts_tables(ctx, to_dev(np.array([[3, 4, 3]], np.uint32)), to_dev(np.array([1, 0, 1], np.float32)),
                             "binary")
    out = train.ts_apply(ctx, tables, torch.zeros((1, 0), dtype=torch.int32, device="cuda"), 0.5)
    cbg.cbg_sync(ctx)
    assert out.shape == (1, 0)


def _model_case(seed, n, F, depth, trees, max_bins):
    """A model with random splits (some levels without a split) and random leaf values,
    and row-major bins of rows to score."""
    rng = np.random.default_rng(seed)
    bins = rng.integers(0, max_bins, size=(n, F)).astype(np.uint8)
    sf = rng.integers(0, F, size=(trees, depth)).astype(np.int32)
    sk = rng.integers(0, max_bins - 1, size=(trees, depth)).astype(np.int32)
    sf[rng.random((trees, depth)) < 0.05] = -1
    sk[sf < 0] = -1
    lv = rng.normal(0.0, 1.0, size=(trees, 1 << depth))
    return bins, sf, sk, lv


def _split_tensor(sf, sk):
    import torch
    T, D = sf.shape
    rec = np.zeros((T, D), dtype=train.SPLIT_DTYPE)
    rec["feature"], rec["border"] = sf, sk
    return torch.from_numpy(rec.view(np.float64).reshape(T, D, 2).copy()).cuda()


@pytest.mark.parametrize("n,F,depth,trees,max_bins", [(1, 3, 1, 1, 2), (33, 5, 2, 7, 3), (3001, 40, 6, 300, 255),
                                                      (10000, 70, 10, 40, 129), (257, 2000, 6, 1100, 129)])
def test_predict_matches_oracle(ctx, n, F, depth, trees, max_bins):
    import torch
    bins, sf, sk, lv = _model_case(n + depth, n, F, depth, trees, max_bins)
    lr = 0.1
    bins_t = to_dev(np.ascontiguousarray(bins.T))
    model = train.Model(_split_tensor(sf, sk), torch.from_numpy(lv).cuda(), None, depth, lr)
    got = to_host(train.predict(ctx, model, bins_t, F)).astype(np.float64)
    cbg.cbg_sync(ctx)
    F_pad = 32 * ((F + 31) // 32)
    rm = np.zeros((n, F_pad), np.uint8)
    rm[:, :F] = bins
    ref = oracle.predict(rm, sf, sk, lv, lr)
    # FP32: every increment float(lr v) rounds once, and the sum of T terms in tree order
    # errs by at most gamma_T times the sum of their magnitudes (gamma_T = T u / (1 - T u))
    u = 2.0**-24
    mag = trees * np.abs(lr * lv).max()
    assert np.all(np.abs(got - ref) <= (trees + 1) * u / (1 - trees * u) * mag + 1e-12)


def test_predict_reproduces_training_predictions_bit_for_bit(ctx):
    """cbg_predict over the training rows from the stored trees gives back the prediction
    the boosting loop accumulated (same FP32 increments in the same order)."""
    w = synth.logloss_1m(n=30000, trees=25)
    prep = train.preprocess(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), "binary", w.max_borders, a=w.a,
                            seed=w.seed)
    model = train.fit(ctx, prep, to_dev(w.y), w.loss, w.depth, w.trees, w.lr, w.l2, use_graph=True)
    again = train.predict(ctx, model, prep.bins_t, prep.F)
    cbg.cbg_sync(ctx)
    assert np.array_equal(to_host(again).view(np.uint32), to_host(model.pred).view(np.uint32))
    # and a second call continues from the given predictions (pred is in/out)
    twice = train.predict(ctx, model, prep.bins_t, prep.F, pred=again.clone())
    cbg.cbg_sync(ctx)
    assert np.allclose(to_host(twice), 2 * to_host(model.pred), rtol=1e-5, atol=1e-5)


def test_new_rows_end_to_end_match_oracle(ctx):
    """Train on one sample and score fresh rows of the same distribution through the whole
    inference path (full-data TS, quantisation with the training borders, prediction).
    The oracle runs the same steps on its own: its own preprocessing of the training
    sample, its own model, its own statistics and bins of the new rows."""
    import dataclasses
    w = synth.logloss_1m(n=16000, trees=15)
    n_tr = 12000
    w_tr = dataclasses.replace(w, x=np.ascontiguousarray(w.x[:, :n_tr]), cat=np.ascontiguousarray(w.cat[:, :n_tr]),
                               y=np.ascontiguousarray(w.y[:n_tr]))
    x_te, c_te = np.ascontiguousarray(w.x[:, n_tr:]), np.ascontiguousarray(w.cat[:, n_tr:])
    # GPU
    prep = train.preprocess(ctx, to_dev(w_tr.x), to_dev(w_tr.cat), to_dev(w_tr.y), "binary", w.max_borders, a=w.a,
                            seed=w.seed)
    model = train.fit(ctx, prep, to_dev(w_tr.y), w.loss, w.depth, w.trees, w.lr, w.l2)
    tables = train.ts_tables(ctx, to_dev(w_tr.cat), to_dev(w_tr.y), "binary")
    bins_t = train.preprocess_new(ctx, prep, tables, to_dev(x_te), to_dev(c_te), a=w.a)
    pred = to_host(train.predict(ctx, model, bins_t, prep.F)).astype(np.float64)
    cbg.cbg_sync(ctx)
    # oracle
    ref = oracle.preprocess(w_tr, prep.F_pad)
    ts_new = np.stack([oracle.ts_full(w_tr.cat[c], w_tr.y, ref["prior"], w.a, c_te[c]) for c in range(w.n_cat)])
    bins_ref = oracle.quantize(np.concatenate([x_te, ts_new]), ref["borders"], ref["n_borders"], prep.F_pad)
    assert np.array_equal(to_host(bins_t), np.ascontiguousarray(bins_ref[:, :prep.F].T))   # binary labels: exact
    res = oracle.fit(ref["bins"], w.n_features, ref["n_borders"], w_tr.y, w.loss, w.depth, w.trees, w.lr, w.l2)
    sp = model.host_splits()
    for t in range(w.trees):
        for d in range(w.depth):
            if res["score"][t, d] - res["second"][t, d] <= 1e-6 * abs(res["score"][t, d]):
                return   # a near-tie: the models may differ from here on
            assert (sp[t, d]["feature"], sp[t, d]["border"]) == (res["split_f"][t, d], res["split_k"][t, d]), (t, d)
    ref_pred = oracle.predict(bins_ref, res["split_f"], res["split_k"], res["leaf_values"], w.lr)
    assert np.all(np.abs(pred - ref_pred) <= 1e-4)
