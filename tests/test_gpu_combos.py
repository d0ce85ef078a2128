"""GPU parity of greedy feature combinations (Section 2 "Feature combinations") against
the oracle, which prepares its own inputs and runs its own boosting with combinations.

Splits (ordinary or combination: the items and the border), the combination's borders
and the leaf values are compared tree by tree; a split may differ only where the
oracle's best and runner-up scores are within 1e-5 relative, and the runs are compared up
to there. Binary labels make every TS, border and bin exact; predictions within 1e-4."""
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


def _run_both(ctx, w, depth, trees, max_borders, mc, lr=0.2, l2=1.0):
    prep = train.preprocess(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), w.label_kind, w.max_borders, a=w.a,
                            seed=w.seed)
    got = train.fit_combos(ctx, prep, to_dev(w.cat), to_dev(w.y), w.label_kind, w.loss, depth, trees, lr, l2,
                           max_borders, mc, a=w.a)
    cbg.cbg_sync(ctx)
    ref_prep = oracle.preprocess(w, prep.F_pad)
    assert np.array_equal(train.rowmajor_from_grouped(to_host(prep.bins), w.n, prep.F_pad), ref_prep["bins"])
    res = oracle.fit_combos(ref_prep["bins"], w.n_features, w.n_float, ref_prep["n_borders"], w.cat, w.y, w.loss,
                            depth, trees, lr, l2, ref_prep["perm"], ref_prep["prior"], w.a, max_borders, mc)
    return got, res


def _compare(got, res, F, depth, trees, near=1e-5):
    sp = got.model.host_splits()
    n_combo = 0
    for t in range(trees):
        for d in range(depth):
            same = (sp[t, d]["feature"], sp[t, d]["border"]) == (res["split_f"][t, d], res["split_k"][t, d])
            if same and res["split_f"][t, d] >= F:
                same = (np.array_equal(got.combo_items[t, d], res["combo_items"][t, d])
                        and got.combo_nb[t, d] == res["combo_nb"][t, d])
            if not same:
                assert res["score"][t, d] - res["second"][t, d] <= near * abs(res["score"][t, d]), (t, d)
                return t, n_combo
            if res["split_f"][t, d] >= F:
                n_combo += 1
                nb = res["combo_nb"][t, d]
                assert np.array_equal(got.combo_borders[t, d, :nb].view(np.uint32),
                                      res["combo_borders"][t, d, :nb].view(np.uint32))
        assert np.allclose(to_host(got.model.leaf_values[t]), res["leaf_values"][t], rtol=1e-4, atol=1e-6), t
    assert np.all(np.abs(to_host(got.model.pred) - res["pred"]) <= 1e-4)
    return trees, n_combo


def _interaction_workload(n, seed=0):
    return synth.interaction_xor(n=n, seed=seed)


@pytest.mark.parametrize("n", [3000, 20001])
def test_combinations_match_oracle_on_an_interaction(ctx, n):
    w = _interaction_workload(n)
    got, res = _run_both(ctx, w, depth=4, trees=3, max_borders=15, mc=3)
    assert (res["split_f"] >= w.n_features).any()       # the oracle does take combinations here
    compared, n_combo = _compare(got, res, w.n_features, 4, 3)
    assert compared >= 1 and n_combo >= 1


@pytest.mark.parametrize("depth,mc", [(3, 2), (5, 4)])
def test_combinations_match_oracle_on_logloss_shaped_data(ctx, depth, mc):
    w = synth.logloss_1m(n=12000, trees=3)
    got, res = _run_both(ctx, w, depth=depth, trees=3, max_borders=31, mc=mc)
    compared, _ = _compare(got, res, w.n_features, depth, 3)
    assert compared >= 1


def test_max_complexity_one_is_classic_boosting(ctx):
    w = synth.logloss_1m(n=8000, trees=3)
    prep = train.preprocess(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), "binary", w.max_borders, a=w.a,
                            seed=w.seed)
    got = train.fit_combos(ctx, prep, to_dev(w.cat), to_dev(w.y), "binary", "logloss", 4, 3, 0.1, 3.0, 15, 1)
    plain = train.fit(ctx, prep, to_dev(w.y), "logloss", 4, 3, 0.1, 3.0)
    cbg.cbg_sync(ctx)
    a, b = got.model.host_splits(), plain.host_splits()
    assert np.array_equal(a["feature"], b["feature"]) and np.array_equal(a["border"], b["border"])
    assert np.allclose(to_host(got.model.pred), to_host(plain.pred), atol=1e-6)
    assert np.all(got.combo_items == -1)


def test_new_rows_with_combinations_match_oracle(ctx):
    """Train with combinations on part of the interaction workload and score the rest: the
    GPU path (full-data TS of every used combination, quantised with its borders, as extra
    columns for cbg_predict) against the oracle doing the same steps with its own model."""
    import dataclasses
    w = _interaction_workload(24000, seed=7)     # the oracle's best and runner-up differ by >= 2.5e-4 everywhere
    n_tr = 20000
    w_tr = dataclasses.replace(w, x=np.ascontiguousarray(w.x[:, :n_tr]), cat=np.ascontiguousarray(w.cat[:, :n_tr]),
                               y=np.ascontiguousarray(w.y[:n_tr]))
    x_te, c_te = np.ascontiguousarray(w.x[:, n_tr:]), np.ascontiguousarray(w.cat[:, n_tr:])
    depth, trees, lr, l2, mb, mc = 4, 3, 0.2, 1.0, 15, 3
    got, res = _run_both(ctx, w_tr, depth, trees, mb, mc, lr=lr, l2=l2)
    compared, n_combo = _compare(got, res, w.n_features, depth, trees)
    assert compared == trees and n_combo >= 1
    # GPU: the new rows' bins, then the combinations as extra columns
    prep = train.preprocess(ctx, to_dev(w_tr.x), to_dev(w_tr.cat), to_dev(w_tr.y), "binary", w.max_borders, a=w.a,
                            seed=w.seed)
    tables = train.ts_tables(ctx, to_dev(w_tr.cat), to_dev(w_tr.y), "binary")
    bins_t_new = train.preprocess_new(ctx, prep, tables, to_dev(x_te), to_dev(c_te), a=w.a)
    pred = to_host(train.predict_combos(ctx, got, prep, to_dev(w_tr.cat), to_dev(w_tr.y), "binary", bins_t_new,
                                        to_dev(c_te), a=w.a)).astype(np.float64)
    cbg.cbg_sync(ctx)
    # oracle: the same steps on its own preprocessing and model
    ref = oracle.preprocess(w_tr, prep.F_pad)
    ts_new = np.stack([oracle.ts_full(w_tr.cat[c], w_tr.y, ref["prior"], w.a, c_te[c]) for c in range(w.n_cat)])
    F = w.n_features
    bins_new = oracle.quantize(np.concatenate([x_te, ts_new]), ref["borders"], ref["n_borders"], 64)
    sf = res["split_f"].copy()
    cols = {}
    for t in range(trees):
        for d in range(depth):
            if sf[t, d] >= F:
                key = tuple(tuple(int(v) for v in it) for it in res["combo_items"][t, d] if it[0] >= 0)
                if key not in cols:
                    cols[key] = (len(cols), t, d)
                sf[t, d] = F + cols[key][0]
    for key, (k, t, d) in cols.items():
        ids_tr = oracle.combo_ids(key, w_tr.cat, ref["bins"])
        ids_new = oracle.combo_ids(key, c_te, bins_new)
        ts = oracle.ts_full(ids_tr, w_tr.y, ref["prior"], w.a, ids_new)
        nb = res["combo_nb"][t, d]
        oracle.quantize(ts[None, :], res["combo_borders"][t, d][None, :], np.array([nb], np.int32), 64,
                        f_offset=F + k, bins=bins_new)
    ref_pred = oracle.predict(bins_new, sf, res["split_k"], res["leaf_values"], lr)
    assert np.all(np.abs(pred - ref_pred) <= 1e-4)


def test_bad_arguments_are_rejected(ctx):
    import torch
    ids = torch.empty(10, dtype=torch.int32, device="cuda")
    cat = torch.zeros((2, 10), dtype=torch.int32, device="cuda")
    bt = torch.zeros((3, 10), dtype=torch.uint8, device="cuda")
    for items in ([(0, 1, 0), (0, 0, 0)],          # not in canonical order
                  [(0, 2, 0)],                     # no such categorical column
                  [(1, 3, 0)],                     # no such feature
                  []):
        with pytest.raises(cbg.CbgError) as e:
            cbg.cbg_combo_ids(ctx, items, cat, 2, bt, 3, 10, ids)
        assert e.value.status == cbg.CBG_EINVAL
    cbg.cbg_combo_ids(ctx, [(0, 0, 0), (1, 2, 0)], cat, 2, bt, 3, 10, ids)
    cbg.cbg_sync(ctx)
    assert torch.all(ids == ids[0])                  # constant columns: one value
    with pytest.raises(cbg.CbgError):
        cbg.cbg_combo_work_bytes(10, 2, 6, 255, 4)    # at most 254 borders


def test_combinations_with_real_labels(ctx):
    """RMSE with real labels: the TS (single columns and candidates) are FP64 prefix sums
    in another order on the GPU, so a border may land one ulp away and a later split may
    differ; the first split must agree and the final training losses agree closely."""
    w = synth.rmse_10k(n=8000)
    prep = train.preprocess(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), "real", w.max_borders, a=w.a, seed=w.seed)
    got = train.fit_combos(ctx, prep, to_dev(w.cat), to_dev(w.y), "real", "rmse", 4, 6, 0.1, 3.0, 15, 3, a=w.a)
    cbg.cbg_sync(ctx)
    rp = oracle.preprocess(w, prep.F_pad)
    res = oracle.fit_combos(rp["bins"], w.n_features, w.n_float, rp["n_borders"], w.cat, w.y, "rmse", 4, 6, 0.1, 3.0,
                            rp["perm"], rp["prior"], w.a, 15, 3)
    gpu_loss = oracle.loss("rmse", w.y, to_host(got.model.pred).astype(np.float64))
    assert abs(gpu_loss - res["losses"][-1]) <= 1e-3 * res["losses"][-1]
    sp = got.model.host_splits()
    assert (sp[0, 0]["feature"], sp[0, 0]["border"]) == (res["split_f"][0, 0], res["split_k"][0, 0])


def test_bf16_gradients_with_combinations_train_close_to_f32(ctx):
    w = _interaction_workload(20000, seed=7)
    prep = train.preprocess(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), "binary", w.max_borders, a=w.a,
                            seed=w.seed)
    losses = {}
    for dt in ("f32", "bf16"):
        m = train.fit_combos(ctx, prep, to_dev(w.cat), to_dev(w.y), "binary", "logloss", 4, 4, 0.2, 1.0, 15, 3,
                             a=w.a, gh_dtype=dt)
        cbg.cbg_sync(ctx)
        losses[dt] = oracle.loss("logloss", w.y, to_host(m.model.pred).astype(np.float64))
        assert (m.model.host_splits()["feature"] >= w.n_features).any(), dt
    assert abs(losses["bf16"] - losses["f32"]) <= 5e-3 * losses["f32"]


def test_depth_one_takes_no_combination(ctx):
    """A depth-1 tree has only the first level, which takes no combination: the run is the
    classic one."""
    w = synth.interaction_xor(5000, seed=2)
    prep = train.preprocess(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), "binary", w.max_borders, a=w.a,
                            seed=w.seed)
    got = train.fit_combos(ctx, prep, to_dev(w.cat), to_dev(w.y), "binary", "logloss", 1, 4, 0.2, 1.0, 15, 4, a=w.a)
    plain = train.fit(ctx, prep, to_dev(w.y), "logloss", 1, 4, 0.2, 1.0)
    cbg.cbg_sync(ctx)
    a, b = got.model.host_splits(), plain.host_splits()
    assert np.array_equal(a["feature"], b["feature"]) and np.array_equal(a["border"], b["border"])
    # the FP32 shared-memory reductions add in a run-dependent order: equal to rounding
    assert np.allclose(to_host(got.model.pred), to_host(plain.pred), rtol=0, atol=1e-6)


@pytest.mark.parametrize("n", [50, 1001])
def test_one_categorical_joins_only_splits(ctx, n):
    """With one categorical column every candidate is that column joined with float splits
    of the tree (kind-1 items); small and ragged n against the oracle."""
    import dataclasses
    w = synth.interaction_xor(n, seed=4)
    w = dataclasses.replace(w, cat=np.ascontiguousarray(w.cat[:1]))
    got, res = _run_both(ctx, w, depth=3, trees=3, max_borders=7, mc=3)
    compared, n_combo = _compare(got, res, w.n_features, 3, 3)
    assert compared >= 1
    items = res["combo_items"][res["split_f"] >= w.n_features]
    for it in items:
        used = it[it[:, 0] >= 0]
        assert used[0, 0] == 0 and np.all(used[1:, 0] == 1)
