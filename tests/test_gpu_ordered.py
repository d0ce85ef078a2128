"""GPU parity of ordered boosting (Section 3, Algorithm 1 with the log-scale supporting
models) against the oracle, which prepares its own inputs (permutations, per-permutation
TS, borders, bins) and runs its own boosting.

Tolerances: permutations, bins and structures exact (the oracle follows the GPU's split
in lock step where it scores within 1e-5 relative of the oracle's best: the FP32
supporting values may pick either side of such a near-tie); leaf values, predictions
and supporting values within 1e-4 absolute (FP32 values against FP64) over every tree."""
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


def _sup_to_oracle_layout(sup_gpu, n):
    """GPU layout (model i at element 2^(i+1)) -> the oracle's packed layout."""
    off = oracle.ordered_sup_offsets(n)
    out = np.empty((sup_gpu.shape[0], off[-1]), np.float64)
    for i in range(len(off) - 1):
        held = off[i + 1] - off[i]
        out[:, off[i]:off[i + 1]] = sup_gpu[:, (2 << i):(2 << i) + held]
    return out


def test_sup_len_and_work_bytes():
    for n in [1, 2, 3, 4, 5, 1000, 1 << 20, (1 << 20) + 1]:
        I = (n - 1).bit_length() - 1 if n > 1 else 0
        assert cbg.cbg_ordered_sup_len(n) == ((2 << I) + n + 63) // 64 * 64
        assert (2 << I) + n - 2 >= oracle.ordered_sup_size(n)
    assert cbg.cbg_ordered_work_bytes(1000, 3, 6) >= 3 * 1000 * 2 + 1000 * 2 + 64 * 16 * (1 + 3 * 10)


@pytest.mark.parametrize("n,F", [(1, 1), (1000, 40), (33333, 70)])
def test_permute_rows(ctx, n, F):
    import torch
    rng = np.random.default_rng(n)
    F_pad = train.f_pad_for(F)
    rm = np.zeros((n, F_pad), np.uint8)
    rm[:, :F] = rng.integers(0, 256, size=(n, F))
    perm = rng.permutation(n).astype(np.uint32)
    y = rng.normal(size=n).astype(np.float32)
    bins = to_dev(train.grouped_from_rowmajor(rm))
    bins_t = to_dev(np.ascontiguousarray(rm[:, :F].T))
    bp = torch.empty_like(bins)
    btp = torch.empty_like(bins_t)
    yp = torch.empty(n, dtype=torch.float32, device="cuda")
    cbg.cbg_permute_rows(ctx, to_dev(perm), n, F, F_pad, bins, bins_t, to_dev(y), bp, btp, yp)
    cbg.cbg_sync(ctx)
    assert np.array_equal(train.rowmajor_from_grouped(to_host(bp), n, F_pad), rm[perm])
    assert np.array_equal(to_host(btp), np.ascontiguousarray(rm[perm, :F].T))
    assert np.array_equal(to_host(yp), y[perm])


def _prepare_both(ctx, w, s):
    op = train.preprocess_ordered(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), w.label_kind, w.max_borders, s,
                                  a=w.a, seed=w.seed)
    ref = oracle.preprocess_ordered(w, op.base.F_pad, s)
    return op, ref


def _from_bins(ctx, bins_all, perms, n_borders, y, F):
    """OrderedPrepared over given row-major bins [s][n][F_pad] and permutations [s][n]
    (the oracle's own), so that a boosting comparison starts from identical inputs."""
    import torch
    s, n, F_pad = bins_all.shape
    bins_pos = torch.empty((s, F_pad * n), dtype=torch.uint8, device="cuda")
    bins_t_pos = torch.empty((s, F, n), dtype=torch.uint8, device="cuda")
    y_pos = torch.empty((s, n), dtype=torch.float32, device="cuda")
    yd = to_dev(y)
    for q in range(s):
        cbg.cbg_permute_rows(ctx, to_dev(perms[q]), n, F, F_pad, to_dev(train.grouped_from_rowmajor(bins_all[q])),
                             to_dev(np.ascontiguousarray(bins_all[q][:, :F].T)), yd, bins_pos[q], bins_t_pos[q],
                             y_pos[q])
    nb = np.asarray(n_borders, np.int32)
    base = train.Prepared(n, F, F, F_pad, None, 0.0, None, None, to_dev(nb),
                          to_dev(train.grouped_from_rowmajor(bins_all[0])),
                          to_dev(np.ascontiguousarray(bins_all[0][:, :F].T)), int(nb.max()) + 1)
    return train.OrderedPrepared(base, s, None, bins_pos, bins_t_pos, y_pos), yd


def test_preprocess_ordered_matches_oracle(ctx):
    w = synth.logloss_1m(n=20000, trees=1)
    s = 3
    op, ref = _prepare_both(ctx, w, s)
    n, F, F_pad = w.n, op.base.F, op.base.F_pad
    perms = to_host(op.perms, np.uint32)
    assert np.array_equal(perms, ref["perms"])
    bins_pos = to_host(op.bins_pos)
    bins_t_pos = to_host(op.bins_t_pos)
    for q in range(s):
        # binary labels: the TS are exact, so are the bins
        assert np.array_equal(train.rowmajor_from_grouped(bins_pos[q], n, F_pad), ref["bins_all"][q][perms[q]])
        assert np.array_equal(bins_t_pos[q], np.ascontiguousarray(ref["bins_all"][q][perms[q], :F].T))
        assert np.array_equal(to_host(op.y_pos)[q], w.y[perms[q]])


def _compare_runs(model, res, n, depth, trees, atol=1e-4):
    """The oracle run followed the GPU's splits (lock step, near-tie margin 1e-5: the FP32
    supporting values may pick either side of a closer tie; exact ties, e.g. a
    permutation's TS leaving a bin empty so that two borders cut the same rows, go to the
    smallest feature then border on both sides). Every split, leaf value, prediction and
    supporting value is then compared. Returns the number of near-ties followed."""
    sp = model.host_splits()
    fl = res["followed"]
    assert np.all(fl >= 0), np.argwhere(fl < 0)[:8].tolist()
    assert np.array_equal(sp["feature"], res["split_f"]) and np.array_equal(sp["border"], res["split_k"])
    assert np.allclose(to_host(model.leaf_values), res["leaf_values"], rtol=1e-4, atol=atol)
    assert np.all(np.abs(to_host(model.pred) - res["pred"]) <= atol)
    sup = _sup_to_oracle_layout(to_host(model.sup).astype(np.float64), n)
    assert np.all(np.abs(sup - res["sup"]) <= atol)
    return int((fl == 1).sum())


@pytest.mark.parametrize("loss,n,s,depth,trees", [
    ("logloss", 3001, 1, 3, 6),
    ("logloss", 20000, 3, 6, 8),
    ("rmse", 9000, 2, 4, 8),
    ("rmse", 4097, 4, 2, 10),
])
def test_ordered_fit_matches_oracle(ctx, loss, n, s, depth, trees):
    w = synth.logloss_1m(n=n, trees=trees) if loss == "logloss" else synth.rmse_10k(n=n)
    ref = oracle.preprocess_ordered(w, train.f_pad_for(w.n_features), s)
    op, yd = _from_bins(ctx, ref["bins_all"], ref["perms"], ref["n_borders"], w.y, w.n_features)
    model = train.fit_ordered(ctx, op, yd, loss, depth, trees, 0.1, 3.0)
    cbg.cbg_sync(ctx)
    res = oracle.fit_ordered(ref["bins_all"], w.n_features, ref["n_borders"], w.y, loss, depth, trees, 0.1, 3.0,
                             ref["perms"], follow=model.host_splits(), follow_tol=1e-5)
    _compare_runs(model, res, n, depth, trees)


def _forced(ctx, n, s, seed):
    """One feature of two bins (every level splits on (0, 0)), a different bin column per
    permutation: the structure cannot diverge, so every supporting value is comparable."""
    rng = np.random.default_rng(seed)
    bins_all = np.zeros((s, n, 32), np.uint8)
    bins_all[:, :, 0] = rng.integers(0, 2, size=(s, n))
    perms = np.stack([oracle.make_permutation(seed * 7 + q, n) for q in range(s)])
    y = (rng.random(n) < 0.45).astype(np.float32)
    op, yd = _from_bins(ctx, bins_all, perms, [1], y, 1)
    return op, bins_all, perms, y, yd


@pytest.mark.parametrize("n,depth", [(n, d) for n in [1, 2, 3, 4, 5, 2048, 2049, 4097, 70001] for d in (1, 3)]
                         + [(5000, 10), (2049, 8)])
def test_supporting_models_match_oracle_at_ragged_sizes(ctx, n, depth):
    s, trees = 2, 6
    op, bins_all, perms, y, yd = _forced(ctx, n, s, n + depth)
    model = train.fit_ordered(ctx, op, yd, "logloss", depth, trees, 0.3, 1.0)
    cbg.cbg_sync(ctx)
    res = oracle.fit_ordered(bins_all, 1, np.array([1], np.int32), y, "logloss", depth, trees, 0.3, 1.0, perms)
    sp = model.host_splits()
    assert np.all(sp["feature"] == 0) and np.all(sp["border"] == 0)
    assert np.all(np.abs(to_host(model.leaf_values) - res["leaf_values"]) <= 1e-5)
    assert np.all(np.abs(to_host(model.pred) - res["pred"]) <= 1e-5)
    sup = _sup_to_oracle_layout(to_host(model.sup).astype(np.float64), n)
    assert np.all(np.abs(sup - res["sup"]) <= 1e-5)


def test_bf16_ordered_gradients_train_close_to_f32(ctx):
    w = synth.logloss_1m(n=30000, trees=20)
    op = train.preprocess_ordered(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), "binary", w.max_borders, 2, a=w.a,
                                  seed=w.seed)
    losses = {}
    for dt in ("f32", "bf16"):
        m = train.fit_ordered(ctx, op, to_dev(w.y), "logloss", 6, 20, 0.1, 3.0, gh_dtype=dt)
        cbg.cbg_sync(ctx)
        losses[dt] = oracle.loss("logloss", w.y, to_host(m.pred).astype(np.float64))
    assert abs(losses["bf16"] - losses["f32"]) <= 2e-3 * losses["f32"]


def test_continuing_a_run_equals_one_run(ctx):
    """Two calls (first_tree 0 and 4, the same sup and pred) give the same model as one
    call of 8 trees."""
    import torch
    w = synth.logloss_1m(n=10000, trees=8)
    op = train.preprocess_ordered(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), "binary", w.max_borders, 3, a=w.a,
                                  seed=w.seed)
    one = train.fit_ordered(ctx, op, to_dev(w.y), "logloss", 4, 8, 0.1, 3.0)
    bufs = train.alloc_fit(op.base, 4, 8)
    a = train.fit_ordered(ctx, op, to_dev(w.y), "logloss", 4, 4, 0.1, 3.0, bufs=bufs)
    sp_a = a.splits.clone()
    b = train.fit_ordered(ctx, op, to_dev(w.y), "logloss", 4, 4, 0.1, 3.0, bufs=bufs, sup=a.sup, first_tree=4)
    cbg.cbg_sync(ctx)
    sp1 = one.host_splits()
    both = np.concatenate([train.decode_splits(sp_a), b.host_splits()])
    assert np.array_equal(both["feature"], sp1["feature"]) and np.array_equal(both["border"], sp1["border"])
    assert np.allclose(to_host(b.pred), to_host(one.pred), atol=1e-5)
    assert torch.allclose(b.sup, one.sup, atol=1e-5)


@pytest.mark.parametrize("s", [1, 3])
def test_graph_replay_equals_direct_launches(ctx, s):
    w = synth.logloss_1m(n=12000, trees=7)
    op = train.preprocess_ordered(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), "binary", w.max_borders, s, a=w.a,
                                  seed=w.seed)
    direct = train.fit_ordered(ctx, op, to_dev(w.y), "logloss", 5, 7, 0.1, 3.0)
    graph = train.fit_ordered(ctx, op, to_dev(w.y), "logloss", 5, 7, 0.1, 3.0, use_graph=True)
    cbg.cbg_sync(ctx)
    a, b = direct.host_splits(), graph.host_splits()
    assert np.array_equal(a["feature"], b["feature"]) and np.array_equal(a["border"], b["border"])
    assert np.allclose(to_host(direct.leaf_values), to_host(graph.leaf_values), rtol=1e-6, atol=1e-9)
    assert np.allclose(to_host(direct.pred), to_host(graph.pred), atol=1e-5)


def test_bad_arguments_are_rejected(ctx):
    """Invalid calls return CBG_EINVAL with a message and launch nothing."""
    import torch
    op, bins_all, perms, y, yd = _forced(ctx, 100, 2, 1)
    with pytest.raises(cbg.CbgError) as e:             # work buffer too small
        bufs = train.alloc_fit(op.base, 2, 1)
        sup = torch.zeros((2, cbg.cbg_ordered_sup_len(100)), dtype=torch.float32, device="cuda")
        cbg.cbg_boost_ordered(ctx, bufs.shape, bufs.state, 2, op.bins_pos, op.bins_t_pos, op.y_pos, op.base.bins,
                              op.base.bins_t, op.base.n_borders, yd, "logloss", "f32", 2, 1, 0, 0.1, 1.0, bufs.pred,
                              sup, bufs.g, bufs.h, bufs.leaf, bufs.splits, bufs.leaf_values, bufs.child_totals,
                              torch.empty(8, dtype=torch.uint8, device="cuda"))
    assert e.value.status == cbg.CBG_EINVAL and "work" in str(e.value)
    with pytest.raises(cbg.CbgError) as e:             # no permutation
        train.fit_ordered(ctx, train.OrderedPrepared(op.base, 0, None, op.bins_pos, op.bins_t_pos, op.y_pos), yd,
                          "logloss", 2, 1, 0.1, 1.0)
    assert e.value.status == cbg.CBG_EINVAL
    with pytest.raises(cbg.CbgError):
        cbg.cbg_ordered_sup_len(0)
    with pytest.raises(cbg.CbgError) as e:             # misaligned grouped bins
        b = torch.empty(32 * 100 + 16, dtype=torch.uint8, device="cuda")
        cbg.cbg_permute_rows(ctx, to_dev(perms[0]), 100, 1, 32, b[1:], None, None, b[1:], None, None)
    assert e.value.status == cbg.CBG_EINVAL
    cbg.cbg_sync(ctx)
