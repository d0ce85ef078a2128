"""Full-size parity of the dense workload (400k x 2000, 129 bins, depth 8) and the
precision workload (10M rows x 50 floats + 20 categoricals, depth 10, FP32 and BF16
gradients), each against the oracle's own preprocessing and boosting:

- dense: bins and borders bit-exact, 5 trees in lock step (splits, leaf values,
  predictions within 1e-4);
- precision: the permutation, every ordered TS column (real labels: 1e-12 of the
  prefix sum of |y|), every border and bin, the histograms, child totals and splits of
  every level of a depth-10 tree, and 3 trees in lock step for FP32 and for BF16
  storage. The error of every result against the FP64 oracle is reported at the end of
  the run (conftest's parity report).
Ordered boosting and feature combinations at 10^6 rows close the module."""
import os

import numpy as np
import pytest

import oracle
from conftest import report
from gpu_util import direct_children, hist_cell_report, lockstep_check, to_dev, to_host
from paper_1810_11363_gb300 import cbg, synth, train

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

# independent oracle calls (columns, runs) side by side on the host's cores
WORKERS = max(1, min(8, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = cbg.Context(0)
    yield c
    c.close()


def _check_bins(prep, ref, n):
    """Borders, border counts and every bin of the GPU's preprocessing against the
    oracle's. Returns the row-major GPU bins."""
    nb = to_host(prep.n_borders)
    assert np.array_equal(nb, ref["n_borders"])
    b_gpu = to_host(prep.borders)
    for f in range(nb.size):
        assert np.array_equal(b_gpu[f, :nb[f]].view(np.uint32), ref["borders"][f, :nb[f]].view(np.uint32)), f
    bins = train.rowmajor_from_grouped(to_host(prep.bins), n, prep.F_pad)
    assert np.array_equal(bins, ref["bins"])
    return bins


# The histogram tiles the bench's autotuner picks on these workloads (the loader-warp
# kernel), so that the full-size parity runs in the launch configuration the bench times.
BENCH_TILES_DENSE = {"kernel": 8, "cluster": 2, "rows_per_item": 8192}
BENCH_TILES_PRECISION = {"kernel": 8, "cluster": 2, "rows_per_item": 16384}


def test_dense_400k_full_size(ctx):
    """The Epsilon-shaped workload at its stated size: 4e5 rows x 2000 N(0,1) features, 128
    borders, depth 8, lr 0.1, with the bench's histogram tiles. Preprocessing bit-exact,
    then 5 trees in lock step."""
    import torch
    w = synth.dense_400k(trees=5)
    y = to_dev(w.y)
    prep = train.preprocess(ctx, to_dev(w.x), torch.zeros((0, w.n), dtype=torch.int32, device="cuda"), y,
                            "binary", w.max_borders, a=w.a, seed=w.seed)
    model = train.fit(ctx, prep, y, w.loss, w.depth, w.trees, w.lr, w.l2, tiles=BENCH_TILES_DENSE, use_graph=True)
    cbg.cbg_sync(ctx)
    assert np.array_equal(to_host(prep.perm, np.uint32), oracle.make_permutation(w.seed, w.n))
    ref = oracle.preprocess(w, prep.F_pad, workers=WORKERS)
    _check_bins(prep, ref, w.n)
    sp = model.host_splits()
    res = oracle.fit(ref["bins"], w.n_features, ref["n_borders"], w.y, w.loss, w.depth, w.trees, w.lr, w.l2,
                     follow=sp)
    rep = lockstep_check(res, sp, to_host(model.pred), to_host(model.leaf_values), where="dense_400k")
    report("dense_400k 4e5 x 2000, 129 bins, depth 8, 5 trees", rep)


@pytest.fixture(scope="module")
def p10m(ctx):
    """The precision workload at its stated size (10^7 rows, 50 floats, 20 categoricals of
    cardinality 10 .. 10^6, Zipf 1.2, RMSE with Student-t(3) noise, 254 borders), prepared
    by the GPU and, independently, by the oracle."""
    w = synth.precision_10m(trees=3)
    P = oracle.prior(w.y, "real")
    yd = to_dev(w.y)
    prep = train.preprocess(ctx, to_dev(w.x), to_dev(w.cat), yd, "real", w.max_borders, a=w.a, seed=w.seed,
                            prior=P)
    cbg.cbg_sync(ctx)
    ref = oracle.preprocess(w, prep.F_pad, workers=WORKERS)
    return w, P, prep, ref, yd


def test_precision_10m_preprocessing(ctx, p10m):
    """Permutation bit-exact; for every categorical column the counts of earlier rows of
    the same category bit-exact, their FP64 label sums and the TS within 1e-12 of the
    prefix sum of |y| (the GPU's segmented scan adds in another order); every border and
    every bin of every column (floats and TS columns) bit-exact."""
    import torch
    w, P, prep, ref, yd = p10m
    perm = to_host(prep.perm, np.uint32)
    assert np.array_equal(perm, ref["perm"])
    C_, n = w.n_cat, w.n
    cnt = torch.empty((C_, n), dtype=torch.int32, device="cuda")
    sums = torch.empty((C_, n), dtype=torch.float64, device="cuda")
    ts = torch.empty((C_, n), dtype=torch.float32, device="cuda")
    cbg.cbg_ordered_ts(ctx, to_dev(w.cat), yd, n, C_, prep.perm, P, w.a, "real", ts, cnt, sums)
    cbg.cbg_sync(ctx)
    ts_gpu = to_host(ts)
    assert np.array_equal(ts_gpu.view(np.uint32), to_host(prep.ts).view(np.uint32))
    cnt_gpu, sums_gpu = to_host(cnt, np.uint32), to_host(sums)
    del cnt, sums, ts

    def one(c):
        t_ref, cnt_ref, s_ref = oracle.ordered_ts(w.cat[c], w.y, perm, P, w.a)
        _, _, abs_ref = oracle.ordered_ts(w.cat[c], np.abs(w.y), perm, 0.0, w.a)
        assert np.array_equal(cnt_gpu[c], cnt_ref), c
        assert np.all(np.abs(sums_gpu[c] - s_ref) <= 1e-12 * abs_ref + 1e-300), c
        scale = (abs_ref + w.a * abs(P)) / (cnt_ref + w.a)
        tol = 1e-12 * scale + np.spacing(np.abs(t_ref)).astype(np.float64)
        err = np.abs(ts_gpu[c].astype(np.float64) - t_ref.astype(np.float64))
        assert np.all(err <= tol), c
        return float(np.max(err / np.maximum(scale, 1e-300))), int(np.count_nonzero(ts_gpu[c] != t_ref))

    out = oracle.pmap(one, range(C_), WORKERS)
    report("precision_10m ordered TS (20 columns)",
           {"max |ts - fp64| / prefix mean |y|": max(o[0] for o in out),
            "rows not bit-identical": sum(o[1] for o in out)})
    _check_bins(prep, ref, n)


def _tree_levels(ctx, prep, ref, w, dtype, levels):
    """One tree of the precision workload, level by level through cbg_build_level with the
    GPU's own split choices, against the oracle at every level: each level's FP64
    histogram (cells built from rows within 1e-5 of their own sum of |g|; siblings by
    subtraction and copied cells reported), the split (identical, or a near-tie that the
    oracle then follows), the leaf index, and the FP64 child totals."""
    import torch
    from test_gpu_tree import Tree
    n, F = w.n, w.n_features
    g64, h64 = oracle.gradients("rmse", w.y, np.zeros(n), dtype)
    g32, _ = oracle.gradients("rmse", w.y, np.zeros(n), "f32")
    gd = torch.empty(n, dtype=torch.float32 if dtype == "f32" else torch.bfloat16, device="cuda")
    hd = torch.empty_like(gd)
    cbg.cbg_gradients(ctx, "rmse", to_dev(w.y), torch.zeros(n, dtype=torch.float32, device="cuda"), n, dtype, gd, hd)
    cbg.cbg_sync(ctx)
    assert np.array_equal(gd.float().cpu().numpy().astype(np.float64), g64)
    t = Tree.from_device(ctx, n, F, prep.F_pad, prep.max_bins, prep.bins, prep.bins_t, prep.n_borders, gd, hd,
                         w.depth, dtype)
    bins, nb, mb = ref["bins"], ref["n_borders"], prep.max_bins
    leaf = np.zeros(n, np.uint16)
    rows = {}
    prev_f = -1
    for d in range(levels):
        hist, sf, sk, ss, gl, child = t.level(d, w.l2, last=(d == w.depth - 1))
        jobs = [(g64, h64), (np.abs(g64), np.abs(h64))] + ([(g32, h64)] if dtype == "bf16" else [])
        hs = oracle.pmap(lambda gh: oracle.histogram(bins, F, gh[0], gh[1], leaf, 1 << d, mb), jobs, WORKERS)
        ref_h, ref_abs = hs[0], hs[1]
        wd, wo = hist_cell_report(hist, ref_h, ref_abs, direct_children(leaf, d), prev_f)
        scores, bf, bk, bs, s2 = oracle.split_scores(ref_h, nb, w.l2)
        tie = (sf, sk) != (bf, bk)
        if tie:
            assert bs - scores[sf, sk] <= oracle.FOLLOW_TOL * abs(bs), (d, (sf, sk), (bf, bk))
        assert ss == pytest.approx(scores[sf, sk], rel=1e-4)
        leaf = oracle.update_leaf(bins, sf, sk, d, leaf)
        assert np.array_equal(gl, leaf), d
        tot = oracle.leaf_totals(g64, h64, leaf, 2 << d)
        tot_abs = oracle.leaf_totals(np.abs(g64), np.abs(h64), leaf, 2 << d)
        # child totals are sums of the level's histogram cells over the split feature
        c_err = float(np.max(np.abs(child - tot) / np.maximum(tot_abs, 1e-300)))
        assert c_err <= 1e-5, d
        r = {"hist direct": wd, "hist other": wo, "child totals": c_err, "near-tie": tie}
        if dtype == "bf16":
            r["hist vs unrounded g (storage)"] = float(np.max(np.abs(hist[..., 0] - hs[2][..., 0]) /
                                                            np.maximum(ref_abs[..., 0], 1e-300)))
        rows[d] = r
        prev_f = sf
    return rows


@pytest.mark.parametrize("dtype,levels", [("f32", 10), ("bf16", 4)])
def test_precision_10m_tree_levels(ctx, p10m, dtype, levels):
    w, P, prep, ref, yd = p10m
    rows = _tree_levels(ctx, prep, ref, w, dtype, levels)
    worst = {k: max(r[k] for r in rows.values()) for k in rows[0] if k != "near-tie"}
    worst["near-ties followed"] = sum(r["near-tie"] for r in rows.values())
    report(f"precision_10m tree 1 levels 0-{levels - 1}, {dtype} g/h (worst over levels)", worst)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_precision_10m_lockstep(ctx, p10m, dtype):
    """3 depth-10 trees on the full 10^7 rows, with the bench's histogram tiles, in lock step
    with the oracle that rounds g and h to the same storage type (splits, leaf values,
    predictions within 1e-4). For BF16 storage, the error against the oracle on unrounded
    (FP32-stored) gradients, with the same tree structure, is reported too."""
    w, P, prep, ref, yd = p10m
    model = train.fit(ctx, prep, yd, w.loss, w.depth, w.trees, w.lr, w.l2, gh_dtype=dtype, tiles=BENCH_TILES_PRECISION,
                      use_graph=True)
    cbg.cbg_sync(ctx)
    sp = model.host_splits()
    pred, lv = to_host(model.pred), to_host(model.leaf_values)
    runs = [dict(dtype=dtype, follow=sp)]
    if dtype == "bf16":
        runs.append(dict(dtype="f32", follow=sp, follow_tol=1e300))   # same structure, FP32-stored g
    res = oracle.pmap(lambda kw: oracle.fit(ref["bins"], w.n_features, ref["n_borders"], w.y, w.loss, w.depth,
                                            w.trees, w.lr, w.l2, **kw), runs, WORKERS)
    rep = lockstep_check(res[0], sp, pred, lv, where=f"precision_10m {dtype}")
    rep["loss gpu / oracle"] = (float(oracle.loss(w.loss, w.y, pred.astype(np.float64))), float(res[0]["losses"][-1]))
    if dtype == "bf16":
        rep["pred vs unrounded-g oracle, max abs"] = float(np.max(np.abs(pred - res[1]["pred"])))
        rep["leaf values vs unrounded-g oracle, max rel"] = float(
            np.max(np.abs(lv - res[1]["leaf_values"]) / np.maximum(np.abs(res[1]["leaf_values"]), 1e-12)))
    report(f"precision_10m {w.trees} trees depth 10, {dtype} g/h", rep)


def test_ordered_boosting_logloss_1m_full_size(ctx):
    """Ordered boosting at the benchmark's full size (10^6 rows x 110 features, s = 4,
    depth 6, 2 trees) against the oracle on every output: the permutations and
    per-permutation bins, the structures (a split may differ only at an oracle near-tie),
    leaf values, predictions and every supporting value."""
    w = synth.logloss_1m(trees=2)
    s = 4
    op = train.preprocess_ordered(ctx, to_dev(w.x), to_dev(w.cat), to_dev(w.y), "binary", w.max_borders, s, a=w.a,
                                  seed=w.seed)
    model = train.fit_ordered(ctx, op, to_dev(w.y), w.loss, w.depth, 2, w.lr, w.l2, use_graph=True)
    cbg.cbg_sync(ctx)
    ref = oracle.preprocess_ordered(w, op.base.F_pad, s)
    perms = to_host(op.perms, np.uint32)
    assert np.array_equal(perms, ref["perms"])
    rows = np.sort(np.random.default_rng(5).choice(w.n, 20000, replace=False))
    bins_pos = to_host(op.bins_pos)
    for q in range(s):
        rm = train.rowmajor_from_grouped(bins_pos[q], w.n, op.base.F_pad)
        inv = np.empty(w.n, np.int64)
        inv[perms[q]] = np.arange(w.n)
        assert np.array_equal(rm[inv[rows]], ref["bins_all"][q][rows]), q
    sp = model.host_splits()
    res = oracle.fit_ordered(ref["bins_all"], w.n_features, ref["n_borders"], w.y, w.loss, w.depth, 2, w.lr, w.l2,
                             ref["perms"], follow=sp, follow_tol=1e-5)
    assert np.all(res["followed"] >= 0), np.argwhere(res["followed"] < 0).tolist()
    assert np.array_equal(sp["feature"], res["split_f"]) and np.array_equal(sp["border"], res["split_k"])
    assert np.allclose(to_host(model.leaf_values), res["leaf_values"], rtol=1e-4, atol=1e-6)
    assert np.all(np.abs(to_host(model.pred) - res["pred"]) <= 1e-4)
    report("ordered boosting logloss_1m s=4, 2 trees",
           {"near_ties_followed": int((res["followed"] == 1).sum()),
            "pred_max_abs": float(np.abs(to_host(model.pred) - res["pred"]).max())})
    off = oracle.ordered_sup_offsets(w.n)
    sup = to_host(model.sup).astype(np.float64)
    for i in range(len(off) - 1):
        held = off[i + 1] - off[i]
        assert np.all(np.abs(sup[:, (2 << i):(2 << i) + held] - res["sup"][:, off[i]:off[i + 1]]) <= 1e-4), i


def test_combinations_interaction_1m(ctx):
    """Feature combinations at 10^6 rows (the XOR interaction workload, depth 3, 3 trees,
    up to 3 items, 15 borders; the oracle's best and runner-up differ by at least 1.1e-2
    at every level) against the oracle: structures, combinations and their borders, leaf
    values and predictions."""
    from test_gpu_combos import _compare, _run_both
    w = synth.interaction_xor(1_000_000, seed=7)
    got, res = _run_both(ctx, w, depth=3, trees=3, max_borders=15, mc=3)
    compared, n_combo = _compare(got, res, w.n_features, 3, 3)
    assert compared == 3 and n_combo >= 4
