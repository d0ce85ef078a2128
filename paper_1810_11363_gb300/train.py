"""Training driver: sequences the library's C-ABI calls over torch-owned device memory.

preprocess(): permutation sigma, prior, ordered target statistics (Section 2, Eq. 1),
quantile borders and uint8 quantisation of float and TS columns (Section 5).
fit(): classic boosting of oblivious trees through cbg_boost (Sections 3-5).
ts_tables() / preprocess_new() / predict(): the inference path: full-data statistics of
new rows, quantisation with the training borders, and the model value (Section 4,
"Fast scorer").
preprocess_ordered() / fit_ordered(): ordered boosting with s permutations and the
log-scale supporting models (Section 3, Algorithm 1).
fit_combos() / predict_combos(): classic boosting with greedy feature combinations, and
their application to new rows (Section 2, "Feature combinations").
fit_batched() / autotune() / autotune_batch(): many independent problems at once, and the
histogram tilings picked by timing.
All arithmetic runs in libcbg's kernels; this module only allocates and marshals.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import cbg

SPLIT_DTYPE = np.dtype([("feature", "<i4"), ("border", "<i4"), ("score", "<f8")])


def f_pad_for(F: int) -> int:
    return max(32, (F + 31) // 32 * 32)


def decode_splits(t) -> np.ndarray:
    """cbg_split records held in a float64 tensor [..., 2] -> numpy structured array."""
    raw = t.detach().cpu().contiguous().numpy()
    return raw.view(SPLIT_DTYPE).reshape(raw.shape[:-1])


@dataclass
class Prepared:
    n: int
    F: int
    F_float: int
    F_pad: int
    perm: object
    prior: float
    ts: object
    borders: object
    n_borders: object
    bins: object
    bins_t: object
    max_bins: int
    bins4: object = None   # 4-bit packed bins (cbg_pack_bins4) when max_bins <= 16
    bits1: object = None   # 1-bit packed bins (cbg_pack_bits1) when max_bins <= 2


def preprocess(ctx: cbg.Context, x, cat, y, label_kind: str, max_borders: int, a: float = 1.0,
               seed: int = 0, prior: float | None = None, with_bins_t: bool = True) -> Prepared:
    """x: float32 [F_float][n], cat: int32/uint32 bits [C][n], y: float32 [n], all on ctx's device."""
    import torch
    dev = y.device
    n = int(y.numel())
    Ff = int(x.shape[0])
    Cc = int(cat.shape[0]) if cat is not None else 0
    F = Ff + Cc
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    cbg.cbg_make_permutation(ctx, seed, n, perm)
    if prior is None:
        pr = torch.empty(1, dtype=torch.float64, device=dev)
        cbg.cbg_prior(ctx, y, n, label_kind, pr)
        cbg.cbg_sync(ctx)
        prior = float(pr.item())
    ts = torch.empty((Cc, n), dtype=torch.float32, device=dev)
    if Cc:
        cbg.cbg_ordered_ts(ctx, cat, y, n, Cc, perm, prior, a, label_kind, ts)
    borders = torch.empty((F, max_borders), dtype=torch.float32, device=dev)
    nb = torch.empty(F, dtype=torch.int32, device=dev)
    if Ff:
        cbg.cbg_select_borders(ctx, x, n, Ff, max_borders, borders[:Ff], nb[:Ff])
    if Cc:
        cbg.cbg_select_borders(ctx, ts, n, Cc, max_borders, borders[Ff:], nb[Ff:])
    F_pad = f_pad_for(F)
    bins = torch.zeros(F_pad * n, dtype=torch.uint8, device=dev)
    bins_t = torch.empty((F, n), dtype=torch.uint8, device=dev) if with_bins_t else None
    if Ff:
        cbg.cbg_quantize(ctx, x, n, Ff, borders[:Ff], nb[:Ff], max_borders, bins, F_pad, 0, bins_t)
    if Cc:
        cbg.cbg_quantize(ctx, ts, n, Cc, borders[Ff:], nb[Ff:], max_borders, bins, F_pad, Ff, bins_t)
    cbg.cbg_sync(ctx)
    max_bins = int(nb.max().item()) + 1
    bins4 = None
    if max_bins <= 16:
        bins4 = torch.empty(((F_pad // 32 + 1) // 2) * 32 * n, dtype=torch.uint8, device=dev)
        cbg.cbg_pack_bins4(ctx, bins, n, F_pad, bins4)
    bits1 = None
    if max_bins <= 2:
        bits1 = torch.empty((F_pad // 32) * n, dtype=torch.int32, device=dev)
        cbg.cbg_pack_bits1(ctx, bins, n, F_pad, bits1)
    return Prepared(n, F, Ff, F_pad, perm, prior, ts, borders, nb, bins, bins_t, max_bins, bins4, bits1)


@dataclass
class Model:
    splits: object        # float64 tensor [T][D][2] holding cbg_split records
    leaf_values: object   # float64 [T][2^D], Newton values before the learning rate
    pred: object          # float32 [n] training predictions
    depth: int
    lr: float
    sup: object = None    # ordered boosting: float32 [s][sup_len] supporting values

    def host_splits(self) -> np.ndarray:
        return decode_splits(self.splits)


@dataclass
class FitBuffers:
    shape: object
    state: object
    pred: object
    g: object
    h: object
    leaf: object
    splits: object
    leaf_values: object
    child_totals: object


def alloc_fit(prep: Prepared, depth: int, trees: int, gh_dtype: str = "f32", tiles: dict | None = None,
              max_depth: int | None = None) -> FitBuffers:
    import torch
    dev = prep.bins.device
    shape = cbg.make_shape(prep.n, prep.F, prep.F_pad, prep.max_bins, max_depth or depth, tiles)
    state = torch.empty(cbg.cbg_tree_state_bytes(shape), dtype=torch.uint8, device=dev)
    tdt = torch.float32 if gh_dtype == "f32" else torch.bfloat16
    return FitBuffers(
        shape=shape, state=state,
        pred=torch.zeros(prep.n, dtype=torch.float32, device=dev),
        g=torch.empty(prep.n, dtype=tdt, device=dev), h=torch.empty(prep.n, dtype=tdt, device=dev),
        leaf=torch.empty(prep.n, dtype=torch.int16, device=dev),
        splits=torch.empty((max(trees, 1), depth, 2), dtype=torch.float64, device=dev),
        leaf_values=torch.empty((max(trees, 1), 1 << depth), dtype=torch.float64, device=dev),
        child_totals=torch.empty((1 << depth, 2), dtype=torch.float64, device=dev))


def fit(ctx: cbg.Context, prep: Prepared, y, loss: str, depth: int, trees: int, lr: float, l2: float,
        gh_dtype: str = "f32", tiles: dict | None = None, bufs: FitBuffers | None = None,
        use_graph: bool = False) -> Model:
    if bufs is None:
        bufs = alloc_fit(prep, depth, trees, gh_dtype, tiles)
    cbg.cbg_boost(ctx, bufs.shape, bufs.state, prep.bins, prep.n_borders, y, loss, gh_dtype, depth, trees, lr,
                  l2, bufs.pred, bufs.g, bufs.h, bufs.leaf, bufs.splits, bufs.leaf_values, bufs.child_totals,
                  bins_t=prep.bins_t, use_graph=use_graph, bins4=prep.bins4, bits1=prep.bits1)
    return Model(bufs.splits[:trees], bufs.leaf_values[:trees], bufs.pred, depth, lr)


@dataclass
class OrderedPrepared:
    """Inputs of ordered boosting: permutation 0's row-order data (the final model's
    bins) and every permutation's data in its own position order."""
    base: Prepared
    s: int
    perms: object        # int32 [s][n], position -> row; perms[0] = base.perm
    bins_pos: object     # uint8 [s][F_pad * n], grouped layout
    bins_t_pos: object   # uint8 [s][F][n]
    y_pos: object        # float32 [s][n]


def preprocess_ordered(ctx: cbg.Context, x, cat, y, label_kind: str, max_borders: int, s: int, a: float = 1.0,
                       seed: int = 0, prior: float | None = None) -> OrderedPrepared:
    """preprocess() for s permutations: sigma_q from seed + q, the ordered TS of every
    categorical column along sigma_q quantised with permutation 0's borders, and every
    permutation's bins and labels gathered into its position order."""
    import torch
    base = preprocess(ctx, x, cat, y, label_kind, max_borders, a=a, seed=seed, prior=prior)
    dev, n, F, Ff, F_pad = y.device, base.n, base.F, base.F_float, base.F_pad
    Cc = F - Ff
    perms = torch.empty((s, n), dtype=torch.int32, device=dev)
    bins_pos = torch.empty((s, F_pad * n), dtype=torch.uint8, device=dev)
    bins_t_pos = torch.empty((s, F, n), dtype=torch.uint8, device=dev)
    y_pos = torch.empty((s, n), dtype=torch.float32, device=dev)
    tmp = torch.empty_like(base.bins) if s > 1 else None
    tmp_t = torch.empty_like(base.bins_t) if s > 1 else None
    ts = torch.empty((Cc, n), dtype=torch.float32, device=dev)
    for q in range(s):
        cbg.cbg_make_permutation(ctx, seed + q, n, perms[q])
        src, src_t = base.bins, base.bins_t
        if q > 0:
            tmp.copy_(base.bins)
            tmp_t.copy_(base.bins_t)
            if Cc:
                cbg.cbg_ordered_ts(ctx, cat, y, n, Cc, perms[q], base.prior, a, label_kind, ts)
                cbg.cbg_quantize(ctx, ts, n, Cc, base.borders[Ff:], base.n_borders[Ff:], max_borders, tmp, F_pad, Ff,
                                 tmp_t)
            src, src_t = tmp, tmp_t
        cbg.cbg_permute_rows(ctx, perms[q], n, F, F_pad, src, src_t, y, bins_pos[q], bins_t_pos[q], y_pos[q])
    cbg.cbg_sync(ctx)
    return OrderedPrepared(base, s, perms, bins_pos, bins_t_pos, y_pos)


def fit_ordered(ctx: cbg.Context, op: OrderedPrepared, y, loss: str, depth: int, trees: int, lr: float, l2: float,
                gh_dtype: str = "f32", tiles: dict | None = None, bufs: FitBuffers | None = None, sup=None,
                first_tree: int = 0, use_graph: bool = False) -> Model:
    """Ordered boosting (cbg_boost_ordered). sup (float32 [s][sup_len], zeros for a fresh
    run) is continued in place when given."""
    import torch
    base = op.base
    if bufs is None:
        bufs = alloc_fit(base, depth, trees, gh_dtype, tiles)
    dev = base.bins.device
    if sup is None:
        sup = torch.zeros((op.s, cbg.cbg_ordered_sup_len(base.n)), dtype=torch.float32, device=dev)
    work = torch.empty(cbg.cbg_ordered_work_bytes(base.n, op.s, depth), dtype=torch.uint8, device=dev)
    cbg.cbg_boost_ordered(ctx, bufs.shape, bufs.state, op.s, op.bins_pos, op.bins_t_pos, op.y_pos, base.bins,
                          base.bins_t, base.n_borders, y, loss, gh_dtype, depth, trees, first_tree, lr, l2, bufs.pred,
                          sup, bufs.g, bufs.h, bufs.leaf, bufs.splits, bufs.leaf_values, bufs.child_totals, work,
                          use_graph=use_graph)
    return Model(bufs.splits[:trees], bufs.leaf_values[:trees], bufs.pred, depth, lr, sup)


@dataclass
class CombosModel:
    """Classic boosting with feature combinations: the model plus, per (tree, level), the
    combination a combination split (feature >= F) uses."""
    model: Model
    combo_items: np.ndarray     # int32 [T][D][max_complexity][3] (kind, a, b); kind -1 = unused
    combo_nb: np.ndarray        # int32 [T][D]
    combo_borders: np.ndarray   # float32 [T][D][max_borders]


def fit_combos(ctx: cbg.Context, prep: Prepared, cat, y, label_kind: str, loss: str, depth: int, trees: int,
               lr: float, l2: float, max_borders: int, max_complexity: int = 4, a: float = 1.0,
               gh_dtype: str = "f32", tiles: dict | None = None) -> CombosModel:
    """Greedy feature combinations (cbg_boost_combos) over preprocess()'s data; cat holds
    the raw category ids [C][n] the TS columns were computed from."""
    import torch
    bufs = alloc_fit(prep, depth, trees, gh_dtype, tiles)
    C_ = prep.F - prep.F_float
    work = torch.empty(cbg.cbg_combo_work_bytes(prep.n, C_, depth, max_borders, max_complexity), dtype=torch.uint8,
                       device=prep.bins.device)
    items = np.empty((max(trees, 1), depth, max_complexity, 3), np.int32)
    nb = np.empty((max(trees, 1), depth), np.int32)
    borders = np.empty((max(trees, 1), depth, max_borders), np.float32)
    cbg.cbg_boost_combos(ctx, bufs.shape, bufs.state, prep.bins, prep.bins_t, prep.n_borders, cat, C_, prep.F_float,
                         prep.perm, y, label_kind, max_borders, prep.prior, a, max_complexity, loss, gh_dtype, depth,
                         trees, lr, l2, bufs.pred, bufs.g, bufs.h, bufs.leaf, bufs.splits, bufs.leaf_values,
                         bufs.child_totals, work, items, nb, borders)
    model = Model(bufs.splits[:trees], bufs.leaf_values[:trees], bufs.pred, depth, lr)
    return CombosModel(model, items[:trees], nb[:trees], borders[:trees])


def predict_combos(ctx: cbg.Context, cm: CombosModel, prep: Prepared, cat, y, label_kind: str, bins_t_new, cat_new,
                   a: float = 1.0, max_borders: int | None = None):
    """Model value of new rows for a model with combination splits. Every combination the
    model uses becomes one extra column of the new rows: its full-data statistic (Eq. 1 with
    every training row before the new ones) from the training rows' combination values
    (cat [C][n], prep.bins_t, y), applied to the new rows' values (cat_new [C][m],
    bins_t_new [F][m]) and quantised with the combination's borders. The model's combination
    splits are renumbered to those columns and cbg_predict scores the rows.
    Returns float32 [m]."""
    import torch
    dev = bins_t_new.device
    F, m, n = prep.F, int(bins_t_new.shape[1]), prep.n
    C_ = F - prep.F_float
    mb = max_borders or cm.combo_borders.shape[-1]
    sp = cm.model.host_splits().copy()
    T, D = sp.shape
    cols = {}
    for t in range(T):
        for d in range(D):
            if sp[t, d]["feature"] >= F:
                key = tuple(tuple(int(v) for v in it) for it in cm.combo_items[t, d] if it[0] >= 0)
                if key not in cols:
                    cols[key] = (len(cols), t, d)
                sp[t, d]["feature"] = F + cols[key][0]
    K = len(cols)
    ext = torch.empty((F + K, m), dtype=torch.uint8, device=dev)
    ext[:F].copy_(bins_t_new)
    if K:
        ids_tr = torch.empty(n, dtype=torch.int32, device=dev)
        ids_new = torch.empty((1, m), dtype=torch.int32, device=dev)
        scratch = torch.empty(32 * m, dtype=torch.uint8, device=dev)
        for key, (k, t, d) in cols.items():
            cbg.cbg_combo_ids(ctx, key, cat, C_, prep.bins_t, F, n, ids_tr)
            cbg.cbg_combo_ids(ctx, key, cat_new, C_, bins_t_new, F, m, ids_new[0])
            tables = ts_tables(ctx, ids_tr[None], y, label_kind)
            ts_new = ts_apply(ctx, tables, ids_new, prep.prior, a)
            nb = int(cm.combo_nb[t, d])
            borders = torch.from_numpy(np.ascontiguousarray(cm.combo_borders[t, d, :mb])).to(dev)
            cbg.cbg_quantize(ctx, ts_new, m, 1, borders, torch.tensor([nb], dtype=torch.int32, device=dev), mb,
                             scratch, 32, 0, ext[F + k])
    rec = np.ascontiguousarray(sp).view(np.float64).reshape(T, D, 2)
    splits = torch.from_numpy(rec.copy()).to(dev)
    pred = torch.zeros(m, dtype=torch.float32, device=dev)
    cbg.cbg_predict(ctx, ext, m, F + K, splits, cm.model.leaf_values, T, D, cm.model.lr, pred)
    return pred


def grouped_from_rowmajor(bins_rm: np.ndarray) -> np.ndarray:
    """[n][F_pad] row-major bins -> the library's grouped layout (flat uint8)."""
    n, F_pad = bins_rm.shape
    return np.ascontiguousarray(bins_rm.reshape(n, F_pad // 32, 32).transpose(1, 0, 2)).reshape(-1)


def rowmajor_from_grouped(flat: np.ndarray, n: int, F_pad: int) -> np.ndarray:
    return np.ascontiguousarray(flat.reshape(F_pad // 32, n, 32).transpose(1, 0, 2)).reshape(n, F_pad)


def autotune(ctx: cbg.Context, prep: Prepared, y, loss: str, depth: int, l2: float = 3.0, gh_dtype: str = "f32",
             reps: int = 2, fixed_point: bool = False):
    """Fastest histogram tiling for this problem (cbg_autotune_tiles), timed on trees built
    from its gradients at prediction 0. fixed_point: also time the fixed-point kernel,
    whose shared-memory accumulation is not FP32. Returns (tiles dict, ms per tree)."""
    import torch
    dev = prep.bins.device
    shape = cbg.make_shape(prep.n, prep.F, prep.F_pad, prep.max_bins, depth)
    state = torch.empty(cbg.cbg_autotune_state_bytes(shape), dtype=torch.uint8, device=dev)
    tdt = torch.float32 if gh_dtype == "f32" else torch.bfloat16
    g = torch.empty(prep.n, dtype=tdt, device=dev)
    h = torch.empty(prep.n, dtype=tdt, device=dev)
    cbg.cbg_gradients(ctx, loss, y, torch.zeros(prep.n, dtype=torch.float32, device=dev), prep.n, gh_dtype, g, h)
    leaf = torch.empty(prep.n, dtype=torch.int16, device=dev)
    splits = torch.empty((depth, 2), dtype=torch.float64, device=dev)
    child = torch.empty((1 << depth, 2), dtype=torch.float64, device=dev)
    return cbg.cbg_autotune_tiles(ctx, shape, state, prep.bins, prep.n_borders, g, h, gh_dtype, depth, l2, leaf,
                                  splits, child, bins_t=prep.bins_t, reps=reps, bins4=prep.bins4,
                                  fixed_point=fixed_point, bits1=prep.bits1)


# Tilings timed on a whole batch: the shared-reduction kernel (whose histograms of a level
# then run as one launch for every problem) with clusters of 1, 2 and 8, and the
# lane-per-feature kernels per problem.
BATCH_CANDIDATES = ([{"kernel": 1, "cluster": c, "rows_per_item": 2048} for c in (1, 2, 8)] +
                    [{"kernel": 4, "cluster": 2, "rows_per_item": r} for r in (8192, 16384)] +
                    [{"kernel": 8, "cluster": 2, "rows_per_item": r} for r in (8192, 16384)] +
                    [{"kernel": 5, "cluster": 2, "rows_per_item": 8192}])


def autotune_batch(ctx: cbg.Context, preps, ys, losses, depth: int, l2: float = 3.0, gh_dtype: str = "f32",
                   rounds: int = 3, candidates=None):
    """Tiles for a batch, timed on the batch itself: every candidate tiling, applied to every
    problem, trains one round of trees and then 1 + rounds rounds (fit_batched); the time of
    the extra rounds, without the graph capture both calls pay, picks the winner. Returns
    one tiles dict per problem (all the same)."""
    import torch
    stream = torch.cuda.current_stream(preps[0].bins.device)
    best, best_ms = None, float("inf")
    for t in candidates or BATCH_CANDIDATES:
        ms = []
        for k in (1, 1 + rounds):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fit_batched(ctx, preps, ys, losses, depth, k, 0.1, l2, gh_dtype, tiles=dict(t))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        per_round = (ms[1] - ms[0]) / rounds
        if per_round < best_ms:
            best, best_ms = t, per_round
    return [dict(best) for _ in preps]


def fit_batched(ctx: cbg.Context, preps, ys, losses, depth: int, trees: int, lr: float, l2: float,
                gh_dtype: str = "f32", tiles=None, branches: int = 0):
    """Boost many independent problems together (cbg_boost_batched): one captured graph per
    round of trees, with the problems on parallel branches. tiles: None (library
    defaults), one dict for every problem, a list with one dict per problem, or "auto"
    (autotune_batch on this batch). Returns one Model per problem and the buffers."""
    if isinstance(tiles, str):
        if tiles != "auto":
            raise ValueError("tiles must be None, a dict, a list of dicts or 'auto'")
        tiles = autotune_batch(ctx, preps, ys, losses, depth, l2, gh_dtype)
    per = tiles if isinstance(tiles, list) else [tiles] * len(preps)
    bufs = [alloc_fit(p, depth, trees, gh_dtype, t) for p, t in zip(preps, per)]
    probs = []
    for p, b, y, loss in zip(preps, bufs, ys, losses):
        pr = cbg.Problem()
        pr.shape = b.shape
        pr.state = b.state.data_ptr()
        pr.state_bytes = b.state.numel()
        pr.bins = p.bins.data_ptr()
        pr.bins_t = p.bins_t.data_ptr() if p.bins_t is not None else None
        pr.n_borders = p.n_borders.data_ptr()
        pr.y = y.data_ptr()
        pr.loss = cbg.LOSS[loss]
        pr.pred = b.pred.data_ptr()
        pr.g = b.g.data_ptr()
        pr.h = b.h.data_ptr()
        pr.leaf = b.leaf.data_ptr()
        pr.splits = b.splits.data_ptr()
        pr.leaf_values = b.leaf_values.data_ptr()
        pr.child_totals = b.child_totals.data_ptr()
        probs.append(pr)
    cbg.cbg_boost_batched(ctx, probs, gh_dtype, depth, trees, lr, l2, branches)
    return [Model(b.splits[:trees], b.leaf_values[:trees], b.pred, depth, lr) for b in bufs], bufs


# ------------------------------------------------------------------ inference
@dataclass
class TSTable:
    ids: object       # uint32 (as int32 tensor) [n]: distinct category ids ascending
    sums: object      # float64 [n]: label sums
    cnts: object      # uint32 (as int32 tensor) [n]: counts
    n_unique: object  # int32 [1] on the device


def ts_tables(ctx: cbg.Context, cat, y, label_kind: str):
    """One full-data statistic table per categorical column of cat [C][n] (cbg_ts_table)."""
    import torch
    dev = y.device
    n = int(y.numel())
    out = []
    for c in range(int(cat.shape[0])):
        t = TSTable(torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.float64, device=dev),
                    torch.empty(n, dtype=torch.int32, device=dev), torch.empty(1, dtype=torch.int32, device=dev))
        cbg.cbg_ts_table(ctx, cat[c], y, n, label_kind, t.ids, t.sums, t.cnts, t.n_unique)
        out.append(t)
    return out


def ts_apply(ctx: cbg.Context, tables, cat_new, prior: float, a: float = 1.0):
    """Statistics of new rows cat_new [C][m] from the training tables: float32 [C][m]."""
    import torch
    m = int(cat_new.shape[1]) if cat_new.dim() == 2 else 0
    ts = torch.empty((len(tables), m), dtype=torch.float32, device=cat_new.device)
    for c, t in enumerate(tables):
        cbg.cbg_ts_apply(ctx, t.ids, t.sums, t.cnts, t.n_unique, cat_new[c], m, prior, a, ts[c])
    return ts


def preprocess_new(ctx: cbg.Context, prep: Prepared, tables, x_new, cat_new, a: float = 1.0):
    """Column-major bins [F][m] of new rows with the training borders: floats as given,
    categoricals through their full-data statistics (ts_apply)."""
    import torch
    m = int(x_new.shape[1]) if x_new.shape[0] else int(cat_new.shape[1])
    dev = x_new.device
    F = prep.F
    max_borders = int(prep.borders.shape[1])
    bins = torch.zeros(prep.F_pad * m, dtype=torch.uint8, device=dev)
    bins_t = torch.empty((F, m), dtype=torch.uint8, device=dev)
    Ff = prep.F_float
    if Ff:
        cbg.cbg_quantize(ctx, x_new, m, Ff, prep.borders[:Ff], prep.n_borders[:Ff], max_borders, bins, prep.F_pad, 0,
                         bins_t)
    if F > Ff:
        ts = ts_apply(ctx, tables, cat_new, prep.prior, a)
        cbg.cbg_quantize(ctx, ts, m, F - Ff, prep.borders[Ff:], prep.n_borders[Ff:], max_borders, bins, prep.F_pad,
                         Ff, bins_t)
    return bins_t


def predict(ctx: cbg.Context, model: Model, bins_t, F: int, trees: int | None = None, pred=None):
    """Model value of every row of bins_t [F][m] (cbg_predict), float32 [m]."""
    import torch
    m = int(bins_t.shape[1])
    T = int(model.splits.shape[0]) if trees is None else trees
    if pred is None:
        pred = torch.zeros(m, dtype=torch.float32, device=bins_t.device)
    cbg.cbg_predict(ctx, bins_t, m, F, model.splits, model.leaf_values, T, model.depth, model.lr, pred)
    return pred
