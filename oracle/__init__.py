"""CPU oracle for the CatBoost training hot path (arXiv 1810.11363).

TEST INFRASTRUCTURE ONLY: a plain single-threaded FP64 restatement of what the
method computes (``oracle.cpp``), loaded through ctypes. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package; the CUDA library never does, and the two share no code.

Each wrapper takes and returns numpy arrays; the passage each step follows is
cited in ``oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

LOSS = {"rmse": 0, "logloss": 1}
DTYPE = {"f32": 0, "bf16": 1}
LABEL = {"binary": 0, "real": 1}


def build(force: bool = False) -> str:
    """Compile oracle.cpp into _build/liboracle.so (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _p(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype)) if arr is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u8p, u16p, u32p = (ctypes.POINTER(t) for t in (ctypes.c_uint8, ctypes.c_uint16, ctypes.c_uint32))
            i32p, i64p = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
            f32p, f64p = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
            i64, i32, f64, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
            sig = {
                "or_splitmix64": (u64, [u64, u64]),
                "or_make_permutation": (None, [u64, i64, u32p]),
                "or_prior": (f64, [f32p, i64, i32]),
                "or_ordered_ts": (None, [u32p, f32p, i64, u32p, f64, f64, f32p, u32p, f64p]),
                "or_ordered_ts_quadratic": (None, [u32p, f32p, i64, u32p, f64, f64, f32p]),
                "or_select_borders": (i32, [f32p, i64, i32, f32p]),
                "or_quantize": (None, [f32p, i64, i32, f32p, i32p, i32, u8p, i32, i32, i64p, i64]),
                "or_gradients": (None, [i32, f32p, f64p, i64, i32, f64p, f64p]),
                "or_round_bf16": (f64, [f64]),
                "or_histogram": (None, [u8p, i64, i32, i32, f64p, f64p, u16p, i32, i32, f64p]),
                "or_split_scores": (i32, [f64p, i32, i32, i32p, i32, f64, f64p, i32p, i32p, f64p, f64p]),
                "or_update_leaf": (None, [u8p, i64, i32, i32, i32, i32, u16p]),
                "or_tree_leaf_index": (None, [u8p, i64, i32, i32p, i32p, i32, u16p]),
                "or_leaf_totals": (None, [f64p, f64p, u16p, i64, i32, f64p]),
                "or_leaf_values": (None, [f64p, i32, f64, f64p]),
                "or_apply_leaf_values": (None, [u16p, i64, f64p, f64, f64p]),
                "or_loss": (f64, [i32, f32p, f64p, i64]),
                "or_fit": (None, [u8p, i64, i32, i32, i32p, i32, f32p, i32, i32, i32, i32, f64, f64,
                                  f64p, i32p, i32p, f64p, f64p, f64p, f64p, i32p, i32p, f64, i32p]),
                "or_ts_full": (None, [u32p, f32p, i64, f64, f64, u32p, i64, f32p]),
                "or_predict": (None, [u8p, i64, i32, i32p, i32p, f64p, i32, i32, f64, f64p]),
                "or_ordered_sup_size": (i64, [i64]),
                "or_combo_ids": (None, [i32p, i32, u32p, i64, u8p, i32, u32p]),
                "or_fit_combos": (None, [u8p, i64, i32, i32, i32, i32p, i32, u32p, f32p, i32, i32, i32, f64, f64,
                                         u32p, f64, f64, i32, i32, f64p, i32p, i32p, f64p, f64p, f64p, f64p, i32p,
                                         i32p, f32p]),
                "or_fit_ordered": (None, [u8p, i64, i32, i32, i32p, i32, f32p, i32, i32, i32, f64, f64, u32p, i32,
                                          f64p, i32p, i32p, f64p, f64p, f64p, f64p, f64p, i32p, i32p, f64,
                                          i32p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


C = ctypes
_u8, _u16, _u32 = C.c_uint8, C.c_uint16, C.c_uint32
_i32, _i64, _f32, _f64 = C.c_int32, C.c_int64, C.c_float, C.c_double


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ wrappers
def splitmix64(seed: int, i: int) -> int:
    return int(lib().or_splitmix64(seed, i))


def make_permutation(seed: int, n: int) -> np.ndarray:
    perm = np.empty(n, np.uint32)
    lib().or_make_permutation(seed, n, _p(perm, _u32))
    return perm


def prior(y, label_kind: str) -> float:
    y = _c(y, np.float32)
    return float(lib().or_prior(_p(y, _f32), y.shape[0], LABEL[label_kind]))


def ordered_ts(cat, y, perm, prior_value: float, a: float = 1.0):
    """One categorical column -> (ts float32, cnt_before uint32, sum_before float64), row order."""
    cat, y, perm = _c(cat, np.uint32), _c(y, np.float32), _c(perm, np.uint32)
    n = y.shape[0]
    ts = np.empty(n, np.float32)
    cnt = np.empty(n, np.uint32)
    s = np.empty(n, np.float64)
    lib().or_ordered_ts(_p(cat, _u32), _p(y, _f32), n, _p(perm, _u32), prior_value, a,
                        _p(ts, _f32), _p(cnt, _u32), _p(s, _f64))
    return ts, cnt, s


def ordered_ts_quadratic(cat, y, perm, prior_value: float, a: float = 1.0):
    cat, y, perm = _c(cat, np.uint32), _c(y, np.float32), _c(perm, np.uint32)
    ts = np.empty(y.shape[0], np.float32)
    lib().or_ordered_ts_quadratic(_p(cat, _u32), _p(y, _f32), y.shape[0], _p(perm, _u32),
                                  prior_value, a, _p(ts, _f32))
    return ts


def select_borders(x, max_borders: int):
    """Columns of x [F][n] -> (borders float32 [F][max_borders] (+inf padded), n_borders int32 [F])."""
    x = _c(x, np.float32)
    if x.ndim == 1:
        x = x[None, :]
    F, n = x.shape
    borders = np.full((F, max_borders), np.inf, np.float32)
    nb = np.empty(F, np.int32)
    for f in range(F):
        col = np.ascontiguousarray(x[f])
        buf = np.empty(max(max_borders, 1), np.float32)
        c = lib().or_select_borders(_p(col, _f32), n, max_borders, _p(buf, _f32))
        if c < 0:
            raise ValueError(f"column {f} holds a non-finite value")
        borders[f, :c] = buf[:c]
        nb[f] = c
    return borders, nb


def quantize(x, borders, n_borders, F_pad: int, f_offset: int = 0, bins=None, rows=None):
    x = _c(x, np.float32)
    F, n = x.shape
    borders = _c(borders, np.float32)
    nb = _c(n_borders, np.int32)
    if bins is None:
        bins = np.zeros((n, F_pad), np.uint8)
    rows_a = _c(rows, np.int64) if rows is not None else None
    lib().or_quantize(_p(x, _f32), n, F, _p(borders, _f32), _p(nb, _i32), borders.shape[1],
                      _p(bins, _u8), F_pad, f_offset, _p(rows_a, _i64),
                      0 if rows_a is None else rows_a.shape[0])
    return bins


def gradients(loss: str, y, pred, dtype: str = "f32"):
    y, pred = _c(y, np.float32), _c(pred, np.float64)
    n = y.shape[0]
    g = np.empty(n, np.float64)
    h = np.empty(n, np.float64)
    lib().or_gradients(LOSS[loss], _p(y, _f32), _p(pred, _f64), n, DTYPE[dtype], _p(g, _f64), _p(h, _f64))
    return g, h


def round_bf16(v: float) -> float:
    return float(lib().or_round_bf16(v))


def histogram(bins, F: int, g, h, leaf, n_leaves: int, max_bins: int):
    bins = _c(bins, np.uint8)
    n, F_pad = bins.shape
    g, h = _c(g, np.float64), _c(h, np.float64)
    leaf_a = _c(leaf, np.uint16) if leaf is not None else None
    hist = np.empty((n_leaves, F, max_bins, 2), np.float64)
    lib().or_histogram(_p(bins, _u8), n, F_pad, F, _p(g, _f64), _p(h, _f64), _p(leaf_a, _u16),
                       n_leaves, max_bins, _p(hist, _f64))
    return hist


def split_scores(hist, n_borders, l2: float):
    """-> (scores [F][max_bins-1], best_f, best_k, best_score, second_score)."""
    hist = _c(hist, np.float64)
    L, F, max_bins, _ = hist.shape
    nb = _c(n_borders, np.int32)
    scores = np.empty((F, max(max_bins - 1, 1)), np.float64)
    bf, bk = _i32(), _i32()
    bs, ss = _f64(), _f64()
    lib().or_split_scores(_p(hist, _f64), L, F, _p(nb, _i32), max_bins, l2, _p(scores, _f64),
                          C.byref(bf), C.byref(bk), C.byref(bs), C.byref(ss))
    return scores[:, :max_bins - 1], bf.value, bk.value, bs.value, ss.value


def update_leaf(bins, f: int, k: int, d: int, leaf):
    bins = _c(bins, np.uint8)
    leaf = _c(leaf, np.uint16).copy()
    lib().or_update_leaf(_p(bins, _u8), bins.shape[0], bins.shape[1], f, k, d, _p(leaf, _u16))
    return leaf


def tree_leaf_index(bins, feats, borders):
    bins = _c(bins, np.uint8)
    f = _c(feats, np.int32)
    k = _c(borders, np.int32)
    leaf = np.empty(bins.shape[0], np.uint16)
    lib().or_tree_leaf_index(_p(bins, _u8), bins.shape[0], bins.shape[1], _p(f, _i32), _p(k, _i32),
                             f.shape[0], _p(leaf, _u16))
    return leaf


def leaf_totals(g, h, leaf, n_leaves: int):
    g, h, leaf = _c(g, np.float64), _c(h, np.float64), _c(leaf, np.uint16)
    tot = np.empty((n_leaves, 2), np.float64)
    lib().or_leaf_totals(_p(g, _f64), _p(h, _f64), _p(leaf, _u16), g.shape[0], n_leaves, _p(tot, _f64))
    return tot


def leaf_values(tot, l2: float):
    tot = _c(tot, np.float64)
    v = np.empty(tot.shape[0], np.float64)
    lib().or_leaf_values(_p(tot, _f64), tot.shape[0], l2, _p(v, _f64))
    return v


def apply_leaf_values(leaf, v, lr: float, pred):
    leaf, v = _c(leaf, np.uint16), _c(v, np.float64)
    pred = _c(pred, np.float64).copy()
    lib().or_apply_leaf_values(_p(leaf, _u16), leaf.shape[0], _p(v, _f64), lr, _p(pred, _f64))
    return pred


def loss(loss_name: str, y, pred) -> float:
    y, pred = _c(y, np.float32), _c(pred, np.float64)
    return float(lib().or_loss(LOSS[loss_name], _p(y, _f32), _p(pred, _f64), y.shape[0]))


FOLLOW_TOL = 1e-6   # relative score margin of a near-tie (the split-identity tolerance)


def _follow_args(follow, T, D):
    """follow: None, or another implementation's splits as (split_f [T][D], split_k [T][D])
    or a structured array with fields feature/border. -> (ff, fk, followed) arrays."""
    if follow is None:
        return None, None, None
    if isinstance(follow, np.ndarray) and follow.dtype.names:
        ff, fk = follow["feature"], follow["border"]
    else:
        ff, fk = follow
    ff = _c(np.asarray(ff)[:T, :D], np.int32)
    fk = _c(np.asarray(fk)[:T, :D], np.int32)
    assert ff.shape == (T, D) and fk.shape == (T, D)
    return ff, fk, np.zeros((T, D), np.int32)


def fit(bins, F: int, n_borders, y, loss_name: str, depth: int, trees: int, lr: float, l2: float,
        dtype: str = "f32", pred=None, follow=None, follow_tol: float = FOLLOW_TOL):
    """Classic boosting of `trees` oblivious trees. Returns a dict with pred (FP64),
    split_f/split_k/score/second [T][D], leaf_values [T][2^D], losses [T].
    follow: another implementation's splits [T][D]; at a level where that split scores
    within follow_tol x |best| of the oracle's best, the oracle takes it (lock step
    through near-ties). "followed" [T][D] then holds 0 (same split), 1 (near-tie,
    followed) or -1 (the followed split scores lower by more than the margin; the oracle
    kept its own)."""
    bins = _c(bins, np.uint8)
    n, F_pad = bins.shape
    nb = _c(n_borders, np.int32)
    max_bins = int(nb.max()) + 1 if nb.size else 1
    y = _c(y, np.float32)
    pred = np.zeros(n, np.float64) if pred is None else _c(pred, np.float64).copy()
    T, D = trees, depth
    sf = np.empty((T, D), np.int32)
    sk = np.empty((T, D), np.int32)
    ss = np.empty((T, D), np.float64)
    s2 = np.empty((T, D), np.float64)
    lv = np.empty((T, 1 << D), np.float64)
    losses = np.empty(T, np.float64)
    ff, fk, fl = _follow_args(follow, T, D)
    lib().or_fit(_p(bins, _u8), n, F_pad, F, _p(nb, _i32), max_bins, _p(y, _f32), LOSS[loss_name],
                 DTYPE[dtype], D, T, lr, l2, _p(pred, _f64), _p(sf, _i32), _p(sk, _i32),
                 _p(ss, _f64), _p(s2, _f64), _p(lv, _f64), _p(losses, _f64), _p(ff, _i32), _p(fk, _i32),
                 follow_tol, _p(fl, _i32))
    return {"pred": pred, "split_f": sf, "split_k": sk, "score": ss, "second": s2,
            "leaf_values": lv, "losses": losses, "max_bins": max_bins, "followed": fl}


def ordered_sup_size(n: int) -> int:
    """Number of supporting values one permutation keeps: sum_i min(2^(i+1), n)."""
    return int(lib().or_ordered_sup_size(n))


def ordered_sup_offsets(n: int) -> np.ndarray:
    """Start of each supporting model M'_i in one permutation's values (length I+2)."""
    I = (n - 1).bit_length() - 1 if n > 1 else 0
    off = [0]
    for i in range(I + 1):
        off.append(off[-1] + min(2 << i, n))
    return np.array(off, np.int64)


def fit_ordered(bins, F: int, n_borders, y, loss_name: str, depth: int, trees: int, lr: float, l2: float,
                perms, pred=None, follow=None, follow_tol: float = FOLLOW_TOL):
    """Ordered boosting (Section 3, Algorithm 1 with the log-scale supporting models).
    bins: [s][n][F_pad], permutation q's bins (row order); perms: [s][n] (position -> row).
    Returns the dict of fit() plus sup [s][n_sup], the supporting models' values.
    follow / follow_tol: the lock step of fit()."""
    bins = _c(bins, np.uint8)
    s, n, F_pad = bins.shape
    perms = _c(perms, np.uint32)
    assert perms.shape == (s, n)
    nb = _c(n_borders, np.int32)
    max_bins = int(nb.max()) + 1 if nb.size else 1
    y = _c(y, np.float32)
    pred = np.zeros(n, np.float64) if pred is None else _c(pred, np.float64).copy()
    T, D = trees, depth
    sf = np.empty((T, D), np.int32)
    sk = np.empty((T, D), np.int32)
    ss = np.empty((T, D), np.float64)
    s2 = np.empty((T, D), np.float64)
    lv = np.empty((T, 1 << D), np.float64)
    losses = np.empty(T, np.float64)
    sup = np.empty((s, ordered_sup_size(n)), np.float64)
    ff, fk, fl = _follow_args(follow, T, D)
    lib().or_fit_ordered(_p(bins, _u8), n, F_pad, F, _p(nb, _i32), max_bins, _p(y, _f32), LOSS[loss_name], D, T,
                         lr, l2, _p(perms, _u32), s, _p(pred, _f64), _p(sf, _i32), _p(sk, _i32), _p(ss, _f64),
                         _p(s2, _f64), _p(lv, _f64), _p(losses, _f64), _p(sup, _f64), _p(ff, _i32), _p(fk, _i32),
                         follow_tol, _p(fl, _i32))
    return {"pred": pred, "split_f": sf, "split_k": sk, "score": ss, "second": s2,
            "leaf_values": lv, "losses": losses, "max_bins": max_bins, "sup": sup, "followed": fl}


def combo_ids(items, cat, bins):
    """Ids of one feature combination for every row (Section 2 "Feature combinations").
    items: [(kind, a, b)] in canonical order, kind 0 = categorical column a of cat [C][n],
    kind 1 = the two-valued feature [bins[:, a] > b] of row-major bins [n][F_pad]."""
    it = _c(np.asarray(items, np.int32).reshape(-1, 3), np.int32)
    cat = _c(cat, np.uint32)
    bins = _c(bins, np.uint8)
    n = bins.shape[0]
    ids = np.empty(n, np.uint32)
    lib().or_combo_ids(_p(it, _i32), it.shape[0], _p(cat, _u32), n, _p(bins, _u8), bins.shape[1], _p(ids, _u32))
    return ids


def fit_combos(bins, F: int, F_float: int, n_borders, cat, y, loss_name: str, depth: int, trees: int, lr: float,
               l2: float, perm, prior_value: float, a: float, max_borders: int, max_complexity: int = 4, pred=None):
    """Classic boosting with greedy categorical feature combinations (Section 2). bins
    [n][F_pad] holds the F_float float columns then one TS column per categorical of cat
    [C][n]. Returns the dict of fit() plus, per (tree, level), the combination chosen
    there (combo_items [T][D][max_complexity][3], kind -1 = unused; combo_nb [T][D];
    combo_borders [T][D][max_borders]); a combination split has feature F + j."""
    bins = _c(bins, np.uint8)
    n, F_pad = bins.shape
    nb = _c(n_borders, np.int32)
    max_bins = int(nb.max()) + 1 if nb.size else 1
    cat = _c(cat, np.uint32).reshape(-1, n) if np.size(cat) else np.zeros((0, n), np.uint32)
    y = _c(y, np.float32)
    perm = _c(perm, np.uint32)
    pred = np.zeros(n, np.float64) if pred is None else _c(pred, np.float64).copy()
    T, D = trees, depth
    sf = np.empty((T, D), np.int32)
    sk = np.empty((T, D), np.int32)
    ss = np.empty((T, D), np.float64)
    s2 = np.empty((T, D), np.float64)
    lv = np.empty((T, 1 << D), np.float64)
    losses = np.empty(T, np.float64)
    items = np.empty((T, D, max_complexity, 3), np.int32)
    cnb = np.empty((T, D), np.int32)
    cbr = np.empty((T, D, max(max_borders, 1)), np.float32)
    lib().or_fit_combos(_p(bins, _u8), n, F_pad, F, F_float, _p(nb, _i32), max_bins, _p(cat, _u32), _p(y, _f32),
                        LOSS[loss_name], D, T, lr, l2, _p(perm, _u32), prior_value, a, max_borders, max_complexity,
                        _p(pred, _f64), _p(sf, _i32), _p(sk, _i32), _p(ss, _f64), _p(s2, _f64), _p(lv, _f64),
                        _p(losses, _f64), _p(items, _i32), _p(cnb, _i32), _p(cbr, _f32))
    return {"pred": pred, "split_f": sf, "split_k": sk, "score": ss, "second": s2, "leaf_values": lv,
            "losses": losses, "max_bins": max_bins, "combo_items": items, "combo_nb": cnb, "combo_borders": cbr}


def ts_full(cat, y, prior_value: float, a: float, cat_new):
    """Full-data TS of new rows (float32 [m]): every training row counts."""
    cat, y, cat_new = _c(cat, np.uint32), _c(y, np.float32), _c(cat_new, np.uint32)
    ts = np.empty(cat_new.shape[0], np.float32)
    lib().or_ts_full(_p(cat, _u32), _p(y, _f32), cat.shape[0], prior_value, a, _p(cat_new, _u32),
                     cat_new.shape[0], _p(ts, _f32))
    return ts


def predict(bins, split_f, split_k, leaf_values, lr: float):
    """Model value of every row of bins [n][F_pad] (FP64): sum over trees of lr x the leaf
    value its bins select."""
    bins = _c(bins, np.uint8)
    sf, sk = _c(split_f, np.int32), _c(split_k, np.int32)
    lv = _c(leaf_values, np.float64)
    T, D = sf.shape
    pred = np.empty(bins.shape[0], np.float64)
    lib().or_predict(_p(bins, _u8), bins.shape[0], bins.shape[1], _p(sf, _i32), _p(sk, _i32), _p(lv, _f64), T, D,
                     lr, _p(pred, _f64))
    return pred


def pmap(fn, items, workers: int = 1):
    """[fn(i) for i in items], optionally on `workers` threads. Each oracle call is
    single-threaded C code that releases the interpreter lock, so independent calls (one
    column, one run) can proceed side by side; nothing in any call changes."""
    items = list(items)
    if workers <= 1 or len(items) <= 1:
        return [fn(i) for i in items]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, items))


def preprocess(workload, F_pad: int, workers: int = 1):
    """The one-off steps of the path on the oracle: permutation, prior, ordered TS
    per categorical column, borders over floats then TS columns, quantisation.
    Returns dict(perm, prior, ts [C][n], borders [F][B], n_borders [F], bins [n][F_pad]).
    workers > 1 runs the per-column steps of different columns on that many threads."""
    w = workload
    perm = make_permutation(w.seed, w.n)
    P = prior(w.y, w.label_kind)
    ts = np.empty((w.n_cat, w.n), np.float32)
    for c, col in enumerate(pmap(lambda c: ordered_ts(w.cat[c], w.y, perm, P, w.a)[0], range(w.n_cat), workers)):
        ts[c] = col
    cols = np.concatenate([w.x, ts], axis=0) if w.n_cat else w.x
    F = cols.shape[0]
    per = pmap(lambda f: select_borders(cols[f:f + 1], w.max_borders), range(F), workers)
    borders = np.concatenate([b for b, _ in per], axis=0) if F else np.empty((0, w.max_borders), np.float32)
    nb = np.concatenate([c for _, c in per]).astype(np.int32) if F else np.empty(0, np.int32)
    bins = np.zeros((w.n, F_pad), np.uint8)
    pmap(lambda f: quantize(cols[f:f + 1], borders[f:f + 1], nb[f:f + 1], F_pad, f_offset=f, bins=bins),
         range(F), workers)
    return {"perm": perm, "prior": P, "ts": ts, "borders": borders, "n_borders": nb, "bins": bins}


def preprocess_ordered(workload, F_pad: int, s: int):
    """preprocess() for s permutations: sigma_q from seed + q, the ordered TS of every
    categorical column along each sigma_q, borders from the float columns and sigma_0's
    TS, and each permutation's bins with those borders. Returns the dict of preprocess()
    (permutation 0) plus perms [s][n] and bins_all [s][n][F_pad]."""
    w = workload
    base = preprocess(w, F_pad)
    perms = np.empty((s, w.n), np.uint32)
    bins_all = np.empty((s, w.n, F_pad), np.uint8)
    perms[0], bins_all[0] = base["perm"], base["bins"]
    for q in range(1, s):
        perms[q] = make_permutation(w.seed + q, w.n)
        bins_all[q] = base["bins"]
        if w.n_cat:
            ts = np.empty((w.n_cat, w.n), np.float32)
            for c in range(w.n_cat):
                ts[c] = ordered_ts(w.cat[c], w.y, perms[q], base["prior"], w.a)[0]
            quantize(ts, base["borders"][w.n_features - w.n_cat:], base["n_borders"][w.n_features - w.n_cat:],
                     F_pad, f_offset=w.n_features - w.n_cat, bins=bins_all[q])
    base.update(perms=perms, bins_all=bins_all)
    return base
