"""Thin ctypes binding of libcbg (include/cbg.h): the same entry points under the same
names, taking torch tensors (device memory) and Python scalars. Only argument
marshalling happens here; every step runs in the library's CUDA kernels.

If the library is missing or cannot be built, importing the binding's loader raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

C = ctypes
c_i32, c_i64, c_u64, c_f64, c_vp = C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_void_p

CBG_OK, CBG_EINVAL, CBG_ENOMEM, CBG_ECUDA, CBG_ETIMEOUT, CBG_EUNSUPPORTED, CBG_EDATA = 0, -1, -2, -3, -4, -5, -6
LABEL = {"binary": 0, "real": 1}
LOSS = {"rmse": 0, "logloss": 1}
DTYPE = {"f32": 0, "bf16": 1}
STATUS_NAMES = {0: "CBG_OK", -1: "CBG_EINVAL", -2: "CBG_ENOMEM", -3: "CBG_ECUDA", -4: "CBG_ETIMEOUT",
                -5: "CBG_EUNSUPPORTED", -6: "CBG_EDATA"}


class CbgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Split(C.Structure):
    _fields_ = [("feature", c_i32), ("border", c_i32), ("score", c_f64)]


class Tiles(C.Structure):
    _fields_ = [("slab_chunks", c_i32), ("rows_per_item", c_i32), ("threads", c_i32), ("blocks_per_sm", c_i32),
                ("cluster", c_i32), ("kernel", c_i32)]


class TreeShape(C.Structure):
    _fields_ = [("n", c_i64), ("F", c_i32), ("F_pad", c_i32), ("max_bins", c_i32), ("max_depth", c_i32),
                ("tiles", Tiles)]


class AutotuneArgs(C.Structure):
    _fields_ = [("shape", C.POINTER(TreeShape)), ("state", c_vp), ("state_bytes", C.c_size_t),
                ("bins", c_vp), ("bins_t", c_vp), ("n_borders", c_vp), ("g", c_vp), ("h", c_vp),
                ("gh_dtype", c_i32), ("depth", c_i32), ("l2", c_f64), ("leaf", c_vp), ("splits", c_vp),
                ("child_totals", c_vp), ("reps", c_i32), ("bins4", c_vp), ("fixed_point", c_i32),
                ("bits1", c_vp)]


class PredictArgs(C.Structure):
    _fields_ = [("bins_t", c_vp), ("n", c_i64), ("F", c_i32), ("splits", c_vp), ("leaf_values", c_vp),
                ("trees", c_i32), ("depth", c_i32), ("lr", c_f64), ("pred", c_vp)]


class LevelArgs(C.Structure):
    _fields_ = [("shape", C.POINTER(TreeShape)), ("state", c_vp), ("state_bytes", C.c_size_t),
                ("bins", c_vp), ("bins_t", c_vp), ("n_borders", c_vp), ("g", c_vp), ("h", c_vp),
                ("gh_dtype", c_i32), ("depth", c_i32), ("l2", c_f64), ("force_feature", c_i32),
                ("force_border", c_i32), ("leaf", c_vp), ("splits", c_vp), ("child_totals", c_vp),
                ("hist_out", c_vp), ("last_level", c_i32), ("challenger", c_vp), ("challenger_bins", c_vp),
                ("challenger_hist", c_vp), ("challenger_max_bins", c_i32), ("bins4", c_vp),
                ("bits1", c_vp)]


class ApplyArgs(C.Structure):
    _fields_ = [("bins", c_vp), ("n", c_i64), ("F_pad", c_i32), ("splits", c_vp), ("depth", c_i32),
                ("leaf_totals", c_vp), ("leaf_values_in", c_vp), ("l2", c_f64), ("lr", c_f64),
                ("leaf_in", c_vp), ("leaf_out", c_vp), ("pred", c_vp), ("leaf_values_out", c_vp),
                ("y", c_vp), ("loss", c_i32), ("gh_dtype", c_i32), ("g", c_vp), ("h", c_vp)]


class BoostArgs(C.Structure):
    _fields_ = [("shape", C.POINTER(TreeShape)), ("state", c_vp), ("state_bytes", C.c_size_t),
                ("bins", c_vp), ("bins_t", c_vp), ("n_borders", c_vp), ("y", c_vp), ("loss", c_i32),
                ("gh_dtype", c_i32), ("depth", c_i32), ("trees", c_i32), ("lr", c_f64), ("l2", c_f64),
                ("pred", c_vp), ("g", c_vp), ("h", c_vp), ("leaf", c_vp), ("splits", c_vp),
                ("leaf_values", c_vp), ("child_totals", c_vp), ("use_graph", c_i32), ("bins4", c_vp),
                ("bits1", c_vp)]


class Problem(C.Structure):
    _fields_ = [("shape", TreeShape), ("state", c_vp), ("state_bytes", C.c_size_t), ("bins", c_vp),
                ("bins_t", c_vp), ("n_borders", c_vp), ("y", c_vp), ("loss", c_i32), ("reserved", c_i32),
                ("pred", c_vp), ("g", c_vp), ("h", c_vp), ("leaf", c_vp), ("splits", c_vp),
                ("leaf_values", c_vp), ("child_totals", c_vp)]


class OrderedArgs(C.Structure):
    _fields_ = [("shape", C.POINTER(TreeShape)), ("state", c_vp), ("state_bytes", C.c_size_t), ("s", c_i32),
                ("bins_pos", c_vp), ("bins_t_pos", c_vp), ("y_pos", c_vp), ("bins", c_vp), ("bins_t", c_vp),
                ("n_borders", c_vp), ("y", c_vp), ("loss", c_i32), ("gh_dtype", c_i32), ("depth", c_i32),
                ("trees", c_i32), ("first_tree", c_i32), ("lr", c_f64), ("l2", c_f64), ("pred", c_vp),
                ("sup", c_vp), ("g", c_vp), ("h", c_vp), ("leaf", c_vp), ("splits", c_vp), ("leaf_values", c_vp),
                ("child_totals", c_vp), ("work", c_vp), ("work_bytes", C.c_size_t), ("use_graph", c_i32)]


class ComboItem(C.Structure):
    _fields_ = [("kind", c_i32), ("a", c_i32), ("b", c_i32)]


class ComboArgs(C.Structure):
    _fields_ = [("shape", C.POINTER(TreeShape)), ("state", c_vp), ("state_bytes", C.c_size_t), ("bins", c_vp),
                ("bins_t", c_vp), ("n_borders", c_vp), ("cat", c_vp), ("C", c_i32), ("F_float", c_i32),
                ("perm", c_vp), ("y", c_vp), ("label_kind", c_i32), ("max_borders", c_i32), ("prior", c_f64),
                ("a", c_f64), ("max_complexity", c_i32), ("loss", c_i32), ("gh_dtype", c_i32), ("depth", c_i32),
                ("trees", c_i32), ("reserved", c_i32), ("lr", c_f64), ("l2", c_f64), ("pred", c_vp), ("g", c_vp),
                ("h", c_vp), ("leaf", c_vp), ("splits", c_vp), ("leaf_values", c_vp), ("child_totals", c_vp),
                ("work", c_vp), ("work_bytes", C.c_size_t), ("combo_items", c_vp), ("combo_nb", c_vp),
                ("combo_borders", c_vp)]


# name -> (restype, argtypes); every entry point declared in include/cbg.h
SIGNATURES = {
    "cbg_version": (C.c_char_p, []),
    "cbg_ctx_create": (c_i32, [C.c_int, c_vp, C.c_size_t, C.POINTER(c_vp)]),
    "cbg_ctx_destroy": (None, [c_vp]),
    "cbg_last_error": (C.c_char_p, [c_vp]),
    "cbg_sync": (c_i32, [c_vp]),
    "cbg_test_force_wait_timeout": (c_i32, [c_vp, c_i32]),
    "cbg_set_stream": (c_i32, [c_vp, c_vp]),
    "cbg_num_sms": (C.c_int, [c_vp]),
    "cbg_make_permutation": (c_i32, [c_vp, c_u64, c_i64, c_vp]),
    "cbg_prior": (c_i32, [c_vp, c_vp, c_i64, C.c_int, c_vp]),
    "cbg_ordered_ts": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_f64, c_f64, C.c_int, c_vp, c_vp, c_vp]),
    "cbg_select_borders": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_vp, c_vp]),
    "cbg_quantize": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_i32, c_vp, c_i32, c_i32, c_vp]),
    "cbg_gradients": (c_i32, [c_vp, C.c_int, c_vp, c_vp, c_i64, C.c_int, c_vp, c_vp]),
    "cbg_tree_state_bytes": (c_i32, [C.POINTER(TreeShape), C.POINTER(C.c_size_t)]),
    "cbg_tree_begin": (c_i32, [c_vp, C.POINTER(TreeShape), c_vp, C.c_size_t, c_vp]),
    "cbg_build_level": (c_i32, [c_vp, C.POINTER(LevelArgs)]),
    "cbg_apply_tree": (c_i32, [c_vp, C.POINTER(ApplyArgs)]),
    "cbg_boost": (c_i32, [c_vp, C.POINTER(BoostArgs)]),
    "cbg_boost_batched": (c_i32, [c_vp, C.POINTER(Problem), c_i32, c_i32, c_i32, c_i32, c_f64, c_f64, c_i32]),
    "cbg_histogram_noalloc": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_i32, c_vp, c_vp, c_i32, c_vp]),
    "cbg_profile_enable": (c_i32, [c_vp, C.c_int]),
    "cbg_profile_read": (c_i32, [c_vp, C.c_int, C.POINTER(c_f64), C.POINTER(c_i64)]),
    "cbg_tree_rows_histogrammed": (c_i32, [c_vp, C.POINTER(TreeShape), c_vp, C.c_int, C.POINTER(c_i64)]),
    "cbg_ts_table": (c_i32, [c_vp, c_vp, c_vp, c_i64, C.c_int, c_vp, c_vp, c_vp, c_vp]),
    "cbg_ts_apply": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, c_f64, c_f64, c_vp]),
    "cbg_predict": (c_i32, [c_vp, C.POINTER(PredictArgs)]),
    "cbg_autotune_state_bytes": (c_i32, [C.POINTER(TreeShape), C.POINTER(C.c_size_t)]),
    "cbg_autotune_tiles": (c_i32, [c_vp, C.POINTER(AutotuneArgs), C.POINTER(Tiles), C.POINTER(c_f64)]),
    "cbg_ordered_sup_len": (c_i32, [c_i64, C.POINTER(c_i64)]),
    "cbg_ordered_work_bytes": (c_i32, [c_i64, c_i32, c_i32, C.POINTER(C.c_size_t)]),
    "cbg_permute_rows": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "cbg_boost_ordered": (c_i32, [c_vp, C.POINTER(OrderedArgs)]),
    "cbg_combo_work_bytes": (c_i32, [c_i64, c_i32, c_i32, c_i32, c_i32, C.POINTER(C.c_size_t)]),
    "cbg_boost_combos": (c_i32, [c_vp, C.POINTER(ComboArgs)]),
    "cbg_pack_bins4": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp]),
    "cbg_pack_bits1": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp]),
    "cbg_combo_ids": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_i32, c_vp, c_i32, c_i64, c_vp]),
}

_lock = threading.Lock()
_lib = None


def load(build_if_stale: bool = True):
    """Load libcbg.so (building it in-tree first when sources changed). Raises if the
    library cannot be built or loaded."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_stale else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libcbg.so not found at {path}; run __graft_entry__.build()")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(t):
    """Device pointer of a tensor (or None)."""
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


class Context:
    """Owns a cbg_ctx on one device, bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, stream=None, workspace_bytes: int = 0):
        import torch
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = c_vp()
        st = self.lib.cbg_ctx_create(device, c_vp(stream.cuda_stream), workspace_bytes, C.byref(h))
        if st != CBG_OK:
            raise CbgError(st, "cbg_ctx_create failed")
        self.h = h

    def check(self, st: int, what: str = ""):
        if st != CBG_OK:
            raise CbgError(st, f"{what}: {self.lib.cbg_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.cbg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------- entry points
def cbg_version() -> str:
    return load().cbg_version().decode()


def cbg_sync(ctx: Context):
    ctx.check(ctx.lib.cbg_sync(ctx.h), "cbg_sync")


def cbg_test_force_wait_timeout(ctx: Context, enable: bool):
    """Test hook: make the bounded waits of batched rounds captured from now on run out."""
    ctx.check(ctx.lib.cbg_test_force_wait_timeout(ctx.h, int(enable)), "cbg_test_force_wait_timeout")


def cbg_num_sms(ctx: Context) -> int:
    return int(ctx.lib.cbg_num_sms(ctx.h))


def cbg_make_permutation(ctx: Context, seed: int, n: int, perm):
    ctx.check(ctx.lib.cbg_make_permutation(ctx.h, seed, n, _p(perm)), "cbg_make_permutation")


def cbg_prior(ctx: Context, y, n: int, label_kind: str, prior_out):
    ctx.check(ctx.lib.cbg_prior(ctx.h, _p(y), n, LABEL[label_kind], _p(prior_out)), "cbg_prior")


def cbg_ordered_ts(ctx: Context, cat, y, n: int, C_: int, perm, prior: float, a: float, label_kind: str, ts,
                   cnt_before=None, sum_before=None):
    ctx.check(ctx.lib.cbg_ordered_ts(ctx.h, _p(cat), _p(y), n, C_, _p(perm), prior, a, LABEL[label_kind],
                                     _p(ts), _p(cnt_before), _p(sum_before)), "cbg_ordered_ts")


def cbg_select_borders(ctx: Context, x, n: int, F: int, max_borders: int, borders, n_borders):
    ctx.check(ctx.lib.cbg_select_borders(ctx.h, _p(x), n, F, max_borders, _p(borders), _p(n_borders)),
              "cbg_select_borders")


def cbg_quantize(ctx: Context, x, n: int, F: int, borders, n_borders, max_borders: int, bins, F_pad: int,
                 f_offset: int = 0, bins_t=None):
    ctx.check(ctx.lib.cbg_quantize(ctx.h, _p(x), n, F, _p(borders), _p(n_borders), max_borders, _p(bins),
                                   F_pad, f_offset, _p(bins_t)), "cbg_quantize")


def cbg_gradients(ctx: Context, loss: str, y, pred, n: int, gh_dtype: str, g, h):
    ctx.check(ctx.lib.cbg_gradients(ctx.h, LOSS[loss], _p(y), _p(pred), n, DTYPE[gh_dtype], _p(g), _p(h)),
              "cbg_gradients")


def make_shape(n: int, F: int, F_pad: int, max_bins: int, max_depth: int, tiles: dict | None = None) -> TreeShape:
    t = Tiles(**(tiles or {}))
    return TreeShape(n, F, F_pad, max_bins, max_depth, t)


def cbg_tree_state_bytes(shape: TreeShape) -> int:
    out = C.c_size_t()
    st = load().cbg_tree_state_bytes(C.byref(shape), C.byref(out))
    if st != CBG_OK:
        raise CbgError(st, "cbg_tree_state_bytes: invalid shape")
    return int(out.value)


def cbg_tree_begin(ctx: Context, shape: TreeShape, state, leaf):
    ctx.check(ctx.lib.cbg_tree_begin(ctx.h, C.byref(shape), _p(state), state.numel() * state.element_size(),
                                     _p(leaf)), "cbg_tree_begin")


def cbg_build_level(ctx: Context, shape: TreeShape, state, bins, n_borders, g, h, gh_dtype: str, depth: int,
                    l2: float, leaf, splits, child_totals, bins_t=None, force=None, hist_out=None,
                    last_level: bool = False, bins4=None, bits1=None):
    ff, fk = force if force is not None else (-1, -1)
    a = LevelArgs(C.pointer(shape), _p(state), state.numel() * state.element_size(), _p(bins), _p(bins_t),
                  _p(n_borders), _p(g), _p(h), DTYPE[gh_dtype], depth, l2, ff, fk, _p(leaf), _p(splits),
                  _p(child_totals), _p(hist_out), int(last_level))
    a.bins4 = _p(bins4)
    a.bits1 = _p(bits1)
    ctx.check(ctx.lib.cbg_build_level(ctx.h, C.byref(a)), "cbg_build_level")


def cbg_apply_tree(ctx: Context, n: int, depth: int, pred, *, bins=None, F_pad: int = 32, splits=None,
                   leaf_totals=None, leaf_values_in=None, l2: float = 0.0, lr: float = 1.0, leaf_in=None,
                   leaf_out=None, leaf_values_out=None, y=None, loss: str = "rmse", gh_dtype: str = "f32",
                   g=None, h=None):
    a = ApplyArgs(_p(bins), n, F_pad, _p(splits), depth, _p(leaf_totals), _p(leaf_values_in), l2, lr,
                  _p(leaf_in), _p(leaf_out), _p(pred), _p(leaf_values_out), _p(y), LOSS[loss],
                  DTYPE[gh_dtype], _p(g), _p(h))
    ctx.check(ctx.lib.cbg_apply_tree(ctx.h, C.byref(a)), "cbg_apply_tree")


def cbg_boost(ctx: Context, shape: TreeShape, state, bins, n_borders, y, loss: str, gh_dtype: str, depth: int,
              trees: int, lr: float, l2: float, pred, g, h, leaf, splits, leaf_values, child_totals,
              bins_t=None, use_graph: bool = False, bins4=None, bits1=None):
    a = BoostArgs(C.pointer(shape), _p(state), state.numel() * state.element_size(), _p(bins), _p(bins_t),
                  _p(n_borders), _p(y), LOSS[loss], DTYPE[gh_dtype], depth, trees, lr, l2, _p(pred), _p(g),
                  _p(h), _p(leaf), _p(splits), _p(leaf_values), _p(child_totals), int(use_graph), _p(bins4),
                  _p(bits1))
    ctx.check(ctx.lib.cbg_boost(ctx.h, C.byref(a)), "cbg_boost")


def cbg_profile_enable(ctx: Context, enable: bool = True):
    ctx.check(ctx.lib.cbg_profile_enable(ctx.h, int(enable)), "cbg_profile_enable")


def cbg_profile_read(ctx: Context, reset: bool = True):
    """-> (histogram device time in ms, histogram launches) since the last reset."""
    ms, launches = c_f64(), c_i64()
    ctx.check(ctx.lib.cbg_profile_read(ctx.h, int(reset), C.byref(ms), C.byref(launches)), "cbg_profile_read")
    return float(ms.value), int(launches.value)


def cbg_tree_rows_histogrammed(ctx: Context, shape: TreeShape, state, reset: bool = True) -> int:
    rows = c_i64()
    ctx.check(ctx.lib.cbg_tree_rows_histogrammed(ctx.h, C.byref(shape), _p(state), int(reset), C.byref(rows)),
              "cbg_tree_rows_histogrammed")
    return int(rows.value)


def cbg_ts_table(ctx: Context, cat, y, n: int, label_kind: str, ids, sums, cnts, n_unique):
    ctx.check(ctx.lib.cbg_ts_table(ctx.h, _p(cat), _p(y), n, LABEL[label_kind], _p(ids), _p(sums), _p(cnts),
                                   _p(n_unique)), "cbg_ts_table")


def cbg_ts_apply(ctx: Context, ids, sums, cnts, n_unique, cat_new, m: int, prior: float, a: float, ts):
    ctx.check(ctx.lib.cbg_ts_apply(ctx.h, _p(ids), _p(sums), _p(cnts), _p(n_unique), _p(cat_new), m, prior, a,
                                   _p(ts)), "cbg_ts_apply")


def cbg_predict(ctx: Context, bins_t, n: int, F: int, splits, leaf_values, trees: int, depth: int, lr: float,
                pred):
    a = PredictArgs(_p(bins_t), n, F, _p(splits), _p(leaf_values), trees, depth, lr, _p(pred))
    ctx.check(ctx.lib.cbg_predict(ctx.h, C.byref(a)), "cbg_predict")


def cbg_autotune_state_bytes(shape: TreeShape) -> int:
    out = C.c_size_t()
    st = load().cbg_autotune_state_bytes(C.byref(shape), C.byref(out))
    if st != CBG_OK:
        raise CbgError(st, "cbg_autotune_state_bytes: invalid shape")
    return int(out.value)


def cbg_autotune_tiles(ctx: Context, shape: TreeShape, state, bins, n_borders, g, h, gh_dtype: str, depth: int,
                       l2: float, leaf, splits, child_totals, bins_t=None, reps: int = 2, bins4=None,
                       fixed_point: bool = False, bits1=None):
    """Fastest histogram tiling for this problem (dict of cbg_tiles fields) and its device
    time per tree in ms. fixed_point: the fixed-point kernel (7) is a candidate too."""
    a = AutotuneArgs(C.pointer(shape), _p(state), state.numel() * state.element_size(), _p(bins), _p(bins_t),
                     _p(n_borders), _p(g), _p(h), DTYPE[gh_dtype], depth, l2, _p(leaf), _p(splits),
                     _p(child_totals), reps, _p(bins4), 1 if fixed_point else 0, _p(bits1))
    best = Tiles()
    ms = c_f64()
    ctx.check(ctx.lib.cbg_autotune_tiles(ctx.h, C.byref(a), C.byref(best), C.byref(ms)), "cbg_autotune_tiles")
    return {f: getattr(best, f) for f, _ in Tiles._fields_}, float(ms.value)


def cbg_histogram_noalloc(ctx: Context, bins, n: int, F: int, F_pad: int, max_bins: int, g, h, gh_dtype: str,
                          hist_out):
    """Root-leaf FP64 histogram into hist_out [F][max_bins][2] without any device allocation
    (scratch is a fixed 16 MiB device array inside the library; see include/cbg.h)."""
    ctx.check(ctx.lib.cbg_histogram_noalloc(ctx.h, _p(bins), n, F, F_pad, max_bins, _p(g), _p(h), DTYPE[gh_dtype],
                                            _p(hist_out)), "cbg_histogram_noalloc")


def cbg_boost_batched(ctx: Context, problems, gh_dtype: str, depth: int, trees: int, lr: float, l2: float,
                      branches: int = 0):
    """problems: sequence of Problem structures (host)."""
    arr = (Problem * len(problems))(*problems)
    ctx.check(ctx.lib.cbg_boost_batched(ctx.h, arr, len(problems), DTYPE[gh_dtype], depth, trees, lr, l2, branches),
              "cbg_boost_batched")


def cbg_ordered_sup_len(n: int) -> int:
    out = c_i64()
    st = load().cbg_ordered_sup_len(n, C.byref(out))
    if st != CBG_OK:
        raise CbgError(st, "cbg_ordered_sup_len: n must be in [1, 2^31-1]")
    return int(out.value)


def cbg_ordered_work_bytes(n: int, s: int, depth: int) -> int:
    out = C.c_size_t()
    st = load().cbg_ordered_work_bytes(n, s, depth, C.byref(out))
    if st != CBG_OK:
        raise CbgError(st, "cbg_ordered_work_bytes: invalid n, s or depth")
    return int(out.value)


def cbg_permute_rows(ctx: Context, perm, n: int, F: int, F_pad: int, bins=None, bins_t=None, y=None, bins_pos=None,
                     bins_t_pos=None, y_pos=None):
    ctx.check(ctx.lib.cbg_permute_rows(ctx.h, _p(perm), n, F, F_pad, _p(bins), _p(bins_t), _p(y), _p(bins_pos),
                                       _p(bins_t_pos), _p(y_pos)), "cbg_permute_rows")


def cbg_boost_ordered(ctx: Context, shape: TreeShape, state, s: int, bins_pos, bins_t_pos, y_pos, bins, bins_t,
                      n_borders, y, loss: str, gh_dtype: str, depth: int, trees: int, first_tree: int, lr: float,
                      l2: float, pred, sup, g, h, leaf, splits, leaf_values, child_totals, work,
                      use_graph: bool = False):
    a = OrderedArgs(C.pointer(shape), _p(state), state.numel() * state.element_size(), s, _p(bins_pos),
                    _p(bins_t_pos), _p(y_pos), _p(bins), _p(bins_t), _p(n_borders), _p(y), LOSS[loss],
                    DTYPE[gh_dtype], depth, trees, first_tree, lr, l2, _p(pred), _p(sup), _p(g), _p(h), _p(leaf),
                    _p(splits), _p(leaf_values), _p(child_totals), _p(work), work.numel() * work.element_size(),
                    int(use_graph))
    ctx.check(ctx.lib.cbg_boost_ordered(ctx.h, C.byref(a)), "cbg_boost_ordered")


def cbg_combo_work_bytes(n: int, C_: int, depth: int, max_borders: int, max_complexity: int) -> int:
    out = C.c_size_t()
    st = load().cbg_combo_work_bytes(n, C_, depth, max_borders, max_complexity, C.byref(out))
    if st != CBG_OK:
        raise CbgError(st, "cbg_combo_work_bytes: invalid arguments")
    return int(out.value)


def cbg_boost_combos(ctx: Context, shape: TreeShape, state, bins, bins_t, n_borders, cat, C_: int, F_float: int,
                     perm, y, label_kind: str, max_borders: int, prior: float, a: float, max_complexity: int,
                     loss: str, gh_dtype: str, depth: int, trees: int, lr: float, l2: float, pred, g, h, leaf,
                     splits, leaf_values, child_totals, work, combo_items, combo_nb, combo_borders):
    """combo_items (numpy int32 [trees][depth][max_complexity][3]), combo_nb (int32
    [trees][depth]) and combo_borders (float32 [trees][depth][max_borders]) are host
    outputs."""
    args = ComboArgs(C.pointer(shape), _p(state), state.numel() * state.element_size(), _p(bins), _p(bins_t),
                     _p(n_borders), _p(cat), C_, F_float, _p(perm), _p(y), LABEL[label_kind], max_borders, prior, a,
                     max_complexity, LOSS[loss], DTYPE[gh_dtype], depth, trees, 0, lr, l2, _p(pred), _p(g), _p(h),
                     _p(leaf), _p(splits), _p(leaf_values), _p(child_totals), _p(work),
                     work.numel() * work.element_size(), combo_items.ctypes.data, combo_nb.ctypes.data,
                     combo_borders.ctypes.data)
    ctx.check(ctx.lib.cbg_boost_combos(ctx.h, C.byref(args)), "cbg_boost_combos")


def cbg_pack_bits1(ctx: Context, bins, n: int, F_pad: int, bits1):
    ctx.check(ctx.lib.cbg_pack_bits1(ctx.h, _p(bins), n, F_pad, _p(bits1)), "cbg_pack_bits1")


def cbg_pack_bins4(ctx: Context, bins, n: int, F_pad: int, bins4):
    ctx.check(ctx.lib.cbg_pack_bins4(ctx.h, _p(bins), n, F_pad, _p(bins4)), "cbg_pack_bins4")


def cbg_combo_ids(ctx: Context, items, cat, C_: int, bins_t, F: int, n: int, ids):
    """items: sequence of (kind, a, b) in canonical order (host)."""
    arr = (ComboItem * len(items))(*[ComboItem(int(k), int(a), int(b)) for k, a, b in items])
    ctx.check(ctx.lib.cbg_combo_ids(ctx.h, arr, len(items), _p(cat), C_, _p(bins_t), F, n, _p(ids)), "cbg_combo_ids")
