#!/usr/bin/env python3
"""Throughput of the CatBoost training hot path on the GPU.

One step = one pass of the whole path over the 1M-row Logloss workload (100 float +
10 categorical features, 254 borders, depth 6, 1000 trees, lr 0.05, L2 3): permutation,
prior, ordered target statistics, borders, quantisation, then 1000 boosting iterations
(gradients, 6 levels of histogram + split search + leaf update/partition, leaf values
and prediction update). Inputs are resident in HBM when a step starts; the L2 is
flushed (256 MB write) between steps.

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "trees/s and row·feature·bins/s at 1M×110 depth 6; HBM roofline %; batched vs plain"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "hist_kernel_traffic_{}.txt")   # per --hist-kernel variant
HIST_SOURCE = os.path.join(ROOT, "paper_1810_11363_gb300", "csrc", "level_hist.cuh")
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--trees", type=int, default=1000)
    p.add_argument("--gh", choices=["f32", "bf16"], default="f32")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--ref-sample-trees", type=int, default=2)
    p.add_argument("--no-graph", action="store_true", help="launch every kernel from the host instead of "
                                                           "replaying one captured tree")
    p.add_argument("--hist-kernel", choices=["auto", "pair", "lane", "lane_ld", "wp", "red", "int", "cas64"],
                   default="auto",
                   help="histogram kernel: the autotuner's pick among the FP32 kernels (auto), lane per feature "
                        "(lane), the same with a loader warp (lane_ld) or with G and H in separate warps (pair), "
                        "warp-private 16-feature "
                        "histograms (wp), shared-memory float reductions (red) or shared-memory integer "
                        "reductions of fixed-point values (int)")
    p.add_argument("--cluster", type=int, default=0, help="CTAs per histogram cluster (0 = library default)")
    p.add_argument("--rows-per-item", type=int, default=0, help="rows per CTA of a histogram work unit")
    p.add_argument("--hist-threads", type=int, default=0, help="threads per histogram CTA (0 = library default)")
    p.add_argument("--batched-problems", type=int, default=256,
                   help="problems of the batched_256 workload for the batched-vs-plain comparison (0 = skip)")
    p.add_argument("--batched-trees", type=int, default=200)
    p.add_argument("--dense-trees", type=int, default=500,
                   help="trees of the dense_400k workload (4e5 x 2000, 128 borders, depth 8; 0 = skip)")
    p.add_argument("--precision-trees", type=int, default=300,
                   help="trees of the precision_10m workload (1e7 rows, depth 10, FP32 and BF16; 0 = skip)")
    p.add_argument("--no-bf16-form", action="store_true", help="skip the BF16-storage comparison step")
    p.add_argument("--no-fixed-point-form", action="store_true",
                   help="skip the fixed-point histogram comparison step")
    p.add_argument("--scorer-trees", type=int, default=8000,
                   help="trees of the model-prediction measurement (0 = skip)")
    p.add_argument("--ordered-trees", type=int, default=200,
                   help="trees of the ordered-boosting comparison (0 skips it)")
    p.add_argument("--ordered-s", type=int, default=4, help="permutations of the ordered-boosting comparison")
    p.add_argument("--binary-trees", type=int, default=200,
                   help="trees of the binary-feature (1-bit kernel) comparison (0 skips it)")
    p.add_argument("--combo-trees", type=int, default=10,
                   help="trees of the feature-combination comparison (0 skips it)")
    p.add_argument("--combo-borders", type=int, default=15, help="borders of a combination's column")
    p.add_argument("--paper-setting-rows", type=int, default=400_000,
                   help="rows of the paper-setting workload (400000 as in the paper; smaller for profiling)")
    p.add_argument("--paper-setting-trees", type=int, default=200,
                   help="trees of the 4e5 x 2000, 15-border, depth-6 measurement (0 = skip)")
    return p.parse_args()


# ------------------------------------------------------------------ helpers
def job_time_ms(rank_ms: float, ws: int, device=None) -> float:
    """The job's timed-region duration: the maximum over ranks of each rank's duration
    (every rank trains its own replica, so the slowest one ends the job)."""
    if ws <= 1:
        return rank_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([rank_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, job_ms: float) -> float:
    """Units processed by all ranks per second of job time (weak scaling: per-rank work
    is fixed as the number of ranks grows)."""
    return units_per_rank * ws / (job_ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    maxes.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": max(maxes) if maxes else None,
                "reasons": sorted(reasons), "samples": len(sms)}


def measured_peak_hbm():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


HIST_ITEM_START = "template <typename GH, int NB, int MODE>\n__device__ __forceinline__ void hist_item("
HIST_KERNEL_START = ("template <typename GH, int NB, int MODE>\n__global__ void __launch_bounds__(512, 3) "
                     "level_hist_kernel(")
LANE_UPDATE_START = "template <int N, int C>\n__device__ __forceinline__ void lane_batched_updates("
LANE_KERNEL_START = "template <typename GH>\n__global__ void __launch_bounds__(LH_MAX_WARPS * 32, 1)\n    level_hist_lane_kernel("
LANE_LD_KERNEL_START = ("template <typename GH>\n__global__ void __launch_bounds__(LH_MAX_WARPS * 32, 1)\n"
                        "    level_hist_lane_ld_kernel(")
SOURCE_MARKERS = {"lane": (LANE_UPDATE_START, LANE_KERNEL_START),
                  "lane_ld": (LANE_UPDATE_START, LANE_LD_KERNEL_START)}


def hist_source_hash(variant="red"):
    """sha256 (first 16 hex digits) of a histogram kernel's source text: the shared-
    reduction kernels' per-item routine and kernel, or the lane kernel's update routine
    and kernel, each from its template line to its closing brace."""
    with open(HIST_SOURCE) as fh:
        src = fh.read()
    parts = []
    for marker in SOURCE_MARKERS.get(variant, (HIST_ITEM_START, HIST_KERNEL_START)):
        start = src.index(marker)
        parts.append(src[start:src.index("\n}\n", start) + 3])
    return hashlib.sha256("".join(parts).encode()).hexdigest()[:16]


def recorded_traffic_per_row(variant):
    """DRAM bytes per histogrammed row from the committed ncu summary, if it was taken on
    the current histogram source and the given kernel variant; else None."""
    try:
        with open(TRAFFIC_FILE.format(variant)) as fh:
            kv = dict(line.split(None, 1) for line in fh if line.strip() and not line.startswith("#"))
        if kv.get("source_sha256_16", "").strip() != hist_source_hash(variant):
            return None
        if kv.get("kernel_variant", "red").strip() != variant:
            return None
        return float(kv["dram_bytes_per_row"])
    except (OSError, KeyError, ValueError):
        return None


def oracle_sample(w, F_pad, trees):
    """The oracle as it stands on the host: one timed preprocessing pass and `trees`
    boosting iterations. Returns (t_prep, t_per_tree)."""
    import oracle
    t0 = time.perf_counter()
    prep = oracle.preprocess(w, F_pad)
    t1 = time.perf_counter()
    oracle.fit(prep["bins"], w.n_features, prep["n_borders"], w.y, w.loss, w.depth, trees, w.lr, w.l2)
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / trees, prep


def training_loss(loss, y, pred):
    """Training loss of float predictions (reporting only): RMSE or mean logloss, in FP64."""
    import torch
    p = pred.double()
    yy = y.double()
    if loss == "rmse":
        return float(torch.sqrt(torch.mean((yy - p) ** 2)).item())
    return float(torch.mean(torch.nn.functional.softplus(p) - yy * p).item())


def batched_comparison(ctx, n_problems, trees, dev):
    """The batching form (cbg_boost_batched: one captured graph per round, problems on
    parallel branches) against the plain form (cbg_boost with graph replay, problem by
    problem) on the first n_problems of batched_256, same trees and final losses."""
    import numpy as np
    import torch
    from paper_1810_11363_gb300 import cbg, synth, train
    ws = synth.batched_256(n_problems=n_problems, trees=trees)

    def dev_arr(a):
        return torch.from_numpy(np.ascontiguousarray(a.view(np.int32) if a.dtype == np.uint32 else a)).to(dev)

    preps, ys = [], []
    for w in ws:
        cat = dev_arr(w.cat) if w.n_cat else torch.zeros((0, w.n), dtype=torch.int32, device=dev)
        preps.append(train.preprocess(ctx, dev_arr(w.x), cat, dev_arr(w.y), w.label_kind, w.max_borders, a=w.a,
                                      seed=w.seed))
        ys.append(dev_arr(w.y))
    depth, lr, l2 = 6, 0.1, 3.0
    stream = torch.cuda.current_stream(dev)
    bufs = [train.alloc_fit(p, depth, trees) for p in preps]

    def plain():
        for p, b, y, w in zip(preps, bufs, ys, ws):
            b.pred.zero_()
            train.fit(ctx, p, y, w.loss, depth, trees, lr, l2, bufs=b, use_graph=True)

    def batched():
        return train.fit_batched(ctx, preps, ys, [w.loss for w in ws], depth, trees, lr, l2)[0]

    # histogram tiles from the autotuner, once per bin count (setup, outside the timing)
    t0 = time.perf_counter()
    auto_tiles = train.autotune_batch(ctx, preps, ys, [w.loss for w in ws], depth, l2)
    tune_s = time.perf_counter() - t0

    def batched_auto():
        return train.fit_batched(ctx, preps, ys, [w.loss for w in ws], depth, trees, lr, l2, tiles=auto_tiles)[0]

    plain()
    batched()                       # warm-up of every form
    batched_auto()
    torch.cuda.synchronize()
    out = {}
    for name, fn in (("plain", plain), ("batched", batched), ("batched_auto", batched_auto)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        preds = [b.pred for b in bufs] if name == "plain" else [m.pred for m in res]
        losses = [training_loss(w.loss, y, pr) for w, y, pr in zip(ws, ys, preds)]
        out[name] = {"trees_per_s": n_problems * trees / (ms / 1e3), "ms": ms, "losses": losses}
    def rel(name):
        return max(abs(a - b) / max(abs(a), 1e-30) for a, b in zip(out["plain"]["losses"], out[name]["losses"]))

    def rel_mean(name):
        a, b = statistics.fmean(out["plain"]["losses"]), statistics.fmean(out[name]["losses"])
        return abs(a - b) / abs(a)
    distinct = sorted({(t["kernel"], t["cluster"], t["rows_per_item"]) for t in auto_tiles})
    return {"workload": f"batched_256 first {n_problems} problems (n log-uniform 1k..200k, 10-200 floats + "
                        f"0-8 categoricals, half RMSE half Logloss), depth 6, {trees} trees each, 128 borders",
            "plain_trees_per_s": out["plain"]["trees_per_s"], "batched_trees_per_s": out["batched"]["trees_per_s"],
            "speedup": out["batched"]["trees_per_s"] / out["plain"]["trees_per_s"],
            "max_rel_final_loss_diff": rel("batched"),
            "rel_mean_final_loss_diff": rel_mean("batched"),
            "mean_final_loss_plain": statistics.fmean(out["plain"]["losses"]),
            "loss_note": "a problem whose two forms take the two sides of a near-tie split (scores within "
                         "rounding) trains on from there along its own path; the mean over problems compares "
                         "the forms",
            "batched_autotuned_trees_per_s": out["batched_auto"]["trees_per_s"],
            "speedup_autotuned": out["batched_auto"]["trees_per_s"] / out["plain"]["trees_per_s"],
            "max_rel_final_loss_diff_autotuned": rel("batched_auto"),
            "rel_mean_final_loss_diff_autotuned": rel_mean("batched_auto"),
            "autotuned_tiles": [{"kernel": k, "cluster": c, "rows_per_item": r} for k, c, r in distinct],
            "autotune_setup_s": tune_s}


def scorer_bench(ctx, dev, trees, rows=100_000, F=2000, depth=6, reps=5):
    """Model prediction (cbg_predict) on the shape of the paper's scorer comparison: 10^5
    Epsilon-shaped rows (2000 features, 129 bins) through `trees` depth-6 trees with
    random splits and leaf values. The 200 MB bin matrix is larger than L2."""
    import torch
    from paper_1810_11363_gb300 import cbg, train
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    bins_t = torch.randint(0, 129, (F, rows), dtype=torch.uint8, device=dev, generator=g)
    rec = torch.zeros((trees, depth, 2), dtype=torch.float64, device=dev)
    fk = rec.view(torch.int32).view(trees, depth, 4)
    fk[:, :, 0] = torch.randint(0, F, (trees, depth), dtype=torch.int32, device=dev, generator=g)
    fk[:, :, 1] = torch.randint(0, 128, (trees, depth), dtype=torch.int32, device=dev, generator=g)
    values = torch.randn((trees, 1 << depth), dtype=torch.float64, device=dev, generator=g)
    model = train.Model(rec, values, None, depth, 0.1)
    pred = torch.zeros(rows, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        pred.zero_()
        train.predict(ctx, model, bins_t, F, pred=pred)
    ms = []
    for _ in range(reps):
        pred.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        train.predict(ctx, model, bins_t, F, pred=pred)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    cbg.cbg_sync(ctx)
    t = statistics.median(ms)
    return {"workload": f"{rows} rows x {F} features (129 bins) through {trees} depth-{depth} trees, random "
                        "splits and leaf values", "ms": t, "rows_x_trees_per_s": rows * trees / (t / 1e3),
            "timing": f"CUDA events, median of {reps} calls after 2 untimed",
            "paper_table3_context": "CatBoost CPU scorer on Epsilon, 8000 trees: 2.4 s (1 thread), 231 ms "
                                    "(32 threads), Intel Xeon E5-2660"}


def hist_profile(ctx, prep, y, loss, depth, trees, lr, l2, gh, tiles, bufs):
    """Histogram launches of `trees` trees run with host launches and CUDA events around
    every histogram launch: (summed ms, launches, rows histogrammed)."""
    from paper_1810_11363_gb300 import cbg, train
    cbg.cbg_tree_rows_histogrammed(ctx, bufs.shape, bufs.state, reset=True)
    cbg.cbg_profile_read(ctx, reset=True)
    cbg.cbg_profile_enable(ctx, True)
    bufs.pred.zero_()
    train.fit(ctx, prep, y, loss, depth, trees, lr, l2, gh_dtype=gh, bufs=bufs, use_graph=False)
    cbg.cbg_profile_enable(ctx, False)
    ms, launches = cbg.cbg_profile_read(ctx, reset=True)
    rows = cbg.cbg_tree_rows_histogrammed(ctx, bufs.shape, bufs.state, reset=True)
    return ms, launches, rows


def config_bench(ctx, dev, w, label_kind, forms, cpu_rows=0, prior=None):
    """One of the stated workloads at its full size (inputs resident on the device,
    histogram tiles from the autotuner, set up outside the timing): preprocessing once,
    then `w.trees` trees with graph replay, timed with CUDA events, for each gradient
    storage form in `forms`. Reports trees/s, row.feature.bins/s, the final training
    loss, and the histogram kernel against the HBM roofline (algorithmic bytes: rows
    read x (F bin bytes + g + h)) from one more tree with host launches. cpu_rows > 0
    also times the oracle on a cpu_rows-row sample of the same generator (preprocessing
    and one tree), extrapolated to the full rows (its cost grows with the rows)."""
    import numpy as np
    import torch
    from paper_1810_11363_gb300 import cbg, synth, train

    def dev_arr(a):
        return torch.from_numpy(np.ascontiguousarray(a.view(np.int32) if a.dtype == np.uint32 else a)).to(dev)

    x, y = dev_arr(w.x), dev_arr(w.y)
    cat = dev_arr(w.cat) if w.n_cat else torch.zeros((0, w.n), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    train.preprocess(ctx, x, cat, y, label_kind, w.max_borders, a=w.a, seed=w.seed, prior=prior)   # warm-up
    torch.cuda.synchronize()
    e0.record(stream)
    prep = train.preprocess(ctx, x, cat, y, label_kind, w.max_borders, a=w.a, seed=w.seed, prior=prior)
    e1.record(stream)
    e1.synchronize()
    prep_ms = e0.elapsed_time(e1)
    peak, peak_kind = measured_peak_hbm()
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {"workload": f"{w.name}: n={w.n}, {w.n_float} float + {w.n_cat} categorical features, {w.max_borders} "
                       f"borders ({prep.max_bins} bins), depth {w.depth}, {w.trees} trees, lr {w.lr}, L2 {w.l2}, "
                       f"{w.loss}", "preprocess_ms": prep_ms, "forms": {}}
    for gh in forms:
        tiles, _ = train.autotune(ctx, prep, y, w.loss, w.depth, w.l2, gh_dtype=gh)
        bufs = train.alloc_fit(prep, w.depth, w.trees, gh, tiles=tiles)
        train.fit(ctx, prep, y, w.loss, w.depth, min(w.trees, 3), w.lr, w.l2, gh_dtype=gh, bufs=bufs, use_graph=True)
        bufs.pred.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        train.fit(ctx, prep, y, w.loss, w.depth, w.trees, w.lr, w.l2, gh_dtype=gh, bufs=bufs, use_graph=True)
        e1.record(stream)
        e1.synchronize()
        cbg.cbg_sync(ctx)
        ms = e0.elapsed_time(e1)
        loss = training_loss(w.loss, y, bufs.pred)
        prof_trees = min(w.trees, 5)
        hms, launches, rows = hist_profile(ctx, prep, y, w.loss, w.depth, prof_trees, w.lr, w.l2, gh, tiles, bufs)
        gh_bytes = 4 if gh == "f32" else 2
        achieved = rows * (prep.F + 2 * gh_bytes) / (hms / 1e3) / 1e9 if hms > 0 else None
        upd = rows * prep.F / (hms / 1e3) if hms > 0 else None
        out["forms"][gh] = {
            "trees_per_s": w.trees / (ms / 1e3), "ms_per_tree": ms / w.trees,
            "row_feature_bins_per_s": w.n * prep.F * prep.max_bins * w.depth * w.trees / (ms / 1e3),
            "final_loss": loss,
            "hist_tiles": {"kernel": tiles["kernel"], "cluster": tiles["cluster"],
                           "rows_per_item": tiles["rows_per_item"]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None, "peak_kind": f"{peak_kind} hbm_gbs",
                         "avg_launch_us": hms * 1e3 / max(launches, 1), "launches": launches,
                         "smem_updates_per_sm_clk": upd / (n_sms * 2070e6) if upd else None,
                         "timing": f"CUDA events around every histogram launch of {prof_trees} trees with host "
                                   "launches"}}
        del bufs
    if len(forms) > 1:
        base = out["forms"][forms[0]]["final_loss"]
        for gh in forms[1:]:
            f = out["forms"][gh]
            f["rel_final_loss_diff_vs_" + forms[0]] = abs(f["final_loss"] - base) / abs(base)
            f["speed_vs_" + forms[0]] = f["trees_per_s"] / out["forms"][forms[0]]["trees_per_s"]
    if cpu_rows > 0:
        import oracle
        gen = {"dense_400k": synth.dense_400k, "precision_10m": synth.precision_10m}[w.name]
        ws = gen(n=cpu_rows, seed=w.seed, trees=1)
        t_prep, t_tree, _ = oracle_sample(ws, train.f_pad_for(ws.n_features), 1)
        scale = w.n / cpu_rows
        t_full = scale * (t_prep + w.trees * t_tree)
        out["cpu_baseline"] = {"value": w.trees / t_full, "unit": "trees/s", "cores": 1, "kind": "oracle",
                               "sample": f"oracle on a {cpu_rows}-row sample of the same generator: preprocessing "
                                         f"{t_prep:.1f} s, one tree {t_tree:.1f} s; extrapolated x{scale:g} rows to "
                                         f"a {w.trees}-tree run (prep + trees x tree)"}
    del prep, x, y, cat
    torch.cuda.empty_cache()
    return out


def paper_setting_bench(ctx, dev, trees, n=400_000, F=2000, borders=15, depth=6):
    """Tree construction on the setting of the paper's own GPU timing (Section 6): an
    Epsilon-shaped dense problem (4e5 x 2000 N(0,1), y ~ Bernoulli(sigmoid(w.x)), w ~
    N(0, 1/2000)), 15 borders, depth 6, classic boosting, no subsampling; histogram
    tiles from the autotuner. Mean construction time per tree with graph replay."""
    import math

    import torch
    from paper_1810_11363_gb300 import cbg, train
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    x = torch.randn((F, n), generator=g, device=dev)
    wv = torch.randn(F, generator=g, device=dev) / math.sqrt(F)
    y = (torch.rand(n, generator=g, device=dev) < torch.sigmoid(wv @ x)).float()
    cat = torch.zeros((0, n), dtype=torch.int32, device=dev)
    prep = train.preprocess(ctx, x, cat, y, "binary", borders, seed=0)
    del x
    stream = torch.cuda.current_stream(dev)

    def timed(fixed_point):
        tiles, _ = train.autotune(ctx, prep, y, "logloss", depth, fixed_point=fixed_point)
        bufs = train.alloc_fit(prep, depth, trees, tiles=tiles)
        train.fit(ctx, prep, y, "logloss", depth, min(trees, 5), 0.1, 3.0, bufs=bufs, use_graph=True)   # warm-up
        bufs.pred.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        train.fit(ctx, prep, y, "logloss", depth, trees, 0.1, 3.0, bufs=bufs, use_graph=True)
        e1.record(stream)
        e1.synchronize()
        cbg.cbg_sync(ctx)
        return e0.elapsed_time(e1), tiles, training_loss("logloss", y, bufs.pred)

    ms, tiles, loss = timed(False)
    ms_fp, tiles_fp, loss_fp = timed(True)
    return {"workload": f"Epsilon-shaped {n} x {F} dense N(0,1), logistic labels, {borders} borders "
                        f"({prep.max_bins} bins), depth {depth}, {trees} trees, lr 0.1, L2 3",
            "ms_per_tree": ms / trees, "trees_per_s": trees / (ms / 1e3), "final_loss": loss,
            "hist_tiles": {"kernel": tiles["kernel"], "cluster": tiles["cluster"],
                           "rows_per_item": tiles["rows_per_item"]},
            "fixed_point_allowed": {"ms_per_tree": ms_fp / trees, "final_loss": loss_fp,
                                    "hist_tiles": {"kernel": tiles_fp["kernel"], "cluster": tiles_fp["cluster"],
                                                   "rows_per_item": tiles_fp["rows_per_item"]}},
            "paper_context": "CatBoost GPU, Epsilon, 15 bins, depth 6, classic scheme: 17.9 ms/tree on "
                             "an NVIDIA P100 (not the same data or hardware)"}


def ordered_bench(ctx, dev, x, cat, y, w, trees, s, tiles):
    """Ordered boosting (Section 3, Algorithm 1 with the log-scale supporting models) on
    logloss_1m with s permutations, against the classic scheme on the same data, both
    with graph replay: mean time per tree (after the one-off preprocessing) and the final
    training loss."""
    import torch
    from paper_1810_11363_gb300 import cbg, train
    stream = torch.cuda.current_stream(dev)
    op = train.preprocess_ordered(ctx, x, cat, y, "binary", w.max_borders, s, a=w.a, seed=w.seed)
    out = {"workload": f"logloss_1m (10^6 x 110, 255 bins), depth {w.depth}, {trees} trees, lr {w.lr}, L2 {w.l2}, "
                       f"s = {s} permutations (own TS per permutation)", "s": s, "trees": trees}
    for name in ("ordered", "classic"):
        bufs = train.alloc_fit(op.base, w.depth, trees, tiles=tiles)

        def run(T):
            bufs.pred.zero_()
            if name == "ordered":
                return train.fit_ordered(ctx, op, y, w.loss, w.depth, T, w.lr, w.l2, tiles=tiles, bufs=bufs,
                                         use_graph=True)
            return train.fit(ctx, op.base, y, w.loss, w.depth, T, w.lr, w.l2, bufs=bufs, use_graph=True)
        run(min(trees, 2 * s))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(trees)
        e1.record(stream)
        e1.synchronize()
        cbg.cbg_sync(ctx)
        ms = e0.elapsed_time(e1)
        out[name] = {"ms_per_tree": ms / trees, "trees_per_s": trees / (ms / 1e3),
                     "final_loss": training_loss(w.loss, y, bufs.pred)}
        del bufs
    out["ordered_time_over_classic"] = out["ordered"]["ms_per_tree"] / out["classic"]["ms_per_tree"]
    out["paper_context"] = ("the paper's GPU implementation: the bias-fighting (ordered) scheme is 2-3x slower "
                            "than classic boosting by design (Section 6, GPU training performance)")
    del op
    torch.cuda.empty_cache()
    return out


def binary_bench(ctx, dev, x, cat, y, w, trees):
    """Binary features (Section 5, "Dense numerical features": 1 bit per binary feature,
    32 to an integer): logloss_1m's columns quantised with one border each (every feature
    has 2 bins), trained with the 1-bit histogram kernel (tiles.kernel 9) and with the
    autotuner's pick among the uint8 kernels, both with graph replay: mean time per tree
    after the one-off preprocessing, final training loss, and the histogram's average
    launch (CUDA events around the histogram launches of 5 trees with host launches)."""
    import dataclasses

    import torch
    from paper_1810_11363_gb300 import cbg, train
    stream = torch.cuda.current_stream(dev)
    prep = train.preprocess(ctx, x, cat, y, "binary", 1, a=w.a, seed=w.seed)
    out = {"workload": f"logloss_1m columns with 1 border each (10^6 x 110, {prep.max_bins} bins), depth {w.depth}, "
                       f"{trees} trees, lr {w.lr}, L2 {w.l2}", "trees": trees}
    tiles_u8, _ = train.autotune(ctx, dataclasses.replace(prep, bins4=None, bits1=None), y, w.loss, w.depth, w.l2)
    for name, tiles in (("bits1", {"kernel": 9, "cluster": 2, "rows_per_item": 8192}), ("uint8", tiles_u8)):
        tiles = {k: tiles[k] for k in ("kernel", "cluster", "rows_per_item")}
        bufs = train.alloc_fit(prep, w.depth, trees, tiles=tiles)

        def run(T, graph=True):
            bufs.pred.zero_()
            return train.fit(ctx, prep, y, w.loss, w.depth, T, w.lr, w.l2, bufs=bufs, use_graph=graph)
        run(min(trees, 5))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(trees)
        e1.record(stream)
        e1.synchronize()
        cbg.cbg_sync(ctx)
        ms = e0.elapsed_time(e1)
        loss = training_loss(w.loss, y, bufs.pred)
        cbg.cbg_profile_read(ctx, reset=True)
        cbg.cbg_profile_enable(ctx, True)
        run(5, graph=False)
        cbg.cbg_profile_enable(ctx, False)
        torch.cuda.synchronize()
        hist_ms, launches = cbg.cbg_profile_read(ctx, reset=True)
        out[name] = {"ms_per_tree": ms / trees, "trees_per_s": trees / (ms / 1e3), "final_loss": loss,
                     "hist_tiles": tiles, "hist_avg_launch_us": hist_ms * 1e3 / max(launches, 1)}
        del bufs
    out["speed_bits1_over_uint8"] = out["uint8"]["ms_per_tree"] / out["bits1"]["ms_per_tree"]
    out["rel_final_loss_diff"] = abs(out["bits1"]["final_loss"] - out["uint8"]["final_loss"]) / out["uint8"]["final_loss"]
    del prep
    torch.cuda.empty_cache()
    return out


def combos_bench(ctx, dev, x, cat, y, w, trees, max_borders, max_complexity, tiles):
    """Classic boosting with greedy feature combinations (Section 2) on logloss_1m against
    plain classic boosting on the same data: mean time per tree (host-driven levels, one
    synchronisation per level), the combinations taken, and the final training loss."""
    import torch
    from paper_1810_11363_gb300 import cbg, train
    stream = torch.cuda.current_stream(dev)
    prep = train.preprocess(ctx, x, cat, y, "binary", w.max_borders, a=w.a, seed=w.seed)
    out = {"workload": f"logloss_1m (10^6 x 110, 255 bins), depth {w.depth}, {trees} trees, lr {w.lr}, L2 {w.l2}; "
                       f"combinations of up to {max_complexity} items, {max_borders} borders each",
           "trees": trees}
    train.fit_combos(ctx, prep, cat, y, "binary", w.loss, w.depth, 1, w.lr, w.l2, max_borders, max_complexity,
                     a=w.a, tiles=tiles)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = train.fit_combos(ctx, prep, cat, y, "binary", w.loss, w.depth, trees, w.lr, w.l2, max_borders,
                           max_complexity, a=w.a, tiles=tiles)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    sp = res.model.host_splits()
    out["combinations"] = {"ms_per_tree": ms / trees, "final_loss": training_loss(w.loss, y, res.model.pred),
                           "combination_splits": int((sp["feature"] >= prep.F).sum()),
                           "splits": int(sp["feature"].size)}
    bufs = train.alloc_fit(prep, w.depth, trees, tiles=tiles)
    train.fit(ctx, prep, y, w.loss, w.depth, 2, w.lr, w.l2, bufs=bufs, use_graph=True)
    bufs.pred.zero_()
    torch.cuda.synchronize()
    e0.record(stream)
    train.fit(ctx, prep, y, w.loss, w.depth, trees, w.lr, w.l2, bufs=bufs, use_graph=True)
    e1.record(stream)
    e1.synchronize()
    cbg.cbg_sync(ctx)
    ms = e0.elapsed_time(e1)
    out["classic"] = {"ms_per_tree": ms / trees, "final_loss": training_loss(w.loss, y, bufs.pred)}
    out["paper_context"] = ("the paper calls statistics on feature combinations the slowest and most memory "
                            "consuming part of its GPU implementation (Section 5, Categorical features)")
    del prep, bufs, res
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ arms
def workload_desc(trees: int) -> str:
    return ("logloss_1m: n=1,000,000, 100 float (40 N(0,1), 30 U(0,1), 30 lognormal) + 10 categorical "
            f"(K 2..100k, Zipf 1.1), 254 borders (255 bins), depth 6, {trees} trees, lr 0.05, L2 3, Logloss")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1810_11363_gb300 import synth, train
    import oracle
    w = synth.logloss_1m(trees=args.trees)
    F_pad = train.f_pad_for(w.n_features)
    t0 = time.perf_counter()
    prep = oracle.preprocess(w, F_pad)
    t_prep = time.perf_counter() - t0
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        oracle.fit(prep["bins"], w.n_features, prep["n_borders"], w.y, w.loss, w.depth, 1, w.lr, w.l2)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    t_tree = sum(times) / len(times)
    step = t_prep + args.trees * t_tree
    value = args.trees / step
    sample = (f"oracle (single-threaded C++ FP64) on logloss_1m: one timed preprocessing pass ({t_prep:.1f} s) "
              f"and {args.steps} timed single-tree boosting iterations after {args.warmup} untimed "
              f"({t_tree:.2f} s/tree); a {args.trees}-tree step extrapolated as prep + {args.trees} x tree")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.trees), "trees_per_step": args.trees},
            "cpu_baseline": {"value": value, "unit": "trees/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "trees/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    from paper_1810_11363_gb300 import cbg, synth, train

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    w = synth.logloss_1m(trees=args.trees)
    T, D = args.trees, w.depth

    def host(a):
        return torch.from_numpy(np.ascontiguousarray(a.view(np.int32) if a.dtype == np.uint32 else a))

    hx, hcat, hy = host(w.x).pin_memory(), host(w.cat).pin_memory(), host(w.y).pin_memory()
    x, cat, y = hx.to(dev), hcat.to(dev), hy.to(dev)
    ctx = cbg.Context(local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    use_graph = not args.no_graph

    def step(bufs, graph=use_graph):
        prep = train.preprocess(ctx, x, cat, y, "binary", w.max_borders, a=w.a, seed=w.seed)
        bufs.pred.zero_()
        model = train.fit(ctx, prep, y, w.loss, D, T, w.lr, w.l2, gh_dtype=args.gh, bufs=bufs, use_graph=graph)
        return prep, model

    prep0 = train.preprocess(ctx, x, cat, y, "binary", w.max_borders, a=w.a, seed=w.seed)
    if args.hist_kernel == "auto":
        # histogram tiles from the autotuner on this workload (setup, outside the timing)
        tiles, _ = train.autotune(ctx, prep0, y, w.loss, D, w.l2, gh_dtype=args.gh)
        tiles = {k: tiles[k] for k in ("kernel", "cluster", "rows_per_item")}
        tiles["threads"] = args.hist_threads
    else:
        tiles = {"kernel": {"wp": 2, "red": 1, "cas64": 3, "lane": 4, "pair": 5, "int": 7, "lane_ld": 8}[
                     args.hist_kernel],
                 "cluster": args.cluster,
                 "rows_per_item": args.rows_per_item, "threads": args.hist_threads}
    variant = {2: "wp", 1: "red", 3: "cas64", 4: "lane", 5: "pair", 7: "int", 0: "red", 6: "lane4",
               8: "lane_ld"}[tiles["kernel"]]
    bufs = train.alloc_fit(prep0, D, T, args.gh, tiles=tiles)
    for _ in range(args.warmup):
        step(bufs)
    torch.cuda.synchronize()
    cbg.cbg_tree_rows_histogrammed(ctx, bufs.shape, bufs.state, reset=True)
    cbg.cbg_profile_read(ctx, reset=True)
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    cbg.cbg_profile_enable(ctx, not use_graph)
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(bufs)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    cbg.cbg_profile_enable(ctx, False)
    torch.cuda.synchronize()
    clk = clocks.stop()
    hist_ms, hist_launches = cbg.cbg_profile_read(ctx, reset=True)
    rows_hist = cbg.cbg_tree_rows_histogrammed(ctx, bufs.shape, bufs.state, reset=True)
    hist_timing = "CUDA events around every histogram launch of the timed steps"
    if use_graph:
        # Events cannot time single launches inside a replayed graph: one more (untimed)
        # step launches every kernel from the host with events around each histogram launch.
        cbg.cbg_profile_enable(ctx, True)
        flush.zero_()
        step(bufs, graph=False)
        cbg.cbg_profile_enable(ctx, False)
        hist_ms, hist_launches = cbg.cbg_profile_read(ctx, reset=True)
        rows_hist = cbg.cbg_tree_rows_histogrammed(ctx, bufs.shape, bufs.state, reset=True)
        hist_timing = ("CUDA events around every histogram launch of one extra step with host launches "
                       "(the timed steps replay a captured graph)")
    total_ms = job_time_ms(sum(step_ms), ws, dev)
    value = whole_job_rate(T * args.steps, ws, total_ms)
    trees_total = T * args.steps * ws
    n, F, mb = w.n, prep0.F, prep0.max_bins
    rfb = n * F * mb * D * T * args.steps * ws / (total_ms / 1e3)

    # roofline of the histogram kernel: algorithmic bytes = rows read x (F bins + g + h)
    gh_bytes = 4 if args.gh == "f32" else 2
    alg_bytes = rows_hist * (F + 2 * gh_bytes)
    achieved = alg_bytes / (hist_ms / 1e3) / 1e9 if hist_ms > 0 else None
    peak, peak_kind = measured_peak_hbm()
    per_row = recorded_traffic_per_row(variant)
    rows_per_launch = rows_hist / max(hist_launches, 1)
    roofline = {"bound": "hbm", "kernel": {"wp": "level_hist_wp_kernel", "lane": "level_hist_lane_kernel",
                                           "pair": "level_hist_pair_kernel", "lane4": "level_hist_lane4_kernel",
                                           "lane_ld": "level_hist_lane_ld_kernel"}.get(
                    variant, "level_hist_kernel"),
                "kernel_variant": variant,
                "achieved": achieved, "peak": peak,
                "peak_kind": f"{peak_kind} hbm_gbs", "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": per_row * rows_per_launch if per_row else None,
                "alg_bytes_per_launch": alg_bytes / max(hist_launches, 1),
                "launches": hist_launches, "avg_launch_us": hist_ms * 1e3 / max(hist_launches, 1),
                "timing": hist_timing}
    # The same kernel against its own bottleneck: every (row, feature) is one read-modify-
    # write of a float2 (G, H) cell in shared memory, 16 bytes through a 128-byte-per-clock
    # shared-memory data path, so an SM can retire at most 8 updates per clock.
    clk_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    upd = rows_hist * F
    upd_rate = upd / (hist_ms / 1e3) if hist_ms > 0 else None
    per_sm_clk = upd_rate / (n_sms * clk_mhz * 1e6) if upd_rate else None
    roofline_smem = {"bound": "shared-memory updates", "kernel": roofline["kernel"],
                     "achieved": per_sm_clk, "peak": 8.0, "unit": "float2 updates per SM per clock",
                     "frac": per_sm_clk / 8.0 if per_sm_clk else None,
                     "derivation": "128 B/clock/SM shared-memory bandwidth / 16 B per float2 read + write",
                     "clock_mhz": clk_mhz, "sms": n_sms,
                     "hbm_frac_at_this_peak": (8.0 * n_sms * clk_mhz * 1e6 * (F + 2 * gh_bytes) / F / 1e9) / peak
                     if peak else None}

    # end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        h2d = hx.numel() * 4 + hcat.numel() * 4 + hy.numel() * 4
        d2h = n * 4 + T * D * 16 + T * (1 << D) * 8
        pred_h = torch.empty(n, dtype=torch.float32).pin_memory()
        sp_h = torch.empty((T, D, 2), dtype=torch.float64).pin_memory()
        lv_h = torch.empty((T, 1 << D), dtype=torch.float64).pin_memory()
        e2e_ms = []
        for i in range(1 + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xd, cd, yd = hx.to(dev, non_blocking=True), hcat.to(dev, non_blocking=True), hy.to(dev, non_blocking=True)
            prep = train.preprocess(ctx, xd, cd, yd, "binary", w.max_borders, a=w.a, seed=w.seed)
            bufs.pred.zero_()
            model = train.fit(ctx, prep, yd, w.loss, D, T, w.lr, w.l2, gh_dtype=args.gh, bufs=bufs,
                              use_graph=use_graph)
            pred_h.copy_(model.pred, non_blocking=True)
            sp_h.copy_(model.splits, non_blocking=True)
            lv_h.copy_(model.leaf_values, non_blocking=True)
            torch.cuda.synchronize()
            if i > 0:
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e = {"value": T * args.steps * ws / (sum(e2e_ms) / 1e3), "unit": "trees/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": sum(e2e_ms) / len(e2e_ms)}

    # BF16 gradient storage against FP32 on the same workload, at equal final loss
    forms = {"f32": {"trees_per_s": value, "final_loss": training_loss(w.loss, y, bufs.pred)}}
    if not args.no_bf16_form and args.gh == "f32":
        bufs16 = train.alloc_fit(prep0, D, T, "bf16", tiles=tiles)
        step(bufs16)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prep = train.preprocess(ctx, x, cat, y, "binary", w.max_borders, a=w.a, seed=w.seed)
        bufs16.pred.zero_()
        train.fit(ctx, prep, y, w.loss, D, T, w.lr, w.l2, gh_dtype="bf16", bufs=bufs16, use_graph=use_graph)
        e1.record(stream)
        e1.synchronize()
        l16 = training_loss(w.loss, y, bufs16.pred)
        forms["bf16"] = {"trees_per_s": T / (e0.elapsed_time(e1) / 1e3), "final_loss": l16,
                         "rel_final_loss_diff_vs_f32": abs(l16 - forms["f32"]["final_loss"]) /
                         abs(forms["f32"]["final_loss"])}
    # the opt-in fixed-point histogram (int32 cells, native shared integer reductions; its
    # shared-memory accumulation is not FP32) against FP32 on the same workload
    if not args.no_fixed_point_form and variant != "int":
        tiles_fp = {"kernel": 7, "cluster": 4, "rows_per_item": 4096}
        bufs_fp = train.alloc_fit(prep0, D, T, args.gh, tiles=tiles_fp)
        step(bufs_fp)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(bufs_fp)
        e1.record(stream)
        e1.synchronize()
        ms_fp = e0.elapsed_time(e1)
        l_fp = training_loss(w.loss, y, bufs_fp.pred)
        cbg.cbg_tree_rows_histogrammed(ctx, bufs_fp.shape, bufs_fp.state, reset=True)
        cbg.cbg_profile_read(ctx, reset=True)
        cbg.cbg_profile_enable(ctx, True)
        step(bufs_fp, graph=False)
        cbg.cbg_profile_enable(ctx, False)
        fp_hist_ms, fp_launches = cbg.cbg_profile_read(ctx, reset=True)
        fp_rows = cbg.cbg_tree_rows_histogrammed(ctx, bufs_fp.shape, bufs_fp.state, reset=True)
        fp_upd = fp_rows * prep0.F / (fp_hist_ms / 1e3) if fp_hist_ms > 0 else None
        fp_clk = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        fp_sms = torch.cuda.get_device_properties(dev).multi_processor_count
        fp_peak, _ = measured_peak_hbm()
        fp_achieved = fp_rows * (prep0.F + 2 * (4 if args.gh == "f32" else 2)) / (fp_hist_ms / 1e3) / 1e9 \
            if fp_hist_ms > 0 else None
        forms["fixed_point"] = {
            "trees_per_s": T / (ms_fp / 1e3), "final_loss": l_fp,
            "rel_final_loss_diff_vs_f32": abs(l_fp - forms["f32"]["final_loss"]) / abs(forms["f32"]["final_loss"]),
            "hist_tiles": tiles_fp, "accumulation": "int32 fixed-point cells in shared memory, dithered rounding, "
                                                    "FP64 cross-cluster (not the FP32 shared-memory accumulation)",
            "hist_avg_launch_us": fp_hist_ms * 1e3 / max(fp_launches, 1),
            "hist_hbm_frac": (fp_achieved / fp_peak) if (fp_achieved and fp_peak) else None,
            "hist_smem_updates_per_sm_clk": fp_upd / (fp_sms * fp_clk * 1e6) if fp_upd else None,
            "timing": "one step (preprocessing + trees) with CUDA events, after one untimed step; histogram "
                      "launches timed in one more step with host launches"}
    batched = None
    if args.batched_problems > 0 and rank == 0:
        batched = batched_comparison(ctx, args.batched_problems, args.batched_trees, dev)
    scorer = None
    if args.scorer_trees > 0 and rank == 0:
        scorer = scorer_bench(ctx, dev, args.scorer_trees)
    paper_setting = None
    if args.paper_setting_trees > 0 and rank == 0:
        paper_setting = paper_setting_bench(ctx, dev, args.paper_setting_trees, n=args.paper_setting_rows)
    ordered = None
    if args.ordered_trees > 0 and rank == 0:
        ordered = ordered_bench(ctx, dev, x, cat, y, w, args.ordered_trees, args.ordered_s, tiles)
    binary = None
    if args.binary_trees > 0 and rank == 0:
        binary = binary_bench(ctx, dev, x, cat, y, w, args.binary_trees)
    combos = None
    if args.combo_trees > 0 and rank == 0:
        combos = combos_bench(ctx, dev, x, cat, y, w, args.combo_trees, args.combo_borders, 4, tiles)
    dense = None
    if args.dense_trees > 0 and rank == 0:
        dense = config_bench(ctx, dev, synth.dense_400k(trees=args.dense_trees), "binary", ["f32"],
                             cpu_rows=0 if args.no_cpu_baseline else 20_000)
    precision = None
    if args.precision_trees > 0 and rank == 0:
        precision = config_bench(ctx, dev, synth.precision_10m(trees=args.precision_trees), "real", ["f32", "bf16"],
                                 cpu_rows=0 if args.no_cpu_baseline else 500_000)

    # kernels of ours per step: the preprocessing launches of logloss_1m (133, counted in
    # its ncu launch list: permutation sort, one sort for the ordered TS of the 10
    # categorical columns, the border sort, quantisation), the first gradients, and per
    # tree: tree_begin, 5 kernels per level (histogram, reduction, scoring, partition
    # flags, scatter; no scatter at the last level), apply, and the record kernel of a
    # graph replay
    launches_per_step = 133 + 1 + T * (1 + 5 * D - 1 + 1 + (1 if use_graph else 0))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t_prep, t_tree, _ = oracle_sample(w, prep0.F_pad, args.ref_sample_trees)
        cpu = {"value": T / (t_prep + T * t_tree), "unit": "trees/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle on logloss_1m: one preprocessing pass ({t_prep:.1f} s) + {args.ref_sample_trees} "
                         f"trees ({t_tree:.2f} s/tree); {T}-tree step extrapolated as prep + {T} x tree"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.gh, "data": "synthetic",
                "config": {"workload": workload_desc(T), "trees_per_step": T,
                           "parallelism": f"replicas x{ws}", "l2_flush": "256 MB write between steps; inputs "
                                                                             "(x 400 MB) larger than L2",
                           "gh_storage": args.gh, "graph_replay": use_graph, "hist_tiles": tiles},
                "row_feature_bins_per_s": rfb, "gpu_launches": launches_per_step * args.steps,
                "roofline": roofline, "roofline_smem": roofline_smem, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk,
                "forms": forms, "batched_vs_plain": batched, "scorer": scorer, "paper_setting": paper_setting,
                "ordered_boosting": ordered, "binary_features": binary, "feature_combinations": combos,
                "dense_400k": dense, "precision_10m": precision,
                "breakdown": {"step_ms": step_ms}}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    ctx.close()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
