"""Seeded synthetic workloads shaped like the paper's benchmarks.

The paper measures on Epsilon (4e5 x 2000 dense, Section 6 "GPU vs CPU training
performance"), Criteo (36e6 rows, 26 categorical + 13 numerical) and the eight
Table 1 datasets; none of them is available here, so these generators stand in
for them by shape: row and feature counts, bin counts, categorical
cardinalities with a Zipf frequency law, and binary or real labels.

This module produces inputs only. It holds none of the method's arithmetic
(no target statistics, no quantisation, no histograms, no scores), so both the
CUDA path and the CPU oracle can consume the same arrays without sharing any
of the method's code.

Layouts: float features are column-major ``x[F][n]`` float32, categorical ids
``cat[C][n]`` uint32 (arbitrary 32-bit ids), labels ``y[n]`` float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "zipf_ids",
    "rmse_10k",
    "logloss_1m",
    "dense_400k",
    "precision_10m",
    "batched_256",
    "interaction_xor",
    "WORKLOADS",
    "random_level_case",
]


@dataclass
class Workload:
    """One boosting problem: inputs plus the training parameters it is run with."""

    name: str
    x: np.ndarray            # float32 [F_float][n]
    cat: np.ndarray          # uint32 [C][n]
    y: np.ndarray            # float32 [n]
    loss: str                # "rmse" or "logloss"
    max_borders: int
    depth: int
    trees: int
    lr: float
    l2: float = 3.0
    a: float = 1.0           # prior weight of the ordered target statistic
    seed: int = 0            # permutation seed
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.y.shape[0])

    @property
    def n_float(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_cat(self) -> int:
        return int(self.cat.shape[0])

    @property
    def n_features(self) -> int:
        return self.n_float + self.n_cat

    @property
    def label_kind(self) -> str:
        return "binary" if self.loss == "logloss" else "real"


def zipf_ids(rng: np.random.Generator, K: int, s: float, n: int) -> np.ndarray:
    """Category indices in [0, K) with P(k) proportional to (k+1)^-s (finite support,
    inverse-CDF sampling), mapped through a random bijection of uint32 so that the
    ids look like arbitrary 32-bit hashes."""
    w = (np.arange(1, K + 1, dtype=np.float64)) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(n)
    k = np.searchsorted(cdf, u, side="right").astype(np.uint64)
    k = np.minimum(k, K - 1)
    mult = np.uint64(int(rng.integers(0, 2**31)) * 2 + 1)          # odd => bijective mod 2^32
    add = np.uint64(int(rng.integers(0, 2**32)))
    return ((k * mult + add) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def _cat_effects(rng, ids: np.ndarray, sigma: float) -> np.ndarray:
    """Per-category additive effect ~N(0, sigma^2), looked up per row."""
    uniq, inv = np.unique(ids, return_inverse=True)
    eff = rng.normal(0.0, sigma, size=uniq.shape[0])
    return eff[inv]


def _random_oblivious_tree_sum(rng, x: np.ndarray, n_trees: int, depth: int) -> np.ndarray:
    """Label model for the binary workloads: a sum of random oblivious trees over the
    float features (feature uniform, threshold = the value at a random row, leaf
    values N(0,1)), divided by sqrt(n_trees)."""
    F, n = x.shape
    z = np.zeros(n, dtype=np.float64)
    for _ in range(n_trees):
        leaf = np.zeros(n, dtype=np.int64)
        for i in range(depth):
            f = int(rng.integers(0, F))
            t = x[f, int(rng.integers(0, n))]
            leaf += (x[f] > t).astype(np.int64) << i
        vals = rng.normal(0.0, 1.0, size=1 << depth)
        z += vals[leaf]
    return z / math.sqrt(n_trees)


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def rmse_10k(n: int = 10_000, seed: int = 0) -> Workload:
    """Small real-label case: 8 N(0,1) floats, 2 categoricals (K=10, 100, Zipf 1.1),
    y = sum_k sin(x_k) + per-category effects N(0,1) + N(0, 0.1^2) noise;
    32 borders, depth 4, 20 trees, lr 0.1, L2 3."""
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, 1.0, size=(8, n)).astype(np.float32)
    cats = [zipf_ids(rng, K, 1.1, n) for K in (10, 100)]
    y = np.sin(x.astype(np.float64)).sum(axis=0)
    for c in cats:
        y += _cat_effects(rng, c, 1.0)
    y += rng.normal(0.0, 0.1, size=n)
    return Workload("rmse_10k", x, np.stack(cats), y.astype(np.float32), "rmse",
                    max_borders=32, depth=4, trees=20, lr=0.1, seed=seed)


def logloss_1m(n: int = 1_000_000, seed: int = 0, trees: int = 1000) -> Workload:
    """Criteo/Epsilon-like binary case: 100 floats (40 N(0,1), 30 U(0,1), 30
    lognormal(0,1)); 10 categoricals with K in {2,5,20,100,1k,5k,10k,30k,60k,100k},
    Zipf 1.1; y ~ Bernoulli(sigmoid(z)), z = 20 random depth-6 oblivious trees /
    sqrt(20) + per-category effects N(0, 0.3^2); 254 borders, depth 6, lr 0.05."""
    rng = np.random.default_rng(seed)
    x = np.empty((100, n), dtype=np.float32)
    x[:40] = rng.normal(0.0, 1.0, size=(40, n))
    x[40:70] = rng.random(size=(30, n))
    x[70:] = rng.lognormal(0.0, 1.0, size=(30, n))
    Ks = (2, 5, 20, 100, 1_000, 5_000, 10_000, 30_000, 60_000, 100_000)
    cats = [zipf_ids(rng, K, 1.1, n) for K in Ks]
    z = _random_oblivious_tree_sum(rng, x, 20, 6)
    for c in cats:
        z += _cat_effects(rng, c, 0.3)
    y = (rng.random(n) < _sigmoid(z)).astype(np.float32)
    return Workload("logloss_1m", x, np.stack(cats), y, "logloss",
                    max_borders=254, depth=6, trees=trees, lr=0.05, seed=seed)


def dense_400k(n: int = 400_000, F: int = 2000, seed: int = 0, trees: int = 500) -> Workload:
    """Epsilon-shaped dense case: n x 2000 N(0,1) floats, no categoricals,
    y ~ Bernoulli(sigmoid(w.x)), w ~ N(0, 1/2000); 128 borders, depth 8, lr 0.1."""
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, 1.0, size=(F, n)).astype(np.float32)
    w = rng.normal(0.0, math.sqrt(1.0 / F), size=F).astype(np.float32)
    z = w @ x
    y = (rng.random(n) < _sigmoid(z.astype(np.float64))).astype(np.float32)
    return Workload("dense_400k", x, np.zeros((0, n), np.uint32), y, "logloss",
                    max_borders=128, depth=8, trees=trees, lr=0.1, seed=seed)


def precision_10m(n: int = 10_000_000, seed: int = 0, trees: int = 300) -> Workload:
    """Large real-label case: 50 floats (25 N(0,1), 25 lognormal(0,1)); 20
    categoricals, K log-spaced 10..1e6, Zipf 1.2; y = sum sin(x_k) over the N(0,1)
    floats + per-category effects N(0,1) + Student-t(3) noise; 254 borders,
    depth 10, lr 0.1."""
    rng = np.random.default_rng(seed)
    x = np.empty((50, n), dtype=np.float32)
    x[:25] = rng.normal(0.0, 1.0, size=(25, n))
    x[25:] = rng.lognormal(0.0, 1.0, size=(25, n))
    Ks = [int(round(10 ** (1 + 5 * c / 19))) for c in range(20)]
    cats = [zipf_ids(rng, K, 1.2, n) for K in Ks]
    y = np.zeros(n, dtype=np.float64)
    for k in range(25):
        y += np.sin(x[k].astype(np.float64))
    for c in cats:
        y += _cat_effects(rng, c, 1.0)
    y += rng.standard_t(3, size=n)
    return Workload("precision_10m", x, np.stack(cats), y.astype(np.float32), "rmse",
                    max_borders=254, depth=10, trees=trees, lr=0.1, seed=seed)


def batched_256(n_problems: int = 256, n_max: int = 200_000, trees: int = 200) -> list[Workload]:
    """Many independent problems of uneven size: problem i uses seed i;
    n = floor(exp(U(ln 1e3, ln n_max))), floats ~U{10..200} N(0,1), 0..8
    categoricals (K log-uniform in 2..1e4, Zipf 1.1); even i real labels as in
    rmse_10k, odd i binary labels as in logloss_1m; 128 borders, depth 6, lr 0.1."""
    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(i)
        n = int(math.floor(math.exp(rng.uniform(math.log(1e3), math.log(n_max)))))
        F = int(rng.integers(10, 201))
        C = int(rng.integers(0, 9))
        x = rng.normal(0.0, 1.0, size=(F, n)).astype(np.float32)
        cats = []
        for _ in range(C):
            K = int(round(math.exp(rng.uniform(math.log(2), math.log(1e4)))))
            cats.append(zipf_ids(rng, max(K, 2), 1.1, n))
        cat = np.stack(cats) if cats else np.zeros((0, n), np.uint32)
        if i % 2 == 0:
            y = np.sin(x.astype(np.float64)).sum(axis=0)
            for c in cats:
                y += _cat_effects(rng, c, 1.0)
            y += rng.normal(0.0, 0.1, size=n)
            loss = "rmse"
        else:
            z = _random_oblivious_tree_sum(rng, x, 20, 6)
            for c in cats:
                z += _cat_effects(rng, c, 0.3)
            y = (rng.random(n) < _sigmoid(z)).astype(np.float64)
            loss = "logloss"
        out.append(Workload(f"batched_{i}", x, cat, y.astype(np.float32), loss,
                            max_borders=128, depth=6, trees=trees, lr=0.1, seed=i))
    return out


def interaction_xor(n: int = 24_000, seed: int = 0, depth: int = 4, trees: int = 3) -> Workload:
    """A label that only a feature combination carries (Section 2 "Feature combinations"):
    2 N(0,1) floats and 3 categoricals of 4 categories each; y ~ Bernoulli(0.85) when the
    parities of c0 and c1 differ, else Bernoulli(0.15). No single column says anything
    about y. 15 borders, Logloss."""
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(2, n)).astype(np.float32)
    k = rng.integers(0, 4, size=(3, n))
    cat = (k * 1000003 + 5).astype(np.uint32)
    z = (k[0] % 2) ^ (k[1] % 2)
    y = (rng.random(n) < np.where(z == 1, 0.85, 0.15)).astype(np.float32)
    return Workload("interaction_xor", x, cat, y, "logloss", 15, depth, trees, 0.2, 1.0, 1.0, seed)


WORKLOADS = {
    "rmse_10k": rmse_10k,
    "logloss_1m": logloss_1m,
    "dense_400k": dense_400k,
    "precision_10m": precision_10m,
}


def random_level_case(seed: int, n: int, F: int, F_pad: int, max_bins: int,
                      depth: int, integer_grads: bool = False, const_features=()):
    """Inputs for per-call tests of one tree: bins ``[n][F_pad]`` uint8 with feature f
    drawn uniformly in [0, n_bins[f]), gradients/hessians (float32), and forced
    splits (feature, border) per level. Padding columns are zero."""
    rng = np.random.default_rng(seed)
    n_bins = rng.integers(2, max_bins + 1, size=F).astype(np.int32)
    n_bins[0] = max_bins
    for f in const_features:
        n_bins[f] = 1
    bins = np.zeros((n, F_pad), dtype=np.uint8)
    for f in range(F):
        bins[:, f] = rng.integers(0, n_bins[f], size=n)
    if integer_grads:
        g = rng.integers(-8, 9, size=n).astype(np.float32)
        h = rng.integers(0, 5, size=n).astype(np.float32)
    else:
        g = rng.normal(0.0, 1.0, size=n).astype(np.float32)
        h = rng.uniform(0.0, 0.25, size=n).astype(np.float32)
    splittable = [f for f in range(F) if n_bins[f] > 1]
    forced = []
    for _ in range(depth):
        f = int(rng.choice(splittable))
        k = int(rng.integers(0, n_bins[f] - 1))
        forced.append((f, k))
    return bins, n_bins - 1, g, h, forced
