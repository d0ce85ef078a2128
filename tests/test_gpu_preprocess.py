"""GPU parity of the one-off steps against the oracle: permutation, prior, ordered TS
(Eq. 1), borders and quantisation (Section 5). Integer and selection results are
bit-exact; real-label TS sums within 1e-12 of the prefix sum of |y|."""
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


def _perm(ctx, seed, n):
    import torch
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    cbg.cbg_make_permutation(ctx, seed, n, p)
    cbg.cbg_sync(ctx)
    return to_host(p, np.uint32)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 5), (1000, 0), (4097, 7), (300001, 123)])
def test_permutation_bit_exact(ctx, n, seed):
    assert np.array_equal(_perm(ctx, seed, n), oracle.make_permutation(seed, n))


def test_prior(ctx):
    import torch
    rng = np.random.default_rng(0)
    yb = (rng.random(100003) < 0.37).astype(np.float32)
    yr = rng.standard_t(3, 100003).astype(np.float32)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    cbg.cbg_prior(ctx, to_dev(yb), yb.size, "binary", out)
    cbg.cbg_sync(ctx)
    assert out.item() == oracle.prior(yb, "binary")
    cbg.cbg_prior(ctx, to_dev(yr), yr.size, "real", out)
    cbg.cbg_sync(ctx)
    assert out.item() == pytest.approx(oracle.prior(yr, "real"), rel=1e-12)


def test_prior_rejects_non_binary_labels(ctx):
    import torch
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    cbg.cbg_prior(ctx, to_dev(np.array([0, 1, 0.5], np.float32)), 3, "binary", out)
    with pytest.raises(cbg.CbgError) as e:
        cbg.cbg_sync(ctx)
    assert e.value.status == cbg.CBG_EDATA


def _gpu_ts(ctx, cat, y, perm, prior, a, kind):
    import torch
    C, n = cat.shape
    ts = torch.empty((C, n), dtype=torch.float32, device="cuda")
    cnt = torch.empty((C, n), dtype=torch.int32, device="cuda")
    sb = torch.empty((C, n), dtype=torch.int32 if kind == "binary" else torch.float64, device="cuda")
    cbg.cbg_ordered_ts(ctx, to_dev(cat), to_dev(y), n, C, to_dev(perm), prior, a, kind, ts, cnt, sb)
    cbg.cbg_sync(ctx)
    return to_host(ts), to_host(cnt, np.uint32), (to_host(sb, np.uint32) if kind == "binary" else to_host(sb))


def _cats(n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([synth.zipf_ids(rng, 50, 1.1, n), synth.zipf_ids(rng, 5000, 1.1, n),
                     np.full(n, 77, np.uint32), (np.arange(n, dtype=np.uint32) * 2654435761).astype(np.uint32),
                     rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)])


@pytest.mark.parametrize("n", [1, 3, 2049, 20011])
@pytest.mark.parametrize("a", [1.0, 2.0, 0.5])
def test_ordered_ts_binary_bit_exact(ctx, n, a):
    rng = np.random.default_rng(n)
    cat = _cats(n, n)
    y = (rng.random(n) < 0.3).astype(np.float32)
    perm = oracle.make_permutation(3, n)
    P = oracle.prior(y, "binary")
    ts, cnt, sb = _gpu_ts(ctx, cat, y, perm, P, a, "binary")
    for c in range(cat.shape[0]):
        t_ref, c_ref, s_ref = oracle.ordered_ts(cat[c], y, perm, P, a)
        assert np.array_equal(ts[c].view(np.uint32), t_ref.view(np.uint32)), c
        assert np.array_equal(cnt[c], c_ref)
        assert np.array_equal(sb[c], s_ref.astype(np.uint32))


@pytest.mark.parametrize("n", [5, 4096, 30011])
def test_ordered_ts_real(ctx, n):
    rng = np.random.default_rng(n + 1)
    cat = _cats(n, n + 1)
    y = (rng.standard_t(3, n) * 3).astype(np.float32)
    perm = oracle.make_permutation(11, n)
    P = oracle.prior(y, "real")
    ts, cnt, sb = _gpu_ts(ctx, cat, y, perm, P, 1.0, "real")
    for c in range(cat.shape[0]):
        t_ref, c_ref, s_ref = oracle.ordered_ts(cat[c], y, perm, P, 1.0)
        _, _, abs_ref = oracle.ordered_ts(cat[c], np.abs(y), perm, 0.0, 1.0)
        assert np.array_equal(cnt[c], c_ref)
        assert np.all(np.abs(sb[c] - s_ref) <= 1e-12 * abs_ref + 1e-300)
        den = c_ref.astype(np.float64) + 1.0
        tol = 1e-12 * (abs_ref + abs(P)) / den + np.spacing(np.abs(t_ref).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(ts[c].astype(np.float64) - t_ref.astype(np.float64)) <= tol)


def _gpu_borders(ctx, x, B):
    import torch
    F, n = x.shape
    borders = torch.empty((F, B), dtype=torch.float32, device="cuda")
    nb = torch.empty(F, dtype=torch.int32, device="cuda")
    cbg.cbg_select_borders(ctx, to_dev(x), n, F, B, borders, nb)
    cbg.cbg_sync(ctx)
    return to_host(borders), to_host(nb)


def _columns(n, seed):
    rng = np.random.default_rng(seed)
    cols = [rng.normal(size=n), rng.lognormal(size=n), rng.integers(0, 5, n), np.full(n, -2.5),
            rng.choice([-0.0, 0.0, 1.0], n), np.round(rng.normal(size=n), 1), rng.random(n) * 1e-30,
            -rng.exponential(size=n)]
    return np.stack(cols).astype(np.float32)


@pytest.mark.parametrize("n,B", [(1, 4), (7, 254), (1000, 32), (10007, 254), (65537, 128)])
def test_borders_bit_exact(ctx, n, B):
    x = _columns(n, n)
    b, nb = _gpu_borders(ctx, x, B)
    b_ref, nb_ref = oracle.select_borders(x, B)
    assert np.array_equal(nb, nb_ref)
    for f in range(x.shape[0]):
        assert np.array_equal(b[f, :nb[f]].view(np.uint32), b_ref[f, :nb[f]].view(np.uint32)), f
        assert np.all(np.isinf(b[f, nb[f]:]))


def test_borders_reject_nonfinite(ctx):
    x = np.ones((2, 100), np.float32)
    x[1, 17] = np.nan
    _, _ = None, None
    import torch
    borders = torch.empty((2, 8), dtype=torch.float32, device="cuda")
    nb = torch.empty(2, dtype=torch.int32, device="cuda")
    cbg.cbg_select_borders(ctx, to_dev(x), 100, 2, 8, borders, nb)
    with pytest.raises(cbg.CbgError) as e:
        cbg.cbg_sync(ctx)
    assert e.value.status == cbg.CBG_EDATA


@pytest.mark.parametrize("n,F,B,f_off,F_pad", [(1, 3, 4, 0, 32), (999, 8, 254, 5, 32), (4099, 40, 32, 30, 96)])
def test_quantize_bit_exact(ctx, n, F, B, f_off, F_pad):
    import torch
    rng = np.random.default_rng(F)
    x = np.concatenate([_columns(n, F)] * (F // 8 + 1))[:F]
    x[0] = rng.normal(size=n)
    b_ref, nb_ref = oracle.select_borders(x, B)
    bins = torch.zeros(F_pad * n, dtype=torch.uint8, device="cuda")
    bins_t = torch.zeros((f_off + F, n), dtype=torch.uint8, device="cuda")
    cbg.cbg_quantize(ctx, to_dev(x), n, F, to_dev(b_ref), to_dev(nb_ref), B, bins, F_pad, f_off, bins_t)
    cbg.cbg_sync(ctx)
    want = oracle.quantize(x, b_ref, nb_ref, F_pad, f_offset=f_off)
    got = train.rowmajor_from_grouped(to_host(bins), n, F_pad)
    assert np.array_equal(got, want)
    assert np.array_equal(to_host(bins_t)[f_off:], want[:, f_off:f_off + F].T)


@pytest.mark.slow
def test_full_size_logloss_1m_preprocess(ctx):
    """The 1M x (100 floats + 10 categoricals) workload the benchmark times: TS of every
    categorical and every border bit-exact; bins on 4096 sampled rows bit-exact."""
    w = synth.logloss_1m()
    import torch
    x, cat, y = to_dev(w.x), to_dev(w.cat), to_dev(w.y)
    P = oracle.prior(w.y, "binary")
    prep = train.preprocess(ctx, x, cat, y, "binary", w.max_borders, a=w.a, seed=w.seed)
    assert prep.prior == P
    perm = oracle.make_permutation(w.seed, w.n)
    assert np.array_equal(to_host(prep.perm, np.uint32), perm)
    ts = to_host(prep.ts)
    ts_ref = np.stack([oracle.ordered_ts(w.cat[c], w.y, perm, P, w.a)[0] for c in range(w.n_cat)])
    assert np.array_equal(ts.view(np.uint32), ts_ref.view(np.uint32))
    cols = np.concatenate([w.x, ts_ref])
    b_ref, nb_ref = oracle.select_borders(cols, w.max_borders)
    assert np.array_equal(to_host(prep.n_borders), nb_ref)
    b = to_host(prep.borders)
    for f in range(cols.shape[0]):
        assert np.array_equal(b[f, :nb_ref[f]].view(np.uint32), b_ref[f, :nb_ref[f]].view(np.uint32))
    rows = np.sort(np.random.default_rng(0).choice(w.n, 4096, replace=False)).astype(np.int64)
    want = oracle.quantize(cols, b_ref, nb_ref, prep.F_pad, rows=rows)[rows]
    got = train.rowmajor_from_grouped(to_host(prep.bins), w.n, prep.F_pad)[rows]
    assert np.array_equal(got, want)
    bt = to_host(prep.bins_t)
    assert np.array_equal(bt[:, rows].T, want[:, :cols.shape[0]])
    del x, cat, y, prep
    torch.cuda.empty_cache()
