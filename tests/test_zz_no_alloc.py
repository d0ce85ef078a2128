"""The allocation-free root histogram (cbg_histogram_noalloc) against the regular level
builder (cbg_build_level at depth 0, which needs a caller-allocated tree state).

cbg_histogram_noalloc serves callers that cannot allocate device memory (an application
that owns the whole device memory budget, or plugin code that may not call cudaMalloc):
its scratch is a fixed device array inside the library. Two calls in a row must both
agree with the regular path, and with the FP64 oracle directly, within the histogram
tolerance of the other tests: 1e-5 of the per-bin sum of |g| (|h|). Two shapes fill the
scratch, so that each CTA sums more rows than the regular tiling gives it. This file is
collected last on purpose."""
import numpy as np
import pytest

import oracle
from gpu_util import hist_tolerance_ok, to_dev, to_host
from paper_1810_11363_gb300 import cbg, synth, train

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = cbg.Context(0)
    yield c
    c.close()


def _regular_root_hist(ctx, bins_rm, nb, g, h, dtype):
    """Depth-0 histogram through cbg_build_level (the existing entry point)."""
    import torch
    n, F_pad = bins_rm.shape
    F = nb.shape[0]
    max_bins = int(nb.max()) + 1
    shape = cbg.make_shape(n, F, F_pad, max_bins, 1)
    state = torch.empty(cbg.cbg_tree_state_bytes(shape), dtype=torch.uint8, device="cuda")
    leaf = torch.empty(n, dtype=torch.int16, device="cuda")
    splits = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    child = torch.empty((2, 2), dtype=torch.float64, device="cuda")
    hist = torch.empty((1, F, max_bins, 2), dtype=torch.float64, device="cuda")
    bins = to_dev(train.grouped_from_rowmajor(bins_rm))
    cbg.cbg_tree_begin(ctx, shape, state, leaf)
    cbg.cbg_build_level(ctx, shape, state, bins, to_dev(nb.astype(np.int32)), g, h, dtype, 0, 3.0, leaf, splits,
                        child, hist_out=hist, last_level=True)
    cbg.cbg_sync(ctx)
    return bins, to_host(hist)[0]


@pytest.mark.parametrize("n,F,F_pad,max_bins,dtype", [(200003, 70, 96, 255, "f32"), (4097, 33, 64, 129, "bf16"),
                                                       (1, 3, 32, 5, "f32"),
                                                       # the scratch's unit count binds: ~7k rows per CTA
                                                       (400000, 2000, 2048, 129, "f32"),
                                                       # ~4.4k rows per CTA, 255 bins
                                                       (3000007, 90, 96, 255, "bf16")])
def test_noalloc_root_histogram_matches_build_level_twice(ctx, n, F, F_pad, max_bins, dtype):
    import torch
    bins_rm, nb, g, h, _ = synth.random_level_case(n + F, n, F, F_pad, max_bins, 1)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    gd = torch.from_numpy(g).to(tdt).cuda()
    hd = torch.from_numpy(h).to(tdt).cuda()
    bins, ref = _regular_root_hist(ctx, bins_rm, nb, gd, hd, dtype)
    g64, h64 = gd.double().cpu().numpy(), hd.double().cpu().numpy()
    bound = oracle.histogram(bins_rm, F, np.abs(g64), np.abs(h64), None, 1, ref.shape[1])[0]
    exact = oracle.histogram(bins_rm, F, g64, h64, None, 1, ref.shape[1])[0]
    mb = int(nb.max()) + 1
    for _ in range(2):
        out = torch.full((F, mb, 2), float("nan"), dtype=torch.float64, device="cuda")
        cbg.cbg_histogram_noalloc(ctx, bins, n, F, F_pad, mb, gd, hd, dtype, out)
        cbg.cbg_sync(ctx)
        got = to_host(out)
        assert not np.isnan(got).any()
        assert hist_tolerance_ok(got, ref, bound), np.abs(got - ref).max()
        assert hist_tolerance_ok(got, exact, bound), np.max(np.abs(got - exact) / np.maximum(bound, 1e-300))


def test_noalloc_rejects_what_does_not_fit_its_scratch(ctx):
    import torch
    F_pad = 32 * 300                  # 300 groups x 255 bins of partials exceed the 16 MiB scratch
    n = 8
    bins = torch.zeros(F_pad * n, dtype=torch.uint8, device="cuda")
    g = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.empty((F_pad, 255, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(cbg.CbgError) as e:
        cbg.cbg_histogram_noalloc(ctx, bins, n, F_pad, F_pad, 255, g, g, "f32", out)
    assert e.value.status == cbg.CBG_EINVAL


def test_noalloc_rejects_more_rows_per_cta_than_its_bound(ctx):
    """F_pad 2048 at 128 bins leaves room for 7 work units: 10^6 rows would put more
    than 16384 rows into one CTA's FP32 histogram, which the call refuses."""
    import torch
    n, F_pad = 1_000_000, 2048
    bins = torch.zeros(F_pad * n, dtype=torch.uint8, device="cuda")
    g = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.empty((F_pad, 129, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(cbg.CbgError) as e:
        cbg.cbg_histogram_noalloc(ctx, bins, n, F_pad, F_pad, 129, g, g, "f32", out)
    assert e.value.status == cbg.CBG_EINVAL
    assert "rows" in str(e.value)
