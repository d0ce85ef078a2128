"""Pins of the oracle's border selection, quantisation and gradients."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("n,B", [(1000, 32), (1000, 254), (4097, 128), (10, 254), (255, 254)])
def test_borders_closed_form_on_distinct_values(n, B):
    # Values 0..n-1 (shuffled): the sorted column at index i is i, so candidate k is
    # floor(k*n/(B+1)); keep strictly increasing values below the maximum n-1.
    rng = np.random.default_rng(n + B)
    x = rng.permutation(n).astype(np.float32)
    borders, nb = oracle.select_borders(x, B)
    want = []
    for k in range(1, B + 1):
        c = (k * n) // (B + 1)
        if c < n - 1 and (not want or c > want[-1]):
            want.append(c)
    assert nb[0] == len(want)
    assert borders[0, :nb[0]].tolist() == [float(v) for v in want]


def test_constant_column_has_no_border():
    borders, nb = oracle.select_borders(np.full(100, 3.5, np.float32), 254)
    assert nb[0] == 0


def test_two_valued_column_has_one_border():
    x = np.array([1.0] * 50 + [2.0] * 50, np.float32)
    borders, nb = oracle.select_borders(x, 254)
    assert nb[0] == 1 and borders[0, 0] == 1.0


def test_nonfinite_is_rejected():
    with pytest.raises(ValueError):
        oracle.select_borders(np.array([1.0, np.nan, 2.0], np.float32), 4)


def test_negative_zero_border_is_canonical():
    x = np.array([-0.0] * 10 + [1.0] * 10, np.float32)
    borders, nb = oracle.select_borders(x, 4)
    assert nb[0] == 1
    assert np.signbit(borders[0, 0]) == False  # noqa: E712


@pytest.mark.parametrize("B", [32, 128, 254])
def test_quantile_invariant_counts_per_bin(B):
    # Distinct values: every bin holds n/(B+1) rows up to +-1.
    n = 20000
    rng = np.random.default_rng(B)
    x = rng.normal(size=n).astype(np.float32)
    x = np.unique(x)
    n = x.shape[0]
    x = rng.permutation(x)
    borders, nb = oracle.select_borders(x, B)
    assert nb[0] == B
    bins = oracle.quantize(x[None, :], borders, nb, 16)
    counts = np.bincount(bins[:, 0], minlength=B + 1)
    assert counts.sum() == n
    assert np.all(np.abs(counts - n / (B + 1)) <= 1.0 + 1e-9)


def test_quantize_matches_searchsorted_and_is_monotone():
    rng = np.random.default_rng(1)
    F, n, B = 5, 3000, 31
    x = np.concatenate([rng.normal(size=(3, n)), rng.lognormal(size=(1, n)),
                        rng.integers(0, 4, size=(1, n))]).astype(np.float32)
    borders, nb = oracle.select_borders(x, B)
    bins = oracle.quantize(x, borders, nb, 16, f_offset=3)
    assert np.all(bins[:, :3] == 0) and np.all(bins[:, 3 + F:] == 0)
    for f in range(F):
        want = np.searchsorted(borders[f, :nb[f]], x[f], side="left")
        assert np.array_equal(bins[:, 3 + f], want)
        order = np.argsort(x[f], kind="stable")
        assert np.all(np.diff(bins[order, 3 + f].astype(np.int64)) >= 0)
        assert bins[:, 3 + f].max() <= nb[f]


def test_quantize_row_sampling_matches_full():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 500)).astype(np.float32)
    borders, nb = oracle.select_borders(x, 16)
    full = oracle.quantize(x, borders, nb, 16)
    rows = np.array([0, 7, 499, 250], np.int64)
    part = oracle.quantize(x, borders, nb, 16, rows=rows)
    assert np.array_equal(part[rows], full[rows])


def test_gradients_at_zero_prediction():
    y = np.array([0, 1, 1, 0], np.float32)
    g, h = oracle.gradients("logloss", y, np.zeros(4))
    assert g.tolist() == [0.5, -0.5, -0.5, 0.5]
    assert h.tolist() == [0.25] * 4
    yr = np.array([1.5, -2.25, 0.0], np.float32)
    g, h = oracle.gradients("rmse", yr, np.array([0.5, 0.5, -1.0]))
    assert g.tolist() == [-1.0, 2.75, -1.0]
    assert h.tolist() == [1.0] * 3


def test_logloss_gradient_is_derivative_of_loss():
    # g = dLoss/dpred, h = d2Loss/dpred2 (Section 3), by central differences.
    y = np.array([0.0, 1.0, 1.0, 0.0], np.float32)
    pred = np.array([-1.3, 0.2, 2.5, 0.7])
    g, h = oracle.gradients("logloss", y, pred)
    eps = 1e-5
    for i in range(4):
        def L(p):
            pp = pred.copy()
            pp[i] = p
            return oracle.loss("logloss", y[i:i + 1], pp[i:i + 1])
        num_g = (L(pred[i] + eps) - L(pred[i] - eps)) / (2 * eps)
        num_h = (L(pred[i] + eps) - 2 * L(pred[i]) + L(pred[i] - eps)) / eps**2
        assert g[i] == pytest.approx(num_g, rel=1e-5)
        assert h[i] == pytest.approx(num_h, rel=1e-3)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(size=2000), rng.normal(size=200) * 1e-30,
                        [1.00390625, 1.01171875, -1.00390625, 3.0e38]]).astype(np.float32)
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.round_bf16(float(x)) for x in v], np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_bf16_storage_rounds_gradients():
    y = np.array([0.0, 1.0], np.float32)
    pred = np.array([0.3, -0.7])
    g32, h32 = oracle.gradients("logloss", y, pred, "f32")
    g16, h16 = oracle.gradients("logloss", y, pred, "bf16")
    for a, b in ((g32, g16), (h32, h16)):
        assert np.all([oracle.round_bf16(float(v)) == w for v, w in zip(a, b)])
        assert np.all(np.abs(a - b) <= np.abs(a) * 2.0**-8)


def test_loss_values():
    y = np.array([1.0, 3.0], np.float32)
    assert oracle.loss("rmse", y, np.array([0.0, 0.0])) == pytest.approx(np.sqrt(5.0))
    yb = np.array([1.0, 0.0], np.float32)
    assert oracle.loss("logloss", yb, np.zeros(2)) == pytest.approx(np.log(2.0))
