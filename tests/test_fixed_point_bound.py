"""The rounding bound the GPU tests allow the opt-in fixed-point histogram kernel
(tiles.kernel 7), checked on the CPU against a numpy restatement of that kernel's
arithmetic. Per CTA:
- S = the FP32 sum of |v| over the CTA's rows;
- k: 1.001 S < 2^k, by frexp;
- e = 30 - k;
- each value becomes q = floor(v 2^e + u), u a dither in [0, 1).
The restatement checks three things:
- no int32 cell can overflow (sum of |q| < 2^31, even with every row in one cell);
- each row's error is below the per-row bound of tests/gpu_util.py;
- integer values with e >= 0 are exact.
This is test infrastructure only: it pins the bound's derivation, not the kernel."""
import numpy as np
import pytest

from gpu_util import fixed_point_row_error, fixed_point_slack


def _kernel_rounding(v, u):
    """One CTA's fixed-point values, as the kernel forms them (FP32 products and floors)."""
    v = np.asarray(v, np.float32)
    S = np.float32(np.sum(np.abs(v), dtype=np.float32))
    b = np.float32(S * np.float32(1.001))
    if not b > 0:
        e = 0
    else:
        _, k = np.frexp(b)
        e = int(np.clip(30 - k, -120, 120))
    x = v * np.float32(2.0 ** e)                      # exact: a power-of-two scale
    xi = np.floor(x)
    q = xi.astype(np.int64) + ((x - xi) + u.astype(np.float32) >= np.float32(1.0)).astype(np.int64)
    return q, e


@pytest.mark.parametrize("seed,rows,scale", [(0, 4096, 1.0), (1, 4096, 1e-3), (2, 2048, 50.0), (3, 1, 0.3),
                                             (4, 8192, 1e4), (5, 300, 1e-20)])
def test_fixed_point_rounding_stays_inside_the_bound(seed, rows, scale):
    rng = np.random.default_rng(seed)
    v = (rng.standard_normal(rows) * scale).astype(np.float32)
    u = (rng.integers(0, 1 << 24, rows) * 2.0 ** -24).astype(np.float32)
    q, e = _kernel_rounding(v, u)
    assert np.abs(q).sum() < 2 ** 31                  # every row in one cell still fits int32
    err = np.abs(q * 2.0 ** -e - v.astype(np.float64))
    assert np.all(err < fixed_point_row_error(v.astype(np.float64), rows_per_cta=rows))
    assert np.all(err < 2.0 ** -e)


def test_fixed_point_rounding_is_unbiased_where_round_to_nearest_is_not():
    """Many rows sharing one value (g after a few trees): the dithered sum stays within a
    few sqrt(m) units of the exact one, while rounding to nearest is off by m times one
    value's error."""
    m = 4096
    v = np.full(m, 0.123456789, np.float32)
    rng = np.random.default_rng(7)
    u = (rng.integers(0, 1 << 24, m) * 2.0 ** -24).astype(np.float32)
    q, e = _kernel_rounding(v, u)
    exact = float(v[0]) * m * 2.0 ** e
    assert abs(q.sum() - exact) < 4 * np.sqrt(m)
    nearest = np.rint(v.astype(np.float64) * 2.0 ** e).sum()
    assert abs(nearest - exact) > 0.05 * m           # the systematic error the dither removes


def test_integer_values_are_exact():
    rng = np.random.default_rng(3)
    v = rng.integers(-40, 41, 5000).astype(np.float32)
    u = (rng.integers(0, 1 << 24, 5000) * 2.0 ** -24).astype(np.float32)
    q, e = _kernel_rounding(v, u)
    assert e >= 0 and np.array_equal(q, v.astype(np.int64) << e)


def test_slack_scales_with_the_count_and_the_chain():
    g = np.array([0.5, -0.25, 1.0])
    h = np.array([0.25, 0.25, 0.125])
    count = np.array([[3.0, 3.0], [1.0, 1.0]])
    s1 = fixed_point_slack(count, g, h, chain=1)
    s2 = fixed_point_slack(count, g, h)
    assert np.allclose(s2, 2 * s1)
    assert np.allclose(s1[0], 3 * s1[1])
    assert s1[0, 0] == pytest.approx(3 * 2.002 * 1.75 * 2.0 ** -30)
