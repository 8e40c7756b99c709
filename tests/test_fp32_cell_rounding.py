"""The FP32 cell finding of the deposit and the gather, restated in numpy
float32 (the kernels' arithmetic, CPU only): t = (s - 1/2) + 1.5 2^23 rounds
s - 1/2 to the nearest integer, its low mantissa bits give the cell c and
t - 1.5 2^23 its floor fl, and f = s - fl.  For every scaled position s in
[-1/2, 2^n) (the cell-centred shift reaches -1/2) the CIC weights (1 - f on
node c, f on node c + 1, periodically) must equal those of the exact floor,
including the ties at exact integers, where the rounding may pick the node
below with f = 1, up to the 2^-24 of the one case described below."""
import numpy as np
import pytest

MAGIC = np.float32(12582912.0)  # 1.5 * 2^23


def cell_frac_fp32(s, n):
    s = s.astype(np.float32)
    t = (s - np.float32(0.5)) + MAGIC
    fl = t - MAGIC
    c = (t.view(np.int32) - np.int32(0x4B400000)) & np.int32((1 << n) - 1)
    f = s - fl
    return c.astype(np.int64), f.astype(np.float64), fl


def weights(c, f, N):
    """Dense per-node weights of each position (two nodes each)."""
    w = np.zeros((c.size, N))
    rows = np.arange(c.size)
    np.add.at(w, (rows, c % N), 1.0 - f)
    np.add.at(w, (rows, (c + 1) % N), f)
    return w


@pytest.mark.parametrize("n", [2, 5, 10])
@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_fp32_cell_frac_gives_exact_cic_weights(n, shift):
    N = 1 << n
    rng = np.random.default_rng(n)
    u = rng.random(20000).astype(np.float32)
    # exact node positions (ties), their neighbouring floats, the box edges
    k = np.arange(N, dtype=np.float32)
    special = np.concatenate([(k + shift) / N, np.nextafter((k + shift) / N, np.float32(0)),
                              np.nextafter((k + shift) / N, np.float32(1)),
                              np.array([0.0, np.nextafter(np.float32(1), np.float32(0))], dtype=np.float32)])
    u = np.concatenate([u, special[(special >= 0) & (special < 1)].astype(np.float32)])
    s = u * np.float32(N) - np.float32(shift)  # exact: power-of-two scale, shift exact near 0 and N
    c, f, fl = cell_frac_fp32(s, n)
    assert np.all(f <= 1.0)
    # a tiny negative s (|s| < 2^-24, only with the cell-centred shift, just
    # below the first centre) makes s - 1/2 round to -1/2 and the sum to 0:
    # f = s, negative by at most 2^-24, on the node pair (0, 1) instead of
    # (N-1, 0); the weights then differ from the exact ones by |s|
    neg = f < 0
    assert np.all(s[neg] < 0) and np.all(-f[neg] <= 2.0 ** -24)
    s64 = s.astype(np.float64)
    ref_c = np.floor(s64).astype(np.int64)
    ref_f = s64 - np.floor(s64)
    np.testing.assert_allclose(weights(c, f, N), weights(ref_c, ref_f, N), rtol=0, atol=1e-6)
    # off the ties (and off the tiny-negative case) the cell is the floor itself
    off = (ref_f > 0) & ~neg
    assert np.array_equal(c[off] % N, ref_c[off] % N)


def test_fixed_point_quantisation_is_round_to_nearest_even():
    """The deposit window's FP32 fixed point: bits(fma(a, b, 1.5 2^23)) -
    bits(1.5 2^23) is the integer nearest a*b (ties to even) for |a*b| < 2^22,
    since the sum lands in [2^23, 2^24) where floats are spaced by 1.  fma
    rounds once: emulated as one rounding of the exact double a*b + 1.5 2^23."""
    rng = np.random.default_rng(3)
    a = (rng.standard_normal(200000) * 3e4).astype(np.float32)
    b = rng.random(200000).astype(np.float32)
    ties = np.array([0.5, 1.5, 2.5, -0.5, -1.5, -2.5, 2.0 ** 21 + 0.5, -(2.0 ** 21) - 0.5], dtype=np.float32)
    a = np.concatenate([a, ties])
    b = np.concatenate([b, np.ones(ties.size, dtype=np.float32)])
    exact = a.astype(np.float64) * b.astype(np.float64)
    assert np.all(np.abs(exact) < 2.0 ** 22)
    t = (exact + 12582912.0).astype(np.float32)  # the single rounding of fmaf
    q = t.view(np.int32).astype(np.int64) - 0x4B400000
    np.testing.assert_array_equal(q, np.rint(exact).astype(np.int64))  # rint: ties to even
