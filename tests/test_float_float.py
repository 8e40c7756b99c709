"""The FP32 path's float-float accumulation (the combination's CAcc and the
push's kinetic-energy sums), restated in numpy float32 (CPU only):
two_sum is error-free, a + b = s + e exactly, and the un-renormalised
accumulator (hi by two_sum, the errors summed into lo) keeps an
alternating-sign sum like the combination's to ~2^-44 of its largest
partial sum."""
import numpy as np

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    err = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, err


def test_two_sum_is_error_free():
    rng = np.random.default_rng(1)
    a = (rng.standard_normal(100000) * 10.0 ** rng.integers(-6, 6, 100000)).astype(np.float32)
    b = (rng.standard_normal(100000) * 10.0 ** rng.integers(-6, 6, 100000)).astype(np.float32)
    s, e = two_sum(a, b)
    np.testing.assert_array_equal(a.astype(np.float64) + b.astype(np.float64),
                                  s.astype(np.float64) + e.astype(np.float64))


def test_accumulation_keeps_cancelling_sums():
    """Terms of alternating sign (+1, -1 coefficients of nearly equal
    component fields) added one by one as the combination does: the float-float
    result stays within 2^-40 of the exact sum, where plain float32 loses
    everything below its largest partial sum's 2^-24."""
    rng = np.random.default_rng(2)
    worst_ff, worst_f = 0.0, 0.0
    for _ in range(200):
        base = rng.standard_normal(20).astype(np.float32) * f32(1e3)
        terms = []
        for x in base:
            terms.append(x)
            terms.append(f32(-x + f32(rng.standard_normal() * 1e-3)))
        terms = np.array(terms, dtype=np.float32)
        hi, lo = f32(0.0), f32(0.0)
        plain = f32(0.0)
        for t in terms:
            hi, e = two_sum(hi, t)
            lo = f32(lo + e)
            plain = f32(plain + t)
        hi, lo = two_sum(hi, lo)
        exact = float(np.sum(terms.astype(np.float64)))
        scale = float(np.max(np.abs(np.cumsum(terms.astype(np.float64)))))
        worst_ff = max(worst_ff, abs(float(hi) + float(lo) - exact) / scale)
        worst_f = max(worst_f, abs(float(plain) - exact) / scale)
    assert worst_ff < 2.0 ** -40
    assert worst_f > 2.0 ** -30  # the plain float sum is visibly worse
