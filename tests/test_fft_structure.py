"""The component and regular-grid transforms' structure, restated in numpy
(CPU only): input in bit-reversed order, decimation-in-time stages taken in
pairs (radix 2^2: four elements i, i+h, i+2h, i+3h, the butterflies of stage
s with span 2h and of stage s+1 with span 4h) with an odd last stage as a
plain radix-2 pass, twiddles in a stage-major table (the butterflies of
span 2h read W_{2h}^p = exp(-2 pi i p / 2h), p < h, at entry h - 1 + p,
2^nmax - 1 entries); the inverse conjugates them.  Checked against
numpy.fft.  Also the pairing of two real field components in one inverse
transform."""
import numpy as np
import pytest


def bitrev(t, logn):
    return int(format(t, f"0{logn}b")[::-1], 2) if logn else 0


def stage_twiddles(log_nmax):
    """Entry h - 1 + p holds exp(-2 pi i p / (2h)) for h = 1, 2, ..., 2^(nmax-1), p < h."""
    tw = np.empty((1 << log_nmax) - 1, dtype=complex)
    h = 1
    while h < (1 << log_nmax):
        tw[h - 1:2 * h - 1] = np.exp(-1j * np.pi * np.arange(h) / h)
        h *= 2
    return tw


def test_stage_twiddles_table():
    tw = stage_twiddles(4)
    assert tw.size == 15 and tw[0] == 1
    # span 16 (h = 8): the 16th roots of unity, p < 8; span 4: 1, -i
    np.testing.assert_allclose(tw[7:15], np.exp(-2j * np.pi * np.arange(8) / 16), atol=1e-15)
    np.testing.assert_allclose(tw[1:3], [1, -1j], atol=1e-15)


def fft_pairs(x, logn, log_nmax, inverse=False):
    n = 1 << logn
    tw = stage_twiddles(log_nmax)
    if inverse:
        tw = np.conj(tw)
    buf = np.empty(n, dtype=complex)
    for t in range(n):
        buf[bitrev(t, logn)] = x[t]
    s0 = 1
    while s0 + 1 <= logn:
        h = 1 << (s0 - 1)
        for jj in range(n >> 2):
            pos = jj & (h - 1)
            grp = jj >> (s0 - 1)
            i0 = grp * 4 * h + pos
            w1, w2, w3 = tw[h - 1 + pos], tw[2 * h - 1 + pos], tw[2 * h - 1 + pos + h]
            a0, a1, a2, a3 = buf[i0], buf[i0 + h], buf[i0 + 2 * h], buf[i0 + 3 * h]
            m1, m3 = a1 * w1, a3 * w1
            b0, b1, b2, b3 = a0 + m1, a0 - m1, a2 + m3, a2 - m3
            n2, n3 = b2 * w2, b3 * w3
            buf[i0], buf[i0 + 2 * h] = b0 + n2, b0 - n2
            buf[i0 + h], buf[i0 + 3 * h] = b1 + n3, b1 - n3
        s0 += 2
    for s in range(s0, logn + 1):
        half = 1 << (s - 1)
        for jj in range(n >> 1):
            pos = jj & (half - 1)
            grp = jj >> (s - 1)
            i0 = grp * 2 * half + pos
            w = tw[half - 1 + pos]
            a, b = buf[i0], buf[i0 + half] * w
            buf[i0], buf[i0 + half] = a + b, a - b
    return buf


@pytest.mark.parametrize("logn,log_nmax", [(1, 1), (2, 4), (3, 3), (5, 7), (6, 6), (7, 10)])
def test_radix4_pairs_equal_numpy(logn, log_nmax):
    rng = np.random.default_rng(logn + 10 * log_nmax)
    x = rng.standard_normal(1 << logn) + 1j * rng.standard_normal(1 << logn)
    np.testing.assert_allclose(fft_pairs(x, logn, log_nmax), np.fft.fft(x), rtol=0, atol=1e-11)
    np.testing.assert_allclose(fft_pairs(x, logn, log_nmax, inverse=True), np.fft.ifft(x) * x.size, rtol=0,
                               atol=1e-11)


def test_two_real_components_share_one_inverse():
    """F^-1(E^_a + i E^_b) has E_a as its real and E_b as its imaginary part
    when both spectra are those of real fields, Nyquist planes zeroed."""
    rng = np.random.default_rng(5)
    rho = rng.standard_normal((16, 32))
    rh = np.fft.fft2(rho)
    kx = 2 * np.pi * np.fft.fftfreq(16, d=1 / 16)
    ky = 2 * np.pi * np.fft.fftfreq(32, d=1 / 32)
    KX, KY = np.meshgrid(kx, ky, indexing="ij")
    k2 = KX ** 2 + KY ** 2
    phi = np.where(k2 > 0, rh / np.where(k2 > 0, k2, 1), 0)
    KXn = np.where(np.arange(16)[:, None] == 8, 0.0, KX)
    KYn = np.where(np.arange(32)[None, :] == 16, 0.0, KY)
    Ea, Eb = -1j * KXn * phi, -1j * KYn * phi
    both = np.fft.ifft2(Ea + 1j * Eb)
    np.testing.assert_allclose(both.real, np.real(np.fft.ifft2(Ea)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(both.imag, np.real(np.fft.ifft2(Eb)), rtol=0, atol=1e-12)
    assert np.max(np.abs(np.imag(np.fft.ifft2(Ea)))) < 1e-12  # each alone is real


def _bitrev(t, logn):
    r = 0
    for b in range(logn):
        r |= ((t >> b) & 1) << (logn - 1 - b)
    return r


def inplace_axis_fft(buf, logs, ax, inverse, log_nmax):
    """The one-block solve's in-place transform of a flat grid (x fastest)
    along axis ax, restated: bit-reversal swap along the axis, then radix-2
    stages whose butterfly j takes inner index j mod 2^ls (the axes below
    ax), butterfly p = (j >> ls) mod 2^(logn-1) of its line and outer line
    o = j >> (ls + logn - 1); twiddle entry half - 1 + pos of the stage-major
    table (conjugated for the inverse)."""
    S = buf.size
    logn = logs[ax]
    ls = sum(logs[:ax])
    length = 1 << logn
    for e in range(S):
        t = (e >> ls) & (length - 1)
        r = _bitrev(t, logn)
        if r > t:
            e2 = e + ((r - t) << ls)
            buf[e], buf[e2] = buf[e2], buf[e]
    tw = stage_twiddles(log_nmax)
    half_n = length >> 1
    for s in range(1, logn + 1):
        half = 1 << (s - 1)
        for j in range(S >> 1):
            i = j & ((1 << ls) - 1)
            p = (j >> ls) & (half_n - 1) if half_n > 0 else 0
            o = j >> (ls + logn - 1)
            pos = p & (half - 1)
            grp = p >> (s - 1)
            t0 = grp * 2 * half + pos
            i0 = (((o << logn) + t0) << ls) + i
            i1 = i0 + (half << ls)
            w = tw[half - 1 + pos]
            if inverse:
                w = np.conj(w)
            x0, x1 = buf[i0], buf[i1] * w
            buf[i0], buf[i1] = x0 + x1, x0 - x1


@pytest.mark.parametrize("logs", [(3, 2), (1, 4), (2, 1, 3), (4, 1, 1)])
def test_one_block_axis_mapping_equals_numpy_fft(logs):
    rng = np.random.default_rng(sum(logs))
    shape = tuple(1 << l for l in reversed(logs))  # numpy order [.., i_2, i_1] for an x-fastest flat array
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    for inverse in (False, True):
        buf = x.ravel().copy()
        for ax in range(len(logs)):
            inplace_axis_fft(buf, list(logs), ax, inverse, max(logs))
        ref = np.fft.fftn(x) if not inverse else np.fft.ifftn(x) * x.size
        np.testing.assert_allclose(buf.reshape(shape), ref, atol=1e-9)
