"""The arithmetic of the reduced-precision RK4 forms' right-hand side H y on the FP32 pipe, checked on the
CPU with numpy (an emulation; the CUDA kernels are not involved):

* an FP64 value split by its bits (24 truncated significant bits, then the next 23) is within 2^-46 of
  itself, both parts are float32 numbers, and the split keeps the sign and maps zero to zero;
* the compensated dot product of double-floats (TwoSum of the high products, residuals and TwoSum errors
  in a second float32 sum; Ogita, Rump and Oishi's Dot2) of a 380-term complex row of H with y is within
  n u^2 = 380 2^-48 (about 2^-39.4) of sum |H_ij| |y_j| of the exact sum (the float32 error sum's own
  rounding; observed near 2^-43), far below the 1e-6 bar of those forms.
"""
from fractions import Fraction

import numpy as np


def _split_bits(x):
    """hi: x truncated to 24 significant bits; lo: the next 23 mantissa bits (integer operations only)."""
    u = np.asarray(x, dtype=np.float64).view(np.uint64)
    h = (u >> np.uint64(32)).astype(np.uint32)
    l = (u & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    e = (h >> np.uint32(20)) & np.uint32(0x7FF)
    sg = h & np.uint32(0x80000000)
    ok = (e >= 897) & (e <= 1150)
    eb = np.where(ok, e, np.uint32(897))
    hb = sg | ((eb - np.uint32(896)) << np.uint32(23)) | ((h & np.uint32(0xFFFFF)) << np.uint32(3)) | (l >> np.uint32(29))
    hi = np.where(ok, hb.view(np.float32), np.float32(0.0))
    r = (l >> np.uint32(6)) & np.uint32(0x7FFFFF)
    rf = ((np.uint32(0x4B000000) | r).view(np.float32) - np.float32(8388608.0)).astype(np.float32)
    el = np.where(e >= 943, e, np.uint32(943))
    sc = ((el - np.uint32(942)) << np.uint32(23)).view(np.float32)
    lo = np.where(ok & (e >= 943), (rf * sc).astype(np.float32), np.float32(0.0))
    lo = (lo.view(np.uint32) | sg).view(np.float32)
    return hi.astype(np.float32), lo.astype(np.float32)


def test_split_bits_is_a_double_float():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(20000) * np.exp2(rng.uniform(-70, 60, 20000))
    hi, lo = _split_bits(x)
    err = np.abs(x - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -46 * np.abs(x))
    assert np.all(np.sign(hi) == np.sign(x)) and np.all((lo == 0) | (np.sign(lo) == np.sign(x)))
    assert np.all(np.abs(hi.astype(np.float64)) <= np.abs(x))          # truncation toward zero
    h0, l0 = _split_bits(np.array([0.0, -0.0, 1e-300]))
    assert np.all(h0 == 0) and np.all(l0 == 0)


def _two_sum(a, b):
    s = (a + b).astype(np.float32)
    bb = (s - a).astype(np.float32)
    return s, ((a - (s - bb).astype(np.float32)).astype(np.float32) + (b - bb).astype(np.float32)).astype(np.float32)


def _dot2_acc(s, c, ah, al, bh, bl):
    f64 = np.float64
    p = (ah * bh).astype(np.float32)
    e = (ah.astype(f64) * bh.astype(f64) - p.astype(f64)).astype(np.float32)      # fma(ah, bh, -p): exact
    e = (ah.astype(f64) * bl.astype(f64) + e.astype(f64)).astype(np.float32)
    e = (al.astype(f64) * bh.astype(f64) + e.astype(f64)).astype(np.float32)
    s, t = _two_sum(s, p)
    c = (c + (t + e).astype(np.float32)).astype(np.float32)
    return s, c


def test_compensated_complex_row_product():
    rng = np.random.default_rng(9)
    N = 380
    worst = 0.0
    for _ in range(20):
        # a row of H (magnitudes over ten orders, like energy phases times couplings) and an amplitude vector
        H = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * np.exp2(rng.uniform(-30, 3, N))
        y = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * np.exp2(rng.uniform(-40, 0, N))
        mrh, mrl = _split_bits(H.real)
        mih, mil = _split_bits(H.imag)
        yrh, yrl = _split_bits(y.real)
        yih, yil = _split_bits(y.imag)
        z = np.float32(0.0)
        sr, cr, si, ci = z, z, z, z
        for j in range(N):
            sr, cr = _dot2_acc(sr, cr, mrh[j:j + 1], mrl[j:j + 1], yrh[j:j + 1], yrl[j:j + 1])
            si, ci = _dot2_acc(si, ci, mrh[j:j + 1], mrl[j:j + 1], yih[j:j + 1], yil[j:j + 1])
            sr, cr = _dot2_acc(sr, cr, -mih[j:j + 1], -mil[j:j + 1], yih[j:j + 1], yil[j:j + 1])
            si, ci = _dot2_acc(si, ci, mih[j:j + 1], mil[j:j + 1], yrh[j:j + 1], yrl[j:j + 1])
        re = float(sr[0]) + float(cr[0])
        im = float(si[0]) + float(ci[0])
        ex_re = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(H.real, y.real)) - \
            sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(H.imag, y.imag))
        ex_im = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(H.real, y.imag)) + \
            sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(H.imag, y.real))
        scale = float(np.sum(np.abs(H) * np.abs(y)))
        err = max(abs(re - float(ex_re)), abs(im - float(ex_im))) / scale
        assert err <= N * 2.0 ** -48
        worst = max(worst, err)
    assert 0.0 < worst
