"""The arithmetic claims behind the tensor-core contractions, checked on the CPU with numpy float32
arithmetic (an emulation of the scheme as published by Ozaki, Ogita, Oishi and Rump with a fixed-point
grid per 128-node window; the CUDA kernels are not involved):

* the seven slices of a double-float value (itself within 2^-47 of the FP64 value) reconstruct it to
  2^-50 of the window's largest value, and
  every slice k 2^(-8 i) with |k| <= 129 is an exact bf16 number;
* every level sum over a 128-node window (at most four products per level for levels 0-3) is an integer
  multiple of 2^(-8 L) below 2^24 units, so an FP32 accumulator holds it exactly;
* the window's dot product assembled from the levels (0-3 exact, 4-6 in one rounded sum) matches the
  exact product sum to about 2^-46 of the largest term;
* with three slices (levels 0-2, six products, all exact) the window's dot product errs by less than
  2^-25 of (128 nodes x the largest term), observed up to 2^-27.5: the FP32 level of precision mode 3
  (each operand keeps 23 bits below its row's window maximum).
"""
import numpy as np

SLICES = 7
NODES = 128


def _f32(x):
    return np.float32(x)


def _slices(h, l, sh, n=SLICES):
    """The slicing rule: p + e is the remaining value; k = rint(p + e); p -= k; scale by 256."""
    p, e = np.ldexp(h, sh).astype(np.float32), np.ldexp(l, sh).astype(np.float32)
    out = []
    for i in range(n):
        k = np.rint((p + e).astype(np.float32)).astype(np.float32)
        p = (p - k).astype(np.float32)
        out.append(k)
        p = (p * _f32(256.0)).astype(np.float32)
        e = (e * _f32(256.0)).astype(np.float32)
    return out


def _window(rng):
    # magnitudes spread over 40 orders of two, random signs: the dynamic range of the node tables
    x = rng.standard_normal(NODES) * np.exp2(-rng.uniform(0.0, 40.0, NODES))
    h = x.astype(np.float32)
    l = (x - h.astype(np.float64)).astype(np.float32)
    E = np.frexp(np.abs(h).max())[1]
    return x, h, l, 7 - E


def _is_bf16(v):
    # a float32 value is a bf16 number when its low 16 bits are zero
    return np.all((np.asarray(v, dtype=np.float32).view(np.uint32) & 0xFFFF) == 0)


def test_slices_reconstruct_and_are_exact_bf16():
    rng = np.random.default_rng(7)
    for _ in range(50):
        x, h, l, sh = _window(rng)
        ks = _slices(h, l, sh)
        rec = sum(k.astype(np.float64) * 2.0 ** (-8 * i) for i, k in enumerate(ks)) * 2.0 ** (-sh)
        df = h.astype(np.float64) + l.astype(np.float64)       # the double-float value being sliced
        assert np.abs(rec - df).max() <= 2.0 ** -50 * np.abs(x).max()
        assert np.all(np.abs(df - x) <= 2.0 ** -47 * np.abs(x))   # hi + lo carries ~48 bits
        for i, k in enumerate(ks):
            assert np.abs(k).max() <= 129
            assert _is_bf16(k * _f32(2.0 ** (-8 * i)))


def test_level_sums_are_exact_in_fp32_and_the_window_product_is_accurate():
    rng = np.random.default_rng(11)
    for _ in range(50):
        xa, ha, la, sa = _window(rng)
        xb, hb, lb, sb = _window(rng)
        A = [k.astype(np.float64) * 2.0 ** (-8 * i) for i, k in enumerate(_slices(ha, la, sa))]
        Bs = [k.astype(np.float64) * 2.0 ** (-8 * j) for j, k in enumerate(_slices(hb, lb, sb))]
        levels = []
        for L in range(SLICES):
            s = sum(np.dot(A[i], Bs[L - i]) for i in range(L + 1))   # exact in float64 (few bits)
            levels.append(s)
            if L <= 3:
                units = s * 2.0 ** (8 * L)
                assert units == np.rint(units) and abs(units) < 2.0 ** 24
                assert float(np.float32(s)) == s                        # an FP32 accumulator holds it
        # the kernel's epilogue: exact parts, the tail rounded in FP32, the window scales applied
        tail = float(np.float32(levels[4] + levels[5] + levels[6]))
        value = (levels[0] + levels[1] + levels[2] + levels[3] + tail) * 2.0 ** (-sa - sb)
        exact = float(np.dot(xa, xb))
        scale = float(np.abs(xa).max() * np.abs(xb).max() * NODES)
        assert abs(value - exact) <= 2.0 ** -46 * scale


def test_three_slices_give_the_fp32_level():
    rng = np.random.default_rng(13)
    worst = 0.0
    for _ in range(50):
        xa, ha, la, sa = _window(rng)
        xb, hb, lb, sb = _window(rng)
        A = [k.astype(np.float64) * 2.0 ** (-8 * i) for i, k in enumerate(_slices(ha, la, sa, 3))]
        Bs = [k.astype(np.float64) * 2.0 ** (-8 * j) for j, k in enumerate(_slices(hb, lb, sb, 3))]
        levels = [sum(np.dot(A[i], Bs[L - i]) for i in range(L + 1)) for L in range(3)]
        for L, v in enumerate(levels):
            assert float(np.float32(v)) == v and abs(v * 2.0 ** (8 * L)) < 2.0 ** 24   # exact in FP32
        value = sum(levels) * 2.0 ** (-sa - sb)
        scale = float(np.abs(xa).max() * np.abs(xb).max() * NODES)
        err = abs(value - float(np.dot(xa, xb))) / scale
        assert err <= 2.0 ** -25
        worst = max(worst, err)
    # and no better than the truncation predicts: the dropped levels (i + j >= 3) are not accidentally kept
    assert worst > 2.0 ** -32
