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
* the kernel's epilogue fold over the 18 windows of a 2304-node rule (L0 + rint(L1) and
  frac(L1) + L2 exact in FP32, L3 + tail rounded, the window terms folded into a double-float running sum
  by two TwoSums) ends within 2^-42 of the largest term of the exact sum (observed 2^-43.8 to 2^-48);
* with three slices (levels 0-2, six products, all exact) the window's dot product errs by less than
  2^-25 of (128 nodes x the largest term), observed up to 2^-27.5: the FP32 level (each operand keeps
  23 bits below its row's window maximum);
* with four slices (levels 0-3, ten products, all exact: precision mode 3) by less than 2^-31;
* the four-slice generated operand sliced by grid rounding (from the unnormalised product pair) and the
  drain's fold with frac(L1) + L2 + L3 rounded once keep that level over a 2304-node rule;
* the wide MMAs A_i [B_0 .. B_{3-i}] written at accumulator column 48 i land every product on its level,
  and the four-slice producer's stores fill the 64-byte-swizzled K-major generated tile exactly once.
"""
from fractions import Fraction

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


def test_four_slices_give_the_reduced_precision_level():
    # precision mode 3: four slices, levels 0-3 (ten products), every level exact in FP32; the dropped
    # levels (i + j >= 4) leave about 2^-32 of (128 nodes x the largest term)
    rng = np.random.default_rng(17)
    worst = 0.0
    for _ in range(50):
        xa, ha, la, sa = _window(rng)
        xb, hb, lb, sb = _window(rng)
        A = [k.astype(np.float64) * 2.0 ** (-8 * i) for i, k in enumerate(_slices(ha, la, sa, 4))]
        Bs = [k.astype(np.float64) * 2.0 ** (-8 * j) for j, k in enumerate(_slices(hb, lb, sb, 4))]
        levels = [sum(np.dot(A[i], Bs[L - i]) for i in range(L + 1)) for L in range(4)]
        for L, v in enumerate(levels):
            assert float(np.float32(v)) == v and abs(v * 2.0 ** (8 * L)) < 2.0 ** 24   # exact in FP32
        # the kernel's epilogue terms: L0 + rint(L1) and frac(L1) + L2 exact in FP32, L3 as it is
        l1h = np.rint(levels[1])
        xa_, xb_ = levels[0] + l1h, (levels[1] - l1h) + levels[2]
        assert float(np.float32(xa_)) == xa_ and float(np.float32(xb_)) == xb_
        value = (xa_ + xb_ + levels[3]) * 2.0 ** (-sa - sb)
        scale = float(np.abs(xa).max() * np.abs(xb).max() * NODES)
        err = abs(value - float(np.dot(xa, xb))) / scale
        assert err <= 2.0 ** -31
        worst = max(worst, err)
    assert worst > 2.0 ** -40


def _two_sum(a, b):
    s = np.float32(a + b)
    bb = np.float32(s - a)
    return s, np.float32(np.float32(a - np.float32(s - bb)) + np.float32(b - bb))


def test_epilogue_fold_over_many_windows():
    f32 = np.float32
    for seed in range(6):
        rng = np.random.default_rng(100 + seed)
        hi, lo = f32(0.0), f32(0.0)
        xs, ys = [], []
        for _ in range(2304 // NODES):
            xa, ha, la, sa = _window(rng)
            xb, hb, lb, sb = _window(rng)
            xs.append(xa)
            ys.append(xb)
            A = [k.astype(np.float64) * 2.0 ** (-8 * i) for i, k in enumerate(_slices(ha, la, sa))]
            Bs = [k.astype(np.float64) * 2.0 ** (-8 * j) for j, k in enumerate(_slices(hb, lb, sb))]
            L0, L1, L2, L3 = (f32(sum(np.dot(A[i], Bs[L - i]) for i in range(L + 1))) for L in range(4))
            tail = f32(0.0)                       # levels 4-6: one FP32 accumulator, product by product
            for L in range(4, SLICES):
                for i in range(L - SLICES + 1 if L >= SLICES else 0, min(L, SLICES - 1) + 1):
                    tail = f32(tail + f32(np.dot(A[i], Bs[L - i])))
            sc = f32(2.0 ** (-sa - sb))
            l1h = f32(np.rint(L1))
            xa_ = f32(L0 + l1h)
            fr = f32(L1 - l1h)
            xb_ = f32(fr + L2)
            assert float(xa_) == float(L0) + float(l1h) and float(xb_) == float(fr) + float(L2)
            xc = f32(L3 + tail)
            hi, r1 = _two_sum(hi, f32(xa_ * sc))
            hi, r2 = _two_sum(hi, f32(xb_ * sc))
            lo = f32(lo + f32(f32(r1 + r2) + f32(xc * sc)))
        a, b = np.concatenate(xs), np.concatenate(ys)
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
        err = abs(float(Fraction(float(hi)) + Fraction(float(lo)) - exact))
        assert err <= 2.0 ** -42 * float(np.abs(a).max() * np.abs(b).max()), seed


def _df(x):
    h = x.astype(np.float32)
    return h, (x - h.astype(np.float64)).astype(np.float32)


def _mul_pe(ah, al, bh, bl):
    """The generated operand's product as an unnormalised pair (p, e): p = fl(ah bh), e = the FMA residual
    plus the cross terms, each FMA rounded once (float64 holds every intermediate exactly here)."""
    f64 = np.float64
    p = (ah * bh).astype(np.float32)
    e = (ah.astype(f64) * bh.astype(f64) - p.astype(f64)).astype(np.float32)
    e = (ah.astype(f64) * bl.astype(f64) + e.astype(f64)).astype(np.float32)
    e = (al.astype(f64) * bh.astype(f64) + e.astype(f64)).astype(np.float32)
    return p, e


def _slices4_pe(p, e, sh):
    """Four slices by rounding to each grid with the constants 1.5 2^23 u (u = 1, 2^-8, 2^-16, 2^-24)."""
    f32, f64 = np.float32, np.float64
    s = f32(2.0 ** sh)
    C = [f32(1.5 * 2.0 ** 23), f32(1.5 * 2.0 ** 15), f32(1.5 * 2.0 ** 7), f32(0.75)]
    ps = (p.astype(f64) * f64(s))                       # exact: a power-of-two scaling
    t0 = (ps + f64(C[0])).astype(f32) - C[0]            # fma(p, s, C0) - C0
    r0 = (ps - t0.astype(f64)).astype(f32)              # fma(p, s, -t0), exact
    t1 = ((r0 + C[1]).astype(f32) - C[1]).astype(f32)
    r1 = (r0 - t1).astype(f32)
    s1 = (e.astype(f64) * f64(s) + r1.astype(f64)).astype(f32)   # fma(e, s, r1)
    t2 = ((s1 + C[2]).astype(f32) - C[2]).astype(f32)
    r2 = (s1 - t2).astype(f32)
    t3 = ((r2 + C[3]).astype(f32) - C[3]).astype(f32)
    return [t0.astype(f32), t1, t2, t3]


def _gen_window(rng):
    # a generated row: W (one node weight) times A_P (one projectile state), each a double-float
    w = rng.standard_normal(NODES) * np.exp2(-rng.uniform(0.0, 20.0, NODES))
    a = rng.standard_normal(NODES) * np.exp2(-rng.uniform(0.0, 20.0, NODES))
    wh, wl = _df(w)
    ah, al = _df(a)
    p, e = _mul_pe(wh, wl, ah, al)
    E = np.frexp(np.abs(p).max())[1]
    return w * a, p, e, min(7 - E, 127)


def test_generated_operand_slices_by_grid_rounding():
    # the four-slice generated operand: p + e reconstructed to 2^-25 + 2^-33 of the window's scaled grid,
    # every slice k 2^(-8 i) with |k| <= 130, an exact bf16 number
    rng = np.random.default_rng(23)
    for _ in range(100):
        x, p, e, sh = _gen_window(rng)
        assert np.all(np.abs(e.astype(np.float64)) <= 3.0 * 2.0 ** -24 * np.abs(p.astype(np.float64)) * (1 + 2.0 ** -20))
        ts = _slices4_pe(p, e, sh)
        pe = (p.astype(np.float64) + e.astype(np.float64)) * 2.0 ** sh
        rec = sum(t.astype(np.float64) for t in ts)
        assert np.abs(rec - pe).max() <= 2.0 ** -25 + 2.0 ** -33
        assert np.all(np.abs(x * 2.0 ** sh - pe) <= 2.0 ** -44 * np.abs(x * 2.0 ** sh) + 2.0 ** -140)
        for i, t in enumerate(ts):
            k = t.astype(np.float64) * 2.0 ** (8 * i)
            assert np.all(k == np.rint(k)) and np.abs(k).max() <= 130
            assert _is_bf16(t)


def test_four_slice_fold_with_generated_slices_over_many_windows():
    # precision mode 3 end to end on the CPU: table slices by the exact rule, generated slices by grid
    # rounding, every level sum exact in FP32, the epilogue's fold (L0 + rint(L1) into a TwoSum high part,
    # frac(L1) + L2 + L3 rounded once into the low part) over the 18 windows of a 2304-node rule
    f32 = np.float32
    worst = 0.0
    for seed in range(6):
        rng = np.random.default_rng(200 + seed)
        hi, lo = f32(0.0), f32(0.0)
        xs, ys = [], []
        for _ in range(2304 // NODES):
            xa, ha, la, sa = _window(rng)
            xb, p, e, sb = _gen_window(rng)
            xs.append(xa)
            ys.append((p.astype(np.float64) + e.astype(np.float64)))
            A = [k.astype(np.float64) * 2.0 ** (-8 * i) for i, k in enumerate(_slices(ha, la, sa, 4))]
            Bs = [t.astype(np.float64) for t in _slices4_pe(p, e, sb)]
            lv = [sum(np.dot(A[i], Bs[L - i]) for i in range(L + 1)) for L in range(4)]
            for L, v in enumerate(lv):
                assert float(np.float32(v)) == v and abs(v * 2.0 ** (8 * L)) < 2.0 ** 24
            L0, L1, L2, L3 = (f32(v) for v in lv)
            sc = f32(2.0 ** (-sa - sb))
            l1h = f32(np.rint(L1))
            xa_ = f32(L0 + l1h)
            xb_ = f32(f32(L1 - l1h) + L2)
            assert float(xa_) == float(L0) + float(l1h) and float(xb_) == float(L1 - l1h) + float(L2)
            hi, r1 = _two_sum(hi, f32(xa_ * sc))
            lo = f32(np.float64(f32(xb_ + L3)) * np.float64(sc) + np.float64(f32(lo + r1)))
        a, b = np.concatenate(xs), np.concatenate(ys)
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
        err = abs(float(Fraction(float(hi)) + Fraction(float(lo)) - exact))
        scale = float(np.abs(a).max() * np.abs(b).max())
        assert err <= 2.0 ** -27 * scale, seed
        worst = max(worst, err / scale)
    assert worst > 2.0 ** -45   # the truncated levels are really dropped


def test_wide_level_mmas_land_each_product_on_its_level():
    # The four-slice contraction issues, per table slice A_i and K step, one MMA A_i [B_0 .. B_{3-i}] into
    # accumulator columns 48 i .. 191 (the generated slices lie one after the other).  Emulated with exact
    # integer arithmetic: column block L then holds sum_{i + j = L} A_i B_j^T, the level sums.
    rng = np.random.default_rng(31)
    M, N, K = 8, 48, 16
    A = [rng.integers(-129, 130, (M, K)) for _ in range(4)]
    B = [rng.integers(-130, 131, (N, K)) for _ in range(4)]
    D = np.zeros((M, 4 * N), dtype=np.int64)
    for i in range(4):
        Bcat = np.concatenate(B[:4 - i])                 # rows of B_0 .. B_{3-i}: N (4 - i) rows
        D[:, N * i:N * 4] += A[i] @ Bcat.T
    for L in range(4):
        want = sum(A[i] @ B[L - i].T for i in range(L + 1))
        assert np.array_equal(D[:, N * L:N * (L + 1)], want)


def test_generated_tile_store_layout_of_the_four_slice_producer():
    # Each producer thread (row n, part p) stores nodes 2p, 2p + 1 and 16 + 2p, 17 + 2p of a 32-node chunk as
    # two 4-byte words at n 64 + ((p >> 2) ^ s) 16 + 4 (p & 3) and n 64 + ((2 + (p >> 2)) ^ s) 16 + 4 (p & 3),
    # s = (n >> 1) & 3.  Every byte of the 48-row tile is written once, and node m of row n lands where the
    # 64-byte-swizzled K-major layout the MMA reads puts it: 16-byte chunk (2m / 16) ^ s, byte 2m % 16.
    owner = {}
    for n in range(48):
        s = (n >> 1) & 3
        for p in range(8):
            for h, nodes in ((0, (2 * p, 2 * p + 1)), (1, (16 + 2 * p, 17 + 2 * p))):
                base = n * 64 + (((h * 2 + (p >> 2)) ^ s) << 4) + 4 * (p & 3)
                for k, m in enumerate(nodes):
                    for byte in (base + 2 * k, base + 2 * k + 1):
                        assert byte not in owner
                        owner[byte] = (n, m)
                    want = n * 64 + ((((2 * m) // 16) ^ s) << 4) + (2 * m) % 16
                    assert base + 2 * k == want
    assert sorted(owner) == list(range(48 * 64))
