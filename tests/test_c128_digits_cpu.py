"""The arithmetic the complex128 fused blocks rely on, restated with Python
integers (no GPU, no CUDA code): the error-free split of Ozaki, Ogita, Oishi
and Rump (2012) in the fixed-point, balanced-digit form the kernel uses.

  - a component x of a row whose largest biased exponent is emax is taken as
    t = trunc(x 2^(47 - E)), E = emax - 1022, so |t| < 2^47;
  - the bytes of |t| + 128 (1 + 256 + ... + 256^5), each less 128 (the top
    one from bit 40 up), times x's sign, are six balanced digits d_i with
    t = sum_i d_i 256^(5 - i) and |d_i| <= 128 (exact in FP16);
  - products of two digits are at most 2^14 and a level l = i + j sums at most
    6 x 32 of them, below 2^22, so an FP32 accumulator holds it exactly and
    the bits of D + 1.5 2^23 are 0x4B400000 + D;
  - pairs of levels combine on those raw bits modulo 2^32 with one constant:
    D_0 256 + D_1 = u_0 256 + u_1 - 257 0x4B400000.

The digit split is checked on rows of random magnitudes, signs, zeros and
subnormals; the bound and the recombination on random level values at their
extremes."""
import math
import struct

import numpy as np

OFF = 0x808080808080
MAGIC = 0x4B400000


def bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def f32_bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def magnitude_plus_offset(x: float, emax: int) -> int:
    """|t| + OFF from the bits of x (zero and subnormal x give t = 0)."""
    b = bits(x)
    e = (b >> 52) & 0x7FF
    if e == 0:
        return OFF
    sh = emax - e + 6
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    return (m >> sh if sh < 64 else 0) + OFF


def digits(x: float, emax: int):
    tp = magnitude_plus_offset(x, emax)
    sign = -1 if bits(x) >> 63 else 1
    top = (tp >> 40) - 128
    low = [((tp >> (8 * (4 - k))) & 255) - 128 for k in range(5)]
    return [sign * d for d in [top] + low]


def rows(rng, count=400):
    for r in range(count):
        scale = 2.0 ** int(rng.integers(-1000, 1000))
        row = rng.standard_normal(32) * np.exp2(rng.integers(-60, 1, 32)) * scale
        if r % 7 == 0:
            row[rng.integers(0, 32)] = 0.0
        if r % 11 == 0:
            row[rng.integers(0, 32)] = -0.0
        if r % 13 == 0:
            row[rng.integers(0, 32)] = 5e-324
        if r % 17 == 0:
            row[:] = np.nextafter(2.0 ** int(rng.integers(-20, 20)), 0.0)   # just below a power of two
        yield [float(v) for v in row]


def test_balanced_digits_are_exact_and_bounded():
    rng = np.random.default_rng(7)
    seen_top = set()
    for row in rows(rng):
        emax = max((bits(v) >> 52) & 0x7FF for v in row)
        E = emax - 1022
        for x in row:
            d = digits(x, emax)
            assert all(abs(v) <= 128 for v in d)
            seen_top.add(abs(d[0]))
            e = (bits(x) >> 52) & 0x7FF
            want = 0 if e == 0 else math.trunc(math.ldexp(x, 47 - E))
            assert abs(want) < 2 ** 47
            assert sum(v * 256 ** (5 - i) for i, v in enumerate(d)) == want
    # the largest components reach the top digit's extreme
    assert 128 in seen_top


def test_level_sums_stay_exact_in_fp32():
    # at most min(l + 1, 6) digit pairs per level, 32 terms each, |d| <= 128
    worst = 6 * 32 * 128 * 128
    assert worst < 2 ** 22
    for D in (worst, -worst, worst - 1, 0, 1, -1):
        assert float(np.float32(D)) == D
        assert f32_bits(float(np.float32(D) + np.float32(1.5 * 2 ** 23))) == MAGIC + D


def test_level_pairs_combine_on_raw_bits():
    rng = np.random.default_rng(11)
    bound = [(l + 1) * 32 * 128 * 128 for l in range(6)]

    def s32(v):
        v &= 0xFFFFFFFF
        return v - (1 << 32) if v >> 31 else v

    for trial in range(5000):
        if trial < 64:
            D = [bound[l] * (1 if (trial >> l) & 1 else -1) for l in range(6)]
        else:
            D = [int(rng.integers(-bound[l], bound[l] + 1)) for l in range(6)]
        u = [f32_bits(float(np.float32(d) + np.float32(1.5 * 2 ** 23))) for d in D]
        a01 = s32(u[0] * 256 + u[1] - 257 * MAGIC)
        a23 = s32(u[2] * 256 + u[3] - 257 * MAGIC)
        a45 = s32(u[4] * 256 + u[5] - 257 * MAGIC)
        T = a01 * 2 ** 32 + a23 * 65536 + a45
        assert T == sum(D[l] * 256 ** (5 - l) for l in range(6))
        assert abs(T) < 2 ** 63
