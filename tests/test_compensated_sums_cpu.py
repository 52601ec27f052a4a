"""The arithmetic scheme of the complex64 reductions, checked on the CPU.

The GPU sums |a|^2 over chunks of 8 complex64 amplitudes (16 squares) with
error-free FP32 transformations and carries each chunk into FP64:
  * the chunk is rescaled by 2^(127 - k), k the biased exponent of its largest
    component clamped to [1, 253] (exact: a power of two);
  * x^2 = h + l exactly (h = fl32(x * x), l = x * x - h: Dekker's product,
    formed on the GPU with an FMA);
  * h enters the running sum s through Knuth's TwoSum, err + l accumulate in e
    (the Dot2 scheme of Ogita, Rump & Oishi, SIAM J. Sci. Comput. 26(6), 2005);
  * (s + e) * 2^(2 (k - 127)) in FP64.
<sum Z> weights popcount bins with small integers through exact products
into one more compensated sum.

This test restates that scheme in numpy, one FP32 rounding per operation, and
checks it against exactly rounded sums of the same squares.  The bounds are
the scheme's own: for m non-negative terms |(s + e) - sum| <= (m + 1)^2 u^2
sum with u = 2^-24.  It does not call the CUDA library; the GPU tests compare
the kernels' norms, <sum Z> and shots with the FP64 oracle."""
import math

import numpy as np

F32 = np.float32
U = 2.0 ** -24


def _two_sum(s, h):
    t = (s + h).astype(F32)
    z = (t - s).astype(F32)
    err = ((s - (t - z).astype(F32)).astype(F32) + (h - z).astype(F32)).astype(F32)
    return t, err


def _pow2(amax):
    bits = amax.astype(F32).view(np.uint32)
    k = np.clip((bits >> 23).astype(np.int64), 1, 253)
    scale = ((254 - k).astype(np.uint32) << 23).view(F32)
    return scale, 2 * (k - 127)


def _chunks(rng, nch, m):
    """nch chunks of m FP32 components: normal, wide dynamic range, sparse,
    and whole chunks scaled from 2^-100 to 2^+60."""
    x = rng.standard_normal((nch, m)).astype(F32)
    mode = np.arange(nch) % 4
    spread = np.ldexp(1.0, rng.integers(-30, 30, (nch, m))).astype(F32)
    x = np.where((mode == 1)[:, None], (x * spread).astype(F32), x)
    x = np.where(((mode == 2)[:, None]) & (rng.random((nch, m)) < 0.6), F32(0), x)
    e = rng.integers(-100, 60, nch)
    return np.ldexp(x.astype(np.float64), e[:, None]).astype(F32)


def _compensated_squares(x):
    """Per chunk (rows of x): the scheme's FP64 result."""
    scale, sh = _pow2(np.max(np.abs(x), axis=1))
    y = (x * scale[:, None]).astype(F32)
    s = np.zeros(len(x), F32)
    e = np.zeros(len(x), F32)
    for j in range(x.shape[1]):
        v = y[:, j]
        h = (v * v).astype(F32)
        l = (v.astype(np.float64) ** 2 - h.astype(np.float64)).astype(F32)   # exact: Dekker's product
        s, err = _two_sum(s, h)
        e = (e + (err + l).astype(F32)).astype(F32)
    return np.ldexp(s.astype(np.float64), sh) + np.ldexp(e.astype(np.float64), sh)


def test_compensated_sum_of_squares_within_its_bound():
    rng = np.random.default_rng(11)
    x = _chunks(rng, 40000, 16)
    got = _compensated_squares(x)
    sq = x.astype(np.float64) ** 2                     # exact squares of FP32 values
    ref = np.array([math.fsum(r) for r in sq])
    nz = ref > 0
    rel = np.abs(got[nz] - ref[nz]) / ref[nz]
    assert np.all(got[~nz] == 0.0)
    assert rel.max() <= (16 + 1) ** 2 * U * U          # ~1.03e-12
    assert np.median(rel) <= 1e-14


def test_rescaling_keeps_tiny_and_huge_chunks_exact_enough():
    # chunks far outside FP32's squaring range: 2^-90 (squares underflow) and
    # 2^+70 (squares overflow) without the power-of-two rescale
    rng = np.random.default_rng(12)
    base = rng.standard_normal((1000, 16)).astype(F32)
    for e in (-90, 70):
        x = np.ldexp(base.astype(np.float64), e).astype(F32)
        got = _compensated_squares(x)
        ref = np.array([math.fsum(r) for r in x.astype(np.float64) ** 2])
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / ref) <= (16 + 1) ** 2 * U * U


def test_weighted_popcount_bins_within_bound():
    """<sum Z> per 16-amplitude chunk: bins by popcount of the low 4 index bits,
    weights n - 2 (popcount(chunk) + j) through exact products; the error is
    relative to sum_j |w_j| bin_j (the weights have both signs)."""
    rng = np.random.default_rng(13)
    nch, n = 20000, 30
    x = _chunks(rng, nch, 32)                          # 16 amplitudes: (re, im) pairs
    scale, sh = _pow2(np.max(np.abs(x), axis=1))
    y = (x * scale[:, None]).astype(F32)
    bs = [np.zeros(nch, F32) for _ in range(5)]
    be = [np.zeros(nch, F32) for _ in range(5)]
    exact = [np.zeros(nch) for _ in range(5)]
    for a in range(16):
        j = bin(a).count("1")
        for c in (2 * a, 2 * a + 1):
            v = y[:, c]
            h = (v * v).astype(F32)
            l = (v.astype(np.float64) ** 2 - h.astype(np.float64)).astype(F32)
            bs[j], err = _two_sum(bs[j], h)
            be[j] = (be[j] + (err + l).astype(F32)).astype(F32)
            exact[j] += x[:, c].astype(np.float64) ** 2      # exact up to FP64 rounding
    pc = rng.integers(0, n - 4, nch)
    ws = np.zeros(nch, F32)
    we = np.zeros(nch, F32)
    ref = np.zeros(nch)
    mag = np.zeros(nch)
    for j in range(5):
        w = (n - 2 * (pc + j)).astype(F32)
        h = (bs[j] * w).astype(F32)
        l = (bs[j].astype(np.float64) * w - h.astype(np.float64)).astype(F32)
        ws, err = _two_sum(ws, h)
        we = (we + err).astype(F32)
        we = (we + l).astype(F32)
        we = (we + (be[j] * w).astype(F32)).astype(F32)     # one FMA on the GPU
        ref += w.astype(np.float64) * exact[j]
        mag += np.abs(w.astype(np.float64)) * exact[j]
    got = np.ldexp(ws.astype(np.float64), sh) + np.ldexp(we.astype(np.float64), sh)
    nz = mag > 0
    assert np.max(np.abs(got[nz] - ref[nz]) / mag[nz]) <= 1e-12
