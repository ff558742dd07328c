"""Pins of the oracle's binary16 rounding, binary16 addition and the three quantizers of paper
Sec. 4.2 (round-to-nearest, exact stochastic rounding, dithered rounding). CPU only.

Independent references: numpy's float16 conversion (round-to-nearest-even from float64) and
numpy's float16 addition (computed in binary32 and rounded once more, which is a correctly rounded
binary16 sum because binary32 carries 2*11+2 significand bits), numpy.nextafter for the directed
roundings, and closed forms for the stochastic-rounding probabilities.
"""
import numpy as np
import pytest

import oracle

rng = np.random.default_rng(2024)


def _interesting_floats(n=40000):
    xs = [0.0, -0.0, 1.0, -1.0, 65504.0, 65519.99, 65520.0, 65536.0, 1e9, -1e9, 2.0**-24, 2.0**-25,
          3 * 2.0**-26, 2.0**-14, 2.0**-15, 6.1e-5, 1.0 + 2.0**-11, 1.0 + 3 * 2.0**-12, np.inf, -np.inf]
    h = rng.integers(0, 0x7C00, size=n // 4, dtype=np.uint16).view(np.float16).astype(np.float64)
    mid = h * (1.0 + rng.uniform(-2.0**-10, 2.0**-10, size=h.size))  # near binary16 values and midpoints
    logs = rng.uniform(-30, 17, size=n // 2)
    rnd = np.sign(rng.standard_normal(logs.size)) * 2.0**logs
    v = np.concatenate([np.array(xs), h, -h, mid, rnd]).astype(np.float32).astype(np.float64)
    return v


def test_round_nearest_matches_numpy_float16():
    for x in _interesting_floats():
        want = np.array([x]).astype(np.float16).view(np.uint16)[0]
        got = oracle.round_to_half(x, 0)
        if np.isnan(x):
            continue
        assert got == want, (x, hex(got), hex(want))


def _directed_ref(x, mode):
    """RD/RU from the round-to-nearest result and numpy.nextafter."""
    h = np.float16(x)
    if np.isinf(h) and np.isfinite(x):
        h = np.float16(np.copysign(65504.0, x)) if abs(x) < 65536 else h
    hv = float(h)
    if mode == 1:  # toward -inf
        if hv > x:
            h = np.nextafter(h, np.float16(-np.inf))
    else:
        if hv < x:
            h = np.nextafter(h, np.float16(np.inf))
    return np.array([h]).view(np.uint16)[0]


@pytest.mark.parametrize("mode", [1, 2])
def test_directed_rounding_matches_nextafter(mode):
    for x in _interesting_floats(8000):
        if not np.isfinite(x) or abs(x) >= 65536:
            continue
        got = oracle.round_to_half(x, mode)
        want = _directed_ref(x, mode)
        assert got == want, (x, mode, hex(got), hex(want))


def test_directed_rounding_overflow():
    assert oracle.round_to_half(1e6, 1) == 0x7BFF  # RD of a large positive: max finite
    assert oracle.round_to_half(1e6, 2) == 0x7C00  # RU: +inf
    assert oracle.round_to_half(-1e6, 1) == 0xFC00
    assert oracle.round_to_half(-1e6, 2) == 0xFBFF


def test_half_to_double_exhaustive():
    bits = np.arange(0, 1 << 16, dtype=np.uint32).astype(np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    for b in range(0, 1 << 16, 7):
        v = oracle.half_to_double(b)
        if np.isnan(ref[b]):
            assert np.isnan(v)
        else:
            assert v == ref[b]


def test_half_add_matches_numpy():
    a = rng.integers(0, 1 << 16, size=60000, dtype=np.uint32).astype(np.uint16)
    # exponents close to each other make carries and ties frequent
    b = (a.astype(np.int32) + rng.integers(-3000, 3000, size=a.size)).clip(0, 0xFFFF).astype(np.uint16)
    b[::3] = rng.integers(0, 1 << 16, size=b[::3].size, dtype=np.uint32).astype(np.uint16)
    fa, fb = a.view(np.float16), b.view(np.float16)
    with np.errstate(all="ignore"):
        ref = (fa + fb).view(np.uint16)
    for i in range(a.size):
        if np.isnan(fa[i]) or np.isnan(fb[i]) or np.isnan(ref.view(np.float16)[i]):
            continue
        got = oracle.half_add(int(a[i]), int(b[i]))
        assert got == ref[i], (hex(a[i]), hex(b[i]), hex(got), hex(ref[i]))


def test_rn_quantizer_is_float16_conversion():
    for x in _interesting_floats(4000):
        if np.isnan(x):
            continue
        assert oracle.quantize(x, 0.3, oracle.FP16_RN) == np.float16(np.float32(x)).view(np.uint16)


def test_sr_returns_a_neighbour_and_exact_values_unchanged():
    for x in _interesting_floats(3000):
        if not np.isfinite(x) or abs(x) > 65504:
            continue
        lo, hi = oracle.round_to_half(x, 1), oracle.round_to_half(x, 2)
        for u in (0.0, 0.25, 0.5, 0.999999):
            q = oracle.quantize(x, u, oracle.FP16_SR)
            assert q in (lo, hi)
    for h in rng.integers(0, 0x7BFF, size=500):
        x = float(np.uint16(h).view(np.float16))
        for u in (0.0, 0.7):
            assert oracle.quantize(x, u, oracle.FP16_SR) == np.uint16(h)


def test_sr_probability_closed_form():
    # P(round up) over the 2^24-point uniform grid equals ceil(((x - rd)/Delta) * 2^24) / 2^24 exactly:
    # round up iff fl32(u * Delta) < x - rd, and u * Delta is exact (Delta a power of two).
    for x in (1.0 + 3 * 2.0**-13, 0.3, -0.3, 1000.7, 2.0**-20 * 1.37, -7.77e-3):
        x = float(np.float32(x))
        rd = oracle.half_to_double(oracle.round_to_half(x, 1))
        ru = oracle.half_to_double(oracle.round_to_half(x, 2))
        delta, e = ru - rd, x - rd
        # threshold count: number of grid points u = j/2^24 with u*delta < e
        expected_up = int(np.ceil(e / delta * 2**24))
        # verify by bisection over j (monotone in u)
        lo, hi = 0, 2**24
        while lo < hi:
            mid = (lo + hi) // 2
            q = oracle.quantize(x, mid / 2**24, oracle.FP16_SR)
            if q == oracle.round_to_half(x, 2) and ru != rd:
                lo = mid + 1
            else:
                hi = mid
        assert lo == expected_up


def test_sr_unbiased_monte_carlo():
    # E[SR(x)] = x (paper Sec. 2.3): mean over 10^5 Philox draws within 4 sigma, sigma <= Delta/2/sqrt(N).
    for x in (0.1, 1.0 + 2.0**-12, -3.14159, 123.456):
        x = float(np.float32(x))
        N = 100_000
        vals = np.array([oracle.half_to_double(oracle.quantize(x, oracle.uniform(5, 0, c, t), oracle.FP16_SR))
                         for c, t in zip(range(N), range(N))])
        delta = oracle.half_to_double(oracle.round_to_half(x, 2)) - oracle.half_to_double(oracle.round_to_half(x, 1))
        assert abs(vals.mean() - x) < 4 * (delta / 2) / np.sqrt(N)


def test_dither_noise_amplitude_and_rn_fallback():
    # noise = (u - 1/2) * x * 2^-10: u = 1/2 gives plain round-to-nearest; any u moves the
    # result by at most one binary16 neighbour of RN(x).
    for x in _interesting_floats(3000):
        if not np.isfinite(x) or abs(x) > 60000 or x == 0:
            continue
        assert oracle.quantize(x, 0.5, oracle.FP16_DITHER) == oracle.round_to_half(x, 0)
        rn = oracle.half_to_double(oracle.round_to_half(x, 0))
        for u in (0.0, 0.999999):
            q = oracle.half_to_double(oracle.quantize(x, u, oracle.FP16_DITHER))
            assert abs(q - rn) <= 2 * abs(x) * 2.0**-10 + 2.0**-24


def _dither_switch_index(x, before, after):
    """Smallest grid index i in [0, 2^24) with dither(x, i / 2^24) != `before` (bisection; the
    result is monotone in u), after checking the two ends of the grid."""
    assert oracle.quantize(x, 0.0, oracle.FP16_DITHER) == before
    assert oracle.quantize(x, (2**24 - 1) / 2**24, oracle.FP16_DITHER) == after
    lo, hi = 0, 2**24
    while lo < hi:
        mid = (lo + hi) // 2
        if oracle.quantize(x, mid / 2**24, oracle.FP16_DITHER) == before:
            lo = mid + 1
        else:
            hi = mid
    return lo


def test_dither_moves_one_to_its_lower_neighbour_on_a_hand_derived_share_of_u():
    # Values derived by hand from Sec. 4.2's operation order with factor 2^-10 (not from the code):
    # for x = 1 and u = i 2^-24, noise = (i - 2^23) 2^-34 is exact, and y = fl32(1 + noise). For
    # D = 2^23 - i > 0, 1 - D 2^-34 rounds to the FP32 grid of [1/2, 1) (spacing 2^-24) as
    # 1 - rne(D / 1024) 2^-24. binary16 round-to-nearest sends y to 0x3BFF = 1 - 2^-11 iff
    # y < 1 - 2^-12 (the midpoint; at the midpoint the tie goes to the even 0x3C00), i.e. iff
    # rne(D / 1024) > 4096, i.e. D > 4096.5 * 1024 = 2^22 + 512, i.e. i < 2^22 - 512 = 4193792.
    # Above u = 1/2, y reaches at most fl32(1 + 2^-11 - 2^-34) = 1 + 2^-11, whose tie also goes to
    # 0x3C00. So the result is 0x3BFF exactly for i < 4193792 and 0x3C00 from there on: dither moves
    # the exactly representable 1.0 to a neighbour with probability (2^22 - 512) / 2^24.
    # A factor of 2^-11 would give no move at all (y >= 1 - 2^-12), 2^-9 would reach 0x3BFE, and
    # rounding the exact 1 + noise without the FP32 step would switch at 2^22.
    assert _dither_switch_index(1.0, 0x3BFF, 0x3C00) == 4193792
    assert oracle.quantize(1.0, (4193792 - 1) / 2**24, oracle.FP16_DITHER) == 0x3BFF
    # x = -1: the noise scales with x, so the same u move -1 towards zero by the same rule.
    assert _dither_switch_index(-1.0, 0xBBFF, 0xBC00) == 4193792
    # factor 2^-9 would reach the second neighbour 1 - 2^-10 (0x3BFE) at u = 0; 2^-10 never does
    assert oracle.quantize(1.0, 0.0, oracle.FP16_DITHER) != 0x3BFE


def test_dither_leaves_the_smallest_normal_unmoved():
    # x = 2^-14 (0x0400): amplitude x 2^-10 = 2^-24, so |noise| <= 2^-25, half the binary16 spacing
    # 2^-24 on both sides of 2^-14; only u = 0 reaches the midpoint 2^-14 - 2^-25, whose tie goes to the
    # even 0x0400. Every u gives 0x0400 (below 2^-14 dither is plain round-to-nearest in effect).
    x = 2.0**-14
    for i in (0, 1, 2**22, 2**23, 2**24 - 1):
        assert oracle.quantize(x, i / 2**24, oracle.FP16_DITHER) == 0x0400


def test_dither_product_order_is_not_observable():
    # (u - 1/2) * (x * 2^-10) and ((u - 1/2) * x) * 2^-10 round to the same binary16 value for every
    # x: multiplying by a power of two is exact outside FP32's subnormal range, and inside it the
    # noise is below binary16's resolution of any x it is added to. So no test can (or needs to) tell
    # the two orders apart; here checked on 20000 sampled (x, u) pairs with numpy float32 arithmetic.
    rng = np.random.default_rng(23)
    xs = np.concatenate([rng.standard_normal(10000), rng.uniform(-60000, 60000, 5000),
                         rng.standard_normal(5000) * 1e-6]).astype(np.float32)
    us = (rng.integers(0, 2**24, size=xs.size) * 2.0**-24).astype(np.float32)
    f = np.float32(2.0**-10)
    a = ((us - np.float32(0.5)) * (xs * f)).astype(np.float32)
    b = (((us - np.float32(0.5)) * xs).astype(np.float32) * f).astype(np.float32)
    assert np.array_equal(oracle.round_to_half_array((xs + a).astype(np.float32), 0),
                          oracle.round_to_half_array((xs + b).astype(np.float32), 0))
    for q in range(0, xs.size, 97):
        assert oracle.quantize(float(xs[q]), float(us[q]), oracle.FP16_DITHER) == \
            oracle.round_to_half_array(np.array([xs[q] + a[q]], dtype=np.float32), 0)[0]


def test_array_forms_equal_scalar_forms():
    # the array entry points (used by the exhaustive GPU pins) are the scalar functions element-wise
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 1 << 32, size=4000, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    for mode in (0, 1, 2):
        arr = oracle.round_to_half_array(x, mode)
        assert all(int(arr[i]) == oracle.round_to_half(float(x[i]), mode) for i in range(0, 4000, 7))
    arr = oracle.round_to_bf16_array(x)
    assert all(int(arr[i]) == oracle.round_to_bf16(float(x[i])) for i in range(0, 4000, 7))
    a = rng.integers(0, 1 << 16, size=4000).astype(np.uint16)
    b = rng.integers(0, 1 << 16, size=4000).astype(np.uint16)
    h = oracle.half_add_array(a, b)
    g = oracle.bf16_add_array(a, b)
    for i in range(0, 4000, 7):
        assert int(h[i]) == oracle.half_add(int(a[i]), int(b[i]))
        assert int(g[i]) == oracle.bf16_add(int(a[i]), int(b[i]))
