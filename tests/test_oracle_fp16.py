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
