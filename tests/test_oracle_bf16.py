"""Pins of the oracle's bfloat16 arithmetic (the BF16 round-to-nearest rule; paper Sec. 4.2 names BF16
beside FP16 as a 16-bit reduction target) against PyTorch's CPU bfloat16 conversion and addition,
an implementation independent of the oracle, and against closed forms."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def _torch_bf16_bits(x32: np.ndarray) -> np.ndarray:
    t = torch.from_numpy(np.ascontiguousarray(x32, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


def _rng_floats(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-140, 128, n)
    sign = rng.choice([-1.0, 1.0], n)
    return (sign * np.ldexp(mant, expo)).astype(np.float32)


def test_bf16_to_double_exhaustive():
    h = np.arange(1 << 16, dtype=np.uint16)
    ref = torch.from_numpy(h.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.bf16_to_double(int(v)) for v in h[::7]])
    r = ref[::7]
    fin = np.isfinite(r)
    assert np.array_equal(got[fin], r[fin])
    assert np.array_equal(np.isnan(got), np.isnan(r))
    assert np.array_equal(oracle.bf16bits_to_f64(h)[np.isfinite(ref)], ref[np.isfinite(ref)])


def test_round_to_bf16_matches_torch_random_and_subnormal():
    x = np.concatenate([_rng_floats(20000, 1), np.float32([0.0, -0.0, 1e-45, -1e-45, 3.4e38, -3.4e38])])
    got = np.array([oracle.round_to_bf16(float(v)) for v in x], dtype=np.uint16)
    assert np.array_equal(got, _torch_bf16_bits(x))


def test_round_to_bf16_ties_go_to_even():
    # x = b + half an ulp of bfloat16 b, exactly representable in binary32: ties to the even pattern.
    rng = np.random.default_rng(2)
    b = oracle.bf16bits_to_f64(rng.integers(0x0080, 0x7F00, 4000, dtype=np.uint16))
    up = oracle.bf16bits_to_f64(np.array([oracle.round_to_bf16(v) for v in b], dtype=np.uint16))
    assert np.array_equal(up, b)  # bfloat16 values round to themselves
    ulp = np.ldexp(1.0, np.frexp(b)[1] - 8)
    x = (b + ulp / 2).astype(np.float32)
    assert np.array_equal(x.astype(np.float64), b + ulp / 2)
    got = np.array([oracle.round_to_bf16(float(v)) for v in x], dtype=np.uint16)
    assert np.all(got % 2 == 0)
    assert np.array_equal(got, _torch_bf16_bits(x))


def test_round_to_bf16_overflow_to_inf():
    big = np.float32(np.ldexp(255.5 / 128.0, 127))  # halfway between the largest bfloat16 and 2^128
    assert oracle.round_to_bf16(float(big)) == 0x7F80
    assert oracle.round_to_bf16(float(np.nextafter(big, np.float32(0)))) == 0x7F7F
    assert oracle.round_to_bf16(float("inf")) == 0x7F80 and oracle.round_to_bf16(-float("inf")) == 0xFF80


def test_bf16_add_matches_torch():
    rng = np.random.default_rng(3)
    a = _torch_bf16_bits(_rng_floats(20000, 4))
    b = _torch_bf16_bits(_rng_floats(20000, 5))
    # add close-in-magnitude pairs and cancellations as well
    b[:5000] = _torch_bf16_bits(-oracle.bf16bits_to_f64(a[:5000]).astype(np.float32) * np.float32(0.999))
    ta = torch.from_numpy(a.view(np.int16)).view(torch.bfloat16)
    tb = torch.from_numpy(b.view(np.int16)).view(torch.bfloat16)
    ref = (ta + tb).view(torch.int16).numpy().view(np.uint16)
    got = np.array([oracle.bf16_add(int(x), int(y)) for x, y in zip(a, b)], dtype=np.uint16)
    fin = np.isfinite(oracle.bf16bits_to_f64(ref))
    assert np.array_equal(got[fin], ref[fin])


def test_quantize_bf16_ignores_u():
    for x in _rng_floats(500, 6):
        q = oracle.round_to_bf16(float(x))
        for u in (0.0, 0.3, 0.999):
            assert oracle.quantize(float(x), u, oracle.BF16_RN) == q


def test_canonical_bf16_exact_on_small_integers():
    # k = 4: scale 1/2 is exact; integer data gives chunk totals and sums representable in bfloat16
    # (|values| well below 2^7 at half-integer spacing), so the BF16 sketch equals the FP64 sketch.
    rng = np.random.default_rng(7)
    m, n, d, k = 3000, 5, 256, 4
    A = rng.integers(-2, 3, size=(m, n)).astype(np.float32)
    Y = oracle.sketch_canonical(A, d, k, 11, oracle.BF16_RN, 500)
    Y64 = oracle.sketch_f64(A, d, k, 11)
    assert np.abs(Y64).max() < 64
    assert np.array_equal(oracle.bf16bits_to_f64(Y), Y64)


def test_canonical_bf16_error_bound():
    # Each chunk total is rounded once and each of the T additions rounds once, relative error at most
    # 2^-8 per rounding: |Y - Y64| <= sum over chunks of |x_t| * 2^-8 * (T + 1) (crude bound).
    rng = np.random.default_rng(8)
    m, n, d, k, R = 4000, 3, 64, 2, 1000
    A = rng.standard_normal((m, n)).astype(np.float32)
    Y = oracle.bf16bits_to_f64(oracle.sketch_canonical(A, d, k, 5, oracle.BF16_RN, R))
    Y64 = oracle.sketch_f64(A, d, k, 5)
    absum = np.abs(oracle.dense_S(d, k, 5, m)) @ np.abs(A).astype(np.float64)
    T = m // R
    assert np.all(np.abs(Y - Y64) <= absum * 2.0 ** -8 * (T + 1) + 1e-30)
    assert oracle.rel_fro(Y, Y64) > 0  # it does round
