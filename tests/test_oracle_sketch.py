"""Pins of the oracle sketches (CPU only): the FP64 sketch against dense S A by brute force, the
canonical FP32/FP16 accumulation against closed forms, exact special cases, invariants and the
arithmetic error bound. Paper Sec. 4.1 (scatter semantics), Sec. 4.2 (quantized accumulation).
"""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

RULES = [oracle.FP32, oracle.FP16_RN, oracle.FP16_SR, oracle.FP16_DITHER]


def _as64(Y, rule):
    return Y.astype(np.float64) if rule == oracle.FP32 else oracle.halfbits_to_f64(Y)


@pytest.mark.parametrize("d,k,m,n", [(32, 4, 200, 5), (12, 1, 50, 3), (30, 3, 77, 4), (64, 8, 128, 7)])
def test_f64_sketch_equals_dense_product(d, k, m, n):
    A = inputs.host_matrix(m, n, "incoherent", seed=3)
    S = oracle.dense_S(d, k, seed=9, m=m)
    Y = oracle.sketch_f64(A, d, k, 9)
    ref = S @ A.astype(np.float64)
    assert np.allclose(Y, ref, rtol=1e-14, atol=1e-14)


def test_f64_sketch_is_linear_and_row_additive():
    d, k, m, n = 64, 4, 1000, 6
    A = inputs.host_matrix(m, n, "incoherent", seed=1)
    Y = oracle.sketch_f64(A, d, k, 3)
    # rows [0, 400) and [400, m) sketched separately with global row indices sum to the whole
    Y1 = oracle.sketch_f64(A[:400], d, k, 3)
    A2 = A.copy()
    A2[:400] = 0
    Y2 = oracle.sketch_f64(A2, d, k, 3)
    assert np.allclose(Y1 + Y2, Y, rtol=1e-13, atol=1e-13)
    assert np.allclose(oracle.sketch_f64(4 * A, d, k, 3), 4 * Y, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("rule", [oracle.FP32, oracle.FP16_RN, oracle.FP16_SR])
@pytest.mark.parametrize("k", [1, 4])
def test_canonical_exact_on_integer_data(rule, k):
    # Small integers: every partial sum, scaling by 1/sqrt(k) in {1, 1/2} and every binary16 sum
    # below 2048 is exact, so these rules must return the exact dense product (RN and SR leave a
    # representable value unchanged). Dither is excluded: its noise of up to one ulp can move a
    # representable value to a neighbour.
    d, m, n = 64, 300, 8
    A = np.random.default_rng(0).integers(-3, 4, size=(m, n)).astype(np.float32)
    S = oracle.dense_S(d, k, seed=4, m=m)
    exact = S @ A.astype(np.float64)
    assert np.abs(exact).max() < 2048
    for R in (1, 7, m):
        Y = _as64(oracle.sketch_canonical(A, d, k, 4, rule, R), rule)
        assert np.array_equal(Y, exact), (rule, k, R)


def _rows_with_same_target(d, k, seed, m, j, count):
    rows, _ = oracle.s_pattern(d, k, seed, m)
    vals, inv = np.unique(rows[:, j], return_inverse=True)
    for v in range(len(vals)):
        idx = np.flatnonzero(inv == v)
        if len(idx) >= count:
            return int(vals[v]), idx[:count]
    raise AssertionError("no target hit often enough")


def test_canonical_fp32_sums_rows_in_ascending_order():
    # Three rows reaching the same output with values (1e8, 1, -1e8) in ascending row order: the
    # sequential FP32 sum is (1e8 + 1) - 1e8 = 0 (1e8 + 1 rounds to 1e8), not the exact 1.
    d, k, seed, m = 16, 1, 21, 400
    r, idx = _rows_with_same_target(d, k, seed, m, 0, 3)
    rows, signs = oracle.s_pattern(d, k, seed, m)
    A = np.zeros((m, 1), dtype=np.float32)
    vals = [1e8, 1.0, -1e8]
    for q, i in enumerate(idx):
        A[i, 0] = vals[q] * signs[i, 0]  # undo the sign so the contributions are exactly vals
    Y = oracle.sketch_canonical(A, d, k, seed, oracle.FP32, R=m)
    assert Y[r, 0] == 0.0
    # with one row per chunk the contributions are chunk totals added in FP32: the same sequence
    assert oracle.sketch_canonical(A, d, k, seed, oracle.FP32, R=1)[r, 0] == 0.0
    # the FP64 sketch gets the exact value
    assert oracle.sketch_f64(A, d, k, seed)[r, 0] == 1.0


def test_canonical_fp16_chunking_closed_form():
    # 1 + sixteen contributions of 2^-12 to one output (k = 1):
    #  R = 1: each 2^-12 is below half an ulp of 1 in binary16 -> RN keeps 1 every time: Y = 1.
    #  R = all rows: one FP32 partial 1 + 2^-8, exactly representable in binary16: Y = 1 + 2^-8.
    d, k, seed, m = 8, 1, 5, 600
    r, idx = _rows_with_same_target(d, k, seed, m, 0, 17)
    _, signs = oracle.s_pattern(d, k, seed, m)
    A = np.zeros((m, 1), dtype=np.float32)
    A[idx[0], 0] = 1.0 * signs[idx[0], 0]
    for i in idx[1:]:
        A[i, 0] = 2.0**-12 * signs[i, 0]
    y1 = oracle.halfbits_to_f64(oracle.sketch_canonical(A, d, k, seed, oracle.FP16_RN, 1))[r, 0]
    ym = oracle.halfbits_to_f64(oracle.sketch_canonical(A, d, k, seed, oracle.FP16_RN, m))[r, 0]
    assert y1 == 1.0
    assert ym == 1.0 + 2.0**-8


@pytest.mark.parametrize("rule", RULES)
def test_canonical_scale_and_sign_invariance(rule):
    # Multiplying A by 2 or by -1 is exact in FP32 and commutes with every rounding rule (the
    # quantizers are scale- and sign-covariant for binary scalings away from overflow/underflow).
    d, k, m, n = 128, 4, 3000, 6
    A = inputs.host_matrix(m, n, "incoherent", seed=8)
    Y = _as64(oracle.sketch_canonical(A, d, k, 2, rule, 256), rule)
    Y2 = _as64(oracle.sketch_canonical(2 * A, d, k, 2, rule, 256), rule)
    assert np.array_equal(Y2, 2 * Y)
    if rule in (oracle.FP32, oracle.FP16_RN):
        Yn = _as64(oracle.sketch_canonical(-A, d, k, 2, rule, 256), rule)
        assert np.array_equal(Yn, -Y)


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("R", [1, 64, 5000])
def test_canonical_within_arithmetic_error_bound(rule, R):
    # Per output with T chunk contributions x_t (FP32 partials of the exact values):
    # |Y - Y64| <= sum_t |P_t err| * s + sum_t |q_t - x_t| + sum_t (1/2) ulp16(running sum)
    # bounded here crudely by: FP32 partial errors (2^-24 * sum|contrib| * rows), one binary16 ulp of
    # each x_t for the quantizer (SR/dither; half for RN), and half an ulp of |Y|max per addition.
    d, k, m, n = 64, 4, 5000, 4
    A = inputs.host_matrix(m, n, "incoherent", seed=12)
    Y64 = oracle.sketch_f64(A, d, k, 7)
    Y = _as64(oracle.sketch_canonical(A, d, k, 7, rule, R), rule)
    S = oracle.dense_S(d, k, 7, m)
    absY = np.abs(S) @ np.abs(A.astype(np.float64))  # sum of |contributions| per output
    T = min(m, -(-m // R))  # chunks
    if rule == oracle.FP32:
        bound = 2.0**-23 * absY * (m + T + 2)
    else:
        ulp = lambda v: 2.0 ** (np.floor(np.log2(np.maximum(np.abs(v), 2.0**-14))) - 10)
        bound = 2.0**-23 * absY * (m + 2) + (T + 1) * ulp(absY) * 1.5
    assert np.all(np.abs(Y - Y64) <= bound)


def test_canonical_error_shrinks_with_chunking():
    # Expected FP16 error ~ 2e-4 * sqrt(T + 1) for T rounded contributions per output (one binary16
    # rounding of relative size ~2^-12 each, independent signs).
    m, n, d, k = 16384, 16, 256, 4
    A = inputs.host_matrix(m, n, "incoherent", seed=0)
    Y64 = oracle.sketch_f64(A, d, k, 0)
    e1 = oracle.rel_fro(oracle.halfbits_to_f64(oracle.sketch_canonical(A, d, k, 0, oracle.FP16_RN, 1)), Y64)
    e4096 = oracle.rel_fro(oracle.halfbits_to_f64(oracle.sketch_canonical(A, d, k, 0, oracle.FP16_RN, 4096)), Y64)
    assert e1 > 2e-3 > 1e-3 > e4096  # the paper-literal per-element scheme misses the 2e-3 gate here


def test_sampled_matches_full():
    m, n, d, k = 3000, 5, 48, 4
    A = inputs.host_matrix(m, n, "coherent", seed=2)
    rs = np.array([0, 5, 11, 47, 30, 12])
    cs = np.array([0, 4, 2, 1, 3, 0])
    for rule in RULES:
        full = _as64(oracle.sketch_canonical(A, d, k, 6, rule, 128), rule)
        Y64 = oracle.sketch_f64(A, d, k, 6)
        s64, sc = oracle.sketch_sampled(A, d, k, 6, rule, 128, rs, cs)
        assert np.allclose(s64, Y64[rs, cs], rtol=1e-14, atol=0)
        assert np.array_equal(sc, full[rs, cs])
