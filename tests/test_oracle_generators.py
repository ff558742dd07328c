"""Pins of the oracle's random generators and of the SparseStack pattern (CPU only).

Paper Sec. 2.2 (Definition of SparseStack: one nonzero per block of d/zeta rows, Rademacher
signs, uniform position) and Sec. 4.1 (values +-1/sqrt(zeta)); the generators are pinned to
their publishers' known-answer vectors.
"""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_philox_known_answers():
    for row in _rows("philox4x32_10_kat.txt"):
        vals = [int(x, 16) for x in row]
        ctr, key, want = vals[0:4], vals[4:6], tuple(vals[6:10])
        assert oracle.philox4x32_10(ctr, key) == want


def test_splitmix64_known_answers():
    for n, want in _rows("splitmix64_seed0.txt"):
        assert oracle.splitmix64_nth(0, int(n)) == int(want, 16)


def test_splitmix64_stream_is_sequential_generator():
    # The n-th output equals the n-th call of a stateful generator (state += gamma; mix(state)).
    seed = 0x1234_5678_9ABC_DEF0
    state = seed
    for n in range(1, 50):
        state = (state + 0x9E3779B97F4A7C15) % 2**64
        assert oracle.splitmix64_nth(seed, n) == oracle.splitmix64_mix(state)


def test_uniform_is_24_bit_grid():
    us = [oracle.uniform(7, r, c, t) for r in range(4) for c in range(8) for t in range(3)]
    for u in us:
        assert 0.0 <= u < 1.0
        assert float(u * 2**24).is_integer()
    # columns 4q..4q+3 use the four words of one Philox call
    w = oracle.philox4x32_10([3, 1, 5, 0], [7, 0])
    for c in range(4, 8):
        assert oracle.uniform(7, 3, c, 5) == (w[c - 4] & 0xFFFFFF) / 2**24


@pytest.mark.parametrize("d,k", [(256, 4), (256, 1), (96, 3), (4096, 8), (30, 5)])
def test_pattern_structure(d, k):
    m = 5000
    rows, signs = oracle.s_pattern(d, k, seed=11, m=m)
    B = d // k
    # exactly one nonzero per block of B rows, in block order
    for j in range(k):
        assert np.all(rows[:, j] >= j * B) and np.all(rows[:, j] < (j + 1) * B)
    assert set(np.unique(signs)) <= {-1, 1}


def test_dense_S_columns_unit_norm_and_k_nonzeros():
    d, k, m = 64, 4, 300
    S = oracle.dense_S(d, k, seed=5, m=m)
    nnz = (S != 0).sum(axis=0)
    assert np.all(nnz == k)
    assert np.allclose(np.linalg.norm(S, axis=0), 1.0, rtol=0, atol=1e-15)
    assert np.all(np.isin(np.abs(S[S != 0]), [1.0 / np.sqrt(k)]))


def test_pattern_uniform_chi2_and_sign_balance():
    # 10^6 draws: position uniform within each block (chi-square, 1e-6 false-alarm level) and
    # signs balanced (5 sigma).
    from scipy import stats
    d, k, m = 512, 4, 250_000
    rows, signs = oracle.s_pattern(d, k, seed=123, m=m)
    B = d // k
    for j in range(k):
        counts = np.bincount(rows[:, j] - j * B, minlength=B)
        chi2 = ((counts - m / B) ** 2 / (m / B)).sum()
        assert stats.chi2.sf(chi2, B - 1) > 1e-6
    s = signs.astype(np.int64).sum()
    assert abs(s) < 5 * np.sqrt(m * k)


def test_k1_is_countsketch_from_definition():
    # With k = 1 the operator is CountSketch: S e_i = rho_i e_{s_i} with the same stream word.
    d, m, seed = 100, 2000, 99
    rows, signs = oracle.s_pattern(d, 1, seed, m)
    for i in range(0, m, 97):
        w = oracle.splitmix64_nth(seed, i + 1) >> 32  # even block -> high half
        assert rows[i, 0] == (w * d) >> 32
        assert signs[i, 0] == (-1 if (w & 1) else 1)


def test_expected_StS_is_identity():
    # diag(S^T S) = 1 exactly for every draw; the off-diagonal mean over N draws is 0 within
    # 5 sigma, sigma^2 = 1/d per entry per draw (k nonzeros of 1/k, collision prob. 1/B each).
    d, k, m, N = 16, 4, 64, 2000
    acc = np.zeros((m, m))
    for s in range(N):
        S = oracle.dense_S(d, k, seed=1000 + s, m=m)
        G = S.T @ S
        assert np.allclose(np.diag(G), 1.0, atol=1e-15)
        acc += G
    off = acc / N - np.eye(m)
    bound = 5.0 * np.sqrt(1.0 / d) / np.sqrt(N)
    assert np.abs(off).max() < bound
