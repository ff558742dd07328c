"""Global-accumulator kernel (SK_KERNEL_GLOBAL): chunk totals accumulated in device memory with FP32
reductions (one warp per row), then added into Y in chunk order by the chunk-finish kernel. It serves
blocks of S too tall for the tile kernel's shared-memory accumulator, where AUTO falls back to it.

Bars: on small-integer data every chunk total is exact and Y is accumulated in canonical chunk order,
so the result is bit-exact with the oracle for every rule and chunking; on random data it is within
the atomic-mode tolerance of the FP64 sketch (paper Sec. 4.1-4.2 arithmetic).
"""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu

RULES = [0, 1, 2, 3, 4]  # FP32, the three FP16 rules and bfloat16 round-to-nearest
# bfloat16 (rule 4): the FP16 bar scaled by the ratio of unit roundoffs, 2^-9 / 2^-12 = 8 (reading 13)
TOL = {0: 1e-5, 1: 2e-3, 2: 2e-3, 3: 2e-3, 4: 1.6e-2}


def _run(sk, A_h, d, k, rule, seed, dev, **params):
    import torch
    A = torch.from_numpy(np.ascontiguousarray(A_h)).to(dev)
    plan = sk.Plan(d, A_h.shape[0], k, rule, seed, **params)
    Y = plan.apply(A)
    torch.cuda.synchronize()
    out = Y.cpu().numpy() if rule == 0 else Y.view(torch.int16).cpu().numpy().view(np.uint16)
    info = (plan.get(sk.SK_PARAM_LAST_CHUNK_ROWS), plan.get(sk.SK_PARAM_LAST_KERNEL))
    assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
    plan.close()
    return out, info


def _as64(Yn, rule):
    return Yn.astype(np.float64) if rule == 0 else oracle.bits16_to_f64(Yn, rule)


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("shape", [(20000, 64, 512, 8), (30011, 13, 96, 3), (50001, 1, 1024, 4),
                                   (9000, 130, 64, 64), (7, 5, 16, 2)])
def test_global_exact_on_integer_data(sk, dev, rule, shape):
    m, n, d, k = shape
    A = np.random.default_rng(m + n).integers(-3, 4, size=(m, n)).astype(np.float32)
    got, (R, kern) = _run(sk, A, d, k, rule, 77 + k, dev, kernel=sk.SK_KERNEL_GLOBAL, chunk_rows=2048)
    assert kern == sk.SK_KERNEL_GLOBAL and R == 2048
    ref = oracle.sketch_canonical(A, d, k, 77 + k, rule, R)
    assert np.array_equal(got, ref), np.count_nonzero(got != ref)


@pytest.mark.parametrize("rule", RULES)
def test_global_random_within_tolerance(sk, dev, rule):
    m, n, d, k = 100003, 48, 2048, 8
    A = inputs.host_matrix(m, n, "incoherent", seed=4)
    got, (R, kern) = _run(sk, A, d, k, rule, 5, dev, kernel=sk.SK_KERNEL_GLOBAL)
    assert kern == sk.SK_KERNEL_GLOBAL
    Y64 = oracle.sketch_f64(A, d, k, 5)
    assert oracle.rel_fro(_as64(got, rule), Y64) <= TOL[rule]


@pytest.mark.parametrize("rule", [0, 1])
def test_auto_falls_back_to_global_for_tall_blocks(sk, dev, rule):
    # B = d/k = 32768 rows: even one 4-column block of FP32 (512 KiB) exceeds shared memory.
    m, n, d, k = 20000, 8, 65536, 2
    A = inputs.host_matrix(m, n, "incoherent", seed=2)
    got, (R, kern) = _run(sk, A, d, k, rule, 9, dev)
    assert kern == sk.SK_KERNEL_GLOBAL
    Y64 = oracle.sketch_f64(A, d, k, 9)
    assert oracle.rel_fro(_as64(got, rule), Y64) <= TOL[rule]
    ref = oracle.sketch_canonical(A, d, k, 9, rule, R)
    assert oracle.rel_fro(_as64(got, rule), _as64(ref, rule)) <= TOL[rule]


def test_tile_slices_exact_on_integer_data_any_chunking(sk, dev):
    # The tile kernel's sliced chunks also reach Y through the chunk-finish kernel: on exact data the
    # result is canonical even with several chunks at k = 8 (irrational scale).
    m, n, d, k = 1 << 20, 64, 4096, 8
    A = np.random.default_rng(1).integers(-3, 4, size=(m, n)).astype(np.float32)
    for rule in RULES:
        got, (R, kern) = _run(sk, A, d, k, rule, 3, dev, kernel=sk.SK_KERNEL_TILE)
        assert kern == sk.SK_KERNEL_TILE
        ref = oracle.sketch_canonical(A, d, k, 3, rule, R)
        assert np.array_equal(got, ref), (rule, np.count_nonzero(got != ref))


# Chunk totals too large for L2 (chunks x d x n x 4 bytes above the pass budget of 40 MiB): the
# global kernel runs in passes of chunk batches and column slabs, each finished into Y in chunk order
# before the next. Small-integer data keeps every sum exact, so the result must equal the canonical
# order bit for bit, over slab boundaries (including a ragged last slab) and chunk batches.
@pytest.mark.parametrize("shape,R,rules", [
    ((20000, 256, 65536, 2), 0, [0, 1]),        # 64 MiB per chunk: one chunk per pass, slabs of 160 columns
    ((30000, 100, 16384, 4), 4096, [0, 1, 2]),   # 6.25 MiB per chunk: batches of 6 of the 8 chunks
    ((12000, 402, 32768, 8), 3000, [0, 1]),      # slabs of 320 and 82 columns (82 = 4*20 + 2: ragged quads)
])
def test_global_passes_exact_on_integer_data(sk, dev, shape, R, rules):
    m, n, d, k = shape
    A = np.random.default_rng(m + n).integers(-3, 4, size=(m, n)).astype(np.float32)
    for rule in rules:
        params = {"kernel": sk.SK_KERNEL_GLOBAL}
        if R:
            params["chunk_rows"] = R
        got, (Rg, kern) = _run(sk, A, d, k, rule, 99, dev, **params)
        assert kern == sk.SK_KERNEL_GLOBAL
        ref = oracle.sketch_canonical(A, d, k, 99, rule, Rg)
        assert np.array_equal(got, ref), (rule, np.count_nonzero(got != ref))


@pytest.mark.parametrize("k", [1, 2])
def test_auto_takes_global_for_wide_matrices_at_low_k(sk, dev, k):
    # n >= 256 with k <= 2: AUTO routes to the global kernel (the faster one there); on integer data
    # the result is canonical for every rule (chunk totals exact, finished in chunk order).
    m, n, d = 30000, 300, 600
    A = np.random.default_rng(k).integers(-3, 4, size=(m, n)).astype(np.float32)
    for rule in RULES:
        got, (R, kern) = _run(sk, A, d, k, rule, 5, dev)
        assert kern == sk.SK_KERNEL_GLOBAL
        ref = oracle.sketch_canonical(A, d, k, 5, rule, R)
        assert np.array_equal(got, ref), (rule, np.count_nonzero(got != ref))
