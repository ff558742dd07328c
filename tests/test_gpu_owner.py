"""Owner kernel (SK_KERNEL_OWNER): the chunked sketch in which every accumulator row has one owning
warp, so the on-chip FP32 partial sums take no atomics and receive their rows in ascending order.

Bars: a chunk processed as one work item (one chunk, one slice) is bit-exact with the oracle's
canonical order for every rule (paper Sec. 4.1-4.2 arithmetic, same chunk totals); larger shapes
(several chunks and slices, combined through FP32 atomics) are within the tolerance of the atomic
mode of the FP64 sketch; small-integer data is bit-exact at any chunking; the kernel refuses the
layouts it does not handle.
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
    R = plan.get(sk.SK_PARAM_LAST_CHUNK_ROWS)
    assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
    plan.close()
    return out, R


def _last_kernel(sk, A_h, d, k, dev, **params):
    import torch
    plan = sk.Plan(d, A_h.shape[0], k, 0, 1, **params)
    plan.apply(torch.from_numpy(np.ascontiguousarray(A_h)).to(dev))
    torch.cuda.synchronize()
    kern = plan.get(sk.SK_PARAM_LAST_KERNEL)
    plan.close()
    return kern


def _as64(Yn, rule):
    return Yn.astype(np.float64) if rule == 0 else oracle.bits16_to_f64(Yn, rule)


# One chunk of fewer than 2 * max(4096, 2d) rows is one work item per (pair of blocks, 32 columns):
# the FP32 chunk totals follow the rows in ascending order, exactly as the canonical definition.
@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("shape", [(16000, 64, 4096, 8), (8000, 40, 96, 3), (8100, 36, 512, 1),
                                   (8000, 128, 1024, 4), (4097, 32, 64, 16)])
def test_owner_one_item_per_chunk_is_canonical(sk, dev, rule, shape):
    m, n, d, k = shape
    A = inputs.host_matrix(m, n, "incoherent", seed=m + n)
    R = ((m + 31) // 32) * 32
    got, Rg = _run(sk, A, d, k, rule, 0xC0FFEE + k, dev, kernel=sk.SK_KERNEL_OWNER, chunk_rows=R)
    assert Rg == R
    if rule == 0:
        assert _last_kernel(sk, A, d, k, dev, kernel=sk.SK_KERNEL_OWNER) == sk.SK_KERNEL_OWNER
    ref = oracle.sketch_canonical(A, d, k, 0xC0FFEE + k, rule, R)
    assert np.array_equal(got, ref), np.count_nonzero(got != ref)


_F64 = {}


def _f64(A, d, k, seed):
    key = (A.shape, d, k, seed)
    if key not in _F64:
        _F64.clear()
        _F64[key] = oracle.sketch_f64(A, d, k, seed)
    return _F64[key]


@pytest.mark.parametrize("shape", [(1 << 20, 64, 4096, 8), (300001, 96, 2048, 4), (200003, 48, 1000, 5)])
@pytest.mark.parametrize("rule", RULES)
def test_owner_many_chunks_and_slices_within_tolerance(sk, dev, rule, shape):
    m, n, d, k = shape
    A = inputs.host_matrix(m, n, "incoherent", seed=7)
    got, R = _run(sk, A, d, k, rule, 99, dev, kernel=sk.SK_KERNEL_OWNER)
    Y64 = _f64(A, d, k, 99)
    assert oracle.rel_fro(_as64(got, rule), Y64) <= TOL[rule]
    # and the tile kernel on the same plan parameters agrees within the same bar
    tile, R2 = _run(sk, A, d, k, rule, 99, dev, kernel=sk.SK_KERNEL_TILE)
    assert R2 == R
    assert oracle.rel_fro(_as64(got, rule), _as64(tile, rule)) <= 2 * TOL[rule]


@pytest.mark.parametrize("shape", [(100003, 64, 4096, 8), (70001, 44, 768, 3), (50000, 32, 1024, 1)])
def test_owner_exact_on_integer_data(sk, dev, shape):
    # Small integers: every FP32 chunk total is exact whatever the slice combination order.
    m, n, d, k = shape
    A = np.random.default_rng(m).integers(-3, 4, size=(m, n)).astype(np.float32)
    scale_exact = k in (1, 4, 16)
    for rule in ([0, 1, 2] if scale_exact else RULES):
        R = 0 if scale_exact else ((m + 31) // 32) * 32
        params = {"kernel": sk.SK_KERNEL_OWNER}
        if R:
            params["chunk_rows"] = R
        got, Rg = _run(sk, A, d, k, rule, 5 + k, dev, **params)
        ref = oracle.sketch_canonical(A, d, k, 5 + k, rule, Rg)
        assert np.array_equal(got, ref), (rule, np.count_nonzero(got != ref))


def test_owner_refuses_unsupported_layouts(sk, dev):
    import torch
    # fewer than 32 columns
    plan = sk.Plan(256, 1000, 4, 0, 1, kernel=sk.SK_KERNEL_OWNER)
    with pytest.raises(sk.SkError) as e:
        plan.apply(torch.zeros((1000, 16), device=dev))
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    # row stride not a multiple of 16 bytes (no TMA)
    full = torch.zeros((1000, 34), device=dev)
    Y = torch.zeros((256, 33), device=dev)
    with pytest.raises(sk.SkError) as e:
        sk.sk_apply(plan.handle, full, 34, 33, Y)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    plan.close()
    # a block too large for two (or one) 32-column blocks in shared memory
    plan = sk.Plan(8192, 1000, 1, 0, 1, kernel=sk.SK_KERNEL_OWNER)
    with pytest.raises(sk.SkError):
        plan.apply(torch.zeros((1000, 64), device=dev))
    plan.close()
    torch.cuda.synchronize()


def test_auto_owner_and_tile_agree(sk, dev):
    # On small-integer data (exact arithmetic) AUTO (the register kernel at this shape), the owner
    # kernel and the tile kernel give the same bits, and the same as the oracle.
    m, n, d, k = 20000, 64, 512, 4
    A = np.random.default_rng(3).integers(-3, 4, size=(m, n)).astype(np.float32)
    auto, R = _run(sk, A, d, k, 1, 11, dev)
    assert _last_kernel(sk, A, d, k, dev) == sk.SK_KERNEL_REGISTER
    own, _ = _run(sk, A, d, k, 1, 11, dev, kernel=sk.SK_KERNEL_OWNER)
    tile, _ = _run(sk, A, d, k, 1, 11, dev, kernel=sk.SK_KERNEL_TILE)
    ref = oracle.sketch_canonical(A, d, k, 11, 1, R)
    assert np.array_equal(auto, ref) and np.array_equal(own, ref) and np.array_equal(tile, ref)
