"""Row-sharded sketches through the product path (sk_apply_partials / sk_finish_partials): two plans
over disjoint global row ranges of one matrix, split at a row that is not a multiple of the chunk
length, add their FP32 chunk totals into separate buffers; the buffers are summed on the device (the
all-reduce of a multi-GPU run, emulated on one GPU) and finished into Y.

Bars (paper Sec. 4.1 scatter, Sec. 4.2 rounding after the sum): on small-integer data the chunk
totals are exact and the finish adds them in chunk order, so the sharded result is bit-exact with the
oracle's canonical order for every rule and for the register, tile and owner kernels (and with one
sk_apply of the register kernel over the whole matrix); on random data it is within the atomic-mode
tolerance of the FP64 sketch.
"""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu

RULES = [0, 1, 2, 3, 4]
TOL = {0: 1e-5, 1: 2e-3, 2: 2e-3, 3: 2e-3, 4: 1.6e-2}


def _bits(Y, rule):
    import torch
    return Y.cpu().numpy() if rule == 0 else Y.view(torch.int16).cpu().numpy().view(np.uint16)


def _sharded(sk, A, splits, d, k, rule, seed, R, **params):
    """Y of the matrix A (device) from shards [splits[i], splits[i+1]) via partials summed on the device."""
    import torch
    m, n = A.shape
    nchunks = (m + R - 1) // R
    total = torch.zeros((nchunks, d, n), dtype=torch.float32, device=A.device)
    kernels = []
    for lo, hi in zip(splits[:-1], splits[1:]):
        plan = sk.Plan(d, hi - lo, k, rule, seed, row_offset=lo, chunk_rows=R, **params)
        P = torch.zeros_like(total)
        sk.sk_apply_partials(plan.handle, A[lo:hi], A.stride(0), n, P, 0, nchunks)
        torch.cuda.synchronize()
        assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
        kernels.append(plan.get(sk.SK_PARAM_LAST_KERNEL))
        total += P  # the all-reduce (sum) of the shards' FP32 chunk totals
        plan.close()
    plan = sk.Plan(d, m, k, rule, seed, chunk_rows=R)
    Y = torch.full((d, n), 3.0, dtype=plan.out_dtype(), device=A.device)
    sk.sk_finish_partials(plan.handle, total, 0, nchunks, n, Y)
    torch.cuda.synchronize()
    assert float(total.abs().max()) == 0.0  # cleared by the finish
    plan.close()
    return _bits(Y, rule), kernels


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("kernel", ["auto", "tile", "owner"])
def test_two_shards_exact_on_integer_data(sk, dev, rule, kernel):
    import torch
    m, n, d, k, R, seed = 50001, 64, 4096, 8, 4096, 31
    A_h = np.random.default_rng(5).integers(-3, 4, size=(m, n)).astype(np.float32)
    A = torch.from_numpy(A_h).to(dev)
    params = {} if kernel == "auto" else {"kernel": sk.SK_KERNEL_TILE if kernel == "tile" else sk.SK_KERNEL_OWNER}
    got, kernels = _sharded(sk, A, [0, 23457, m], d, k, rule, seed, R, **params)
    want = {"auto": sk.SK_KERNEL_REGISTER, "tile": sk.SK_KERNEL_TILE, "owner": sk.SK_KERNEL_OWNER}[kernel]
    assert all(kk == want for kk in kernels), kernels
    ref = oracle.sketch_canonical(A_h, d, k, seed, rule, R)
    assert np.array_equal(got, ref), np.count_nonzero(got != ref)
    if kernel == "auto":
        # the same as one sk_apply over the whole matrix with the register kernel, which also
        # finishes its chunk totals in chunk order (the tile and owner kernels add a chunk that is one
        # work item straight into Y, in whatever order the chunks finish)
        plan = sk.Plan(d, m, k, rule, seed, chunk_rows=R, **params)
        Y1 = plan.apply(A)
        torch.cuda.synchronize()
        assert np.array_equal(got, _bits(Y1, rule))
        plan.close()


@pytest.mark.parametrize("rule", [0, 1, 2])
def test_three_uneven_shards_random_within_tolerance(sk, dev, rule):
    import torch
    m, n, d, k, R, seed = 200003, 48, 2048, 4, 16384, 8
    A_h = inputs.host_matrix(m, n, "incoherent", seed=12)
    A = torch.from_numpy(A_h).to(dev)
    got, _ = _sharded(sk, A, [0, 777, 123457, m], d, k, rule, seed, R)
    Y = got.astype(np.float64) if rule == 0 else oracle.bits16_to_f64(got, rule)
    assert oracle.rel_fro(Y, oracle.sketch_f64(A_h, d, k, seed)) <= TOL[rule]


def test_partials_argument_checks(sk, dev):
    import torch
    A = torch.zeros((1000, 64), device=dev)
    P = torch.zeros((4, 1024, 64), device=dev)
    plan = sk.Plan(1024, 1000, 4, 0, 1)  # chunk rows not set
    with pytest.raises(sk.SkError) as e:
        sk.sk_apply_partials(plan.handle, A, 64, 64, P, 0, 4)
    assert e.value.status == sk.SK_ERR_INVALID_ARG and "CHUNK_ROWS" in str(e.value)
    plan.close()
    plan = sk.Plan(1024, 1000, 4, 0, 1, chunk_rows=256, row_offset=512)  # chunks 2..5
    with pytest.raises(sk.SkError) as e:
        sk.sk_apply_partials(plan.handle, A, 64, 64, P, 0, 4)  # P holds chunks 0..3 only
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    sk.sk_apply_partials(plan.handle, A, 64, 64, P, 2, 4)  # P holds chunks 2..5: accepted
    torch.cuda.synchronize()
    plan.close()
