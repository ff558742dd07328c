"""Register kernel (SK_KERNEL_REGISTER): FP32 chunk partials held in registers, rows of A routed to the
lanes that own their target rows through per-row lists in shared memory, then added into the chunk
totals and into Y in chunk order by the chunk-finish kernel (paper Sec. 4.1 scatter, Sec. 4.2 rounding).

Bars: on small-integer data every chunk total is exact, so the result is bit-exact with the oracle's
canonical order for every rule, whatever the summation order inside a chunk; on random data it is
within the atomic-mode tolerance of the FP64 sketch (1e-5 FP32, 2e-3 FP16 rules, 1.6e-2 bfloat16).
The shapes cover: several chunks and slices, ragged column tiles (n not a multiple of 32 or of 4),
block heights below, at and above the 1024 output rows of a work item (groups that hold several
blocks, part of a block, or parts of two), d below 1024, a row offset and a row stride, and forced
small list capacities so that the overflow path (full lists sent to the chunk totals by FP32 vector
reductions) carries most of the rows.
"""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu

RULES = [0, 1, 2, 3, 4]
# bfloat16 (rule 4): the FP16 bar scaled by the ratio of unit roundoffs, 2^-9 / 2^-12 = 8 (reading 13)
TOL = {0: 1e-5, 1: 2e-3, 2: 2e-3, 3: 2e-3, 4: 1.6e-2}


def _bits(Y, rule):
    import torch
    return Y.cpu().numpy() if rule == 0 else Y.view(torch.int16).cpu().numpy().view(np.uint16)


def _as64(Yn, rule):
    return Yn.astype(np.float64) if rule == 0 else oracle.bits16_to_f64(Yn, rule)


def _padded(A, dev):
    """A on the device with a row stride rounded up to a multiple of 4 floats (16 bytes), which the
    register kernel's TMA staging needs; the tensor is a column slice of the padded one."""
    import torch
    m, n = A.shape
    lda = (n + 3) // 4 * 4
    P = torch.zeros((m, lda), dtype=torch.float32, device=dev)
    P[:, :n] = torch.from_numpy(A).to(dev)
    return P[:, :n]


def _run(sk, A_dev, m, d, k, rule, seed, **params):
    import torch
    plan = sk.Plan(d, m, k, rule, seed, kernel=sk.SK_KERNEL_REGISTER, **params)
    Y = torch.full((d, A_dev.shape[1]), 7.0, dtype=plan.out_dtype(), device=A_dev.device)  # overwritten
    plan.apply(A_dev, Y)
    torch.cuda.synchronize()
    info = (plan.get(sk.SK_PARAM_LAST_KERNEL), plan.get(sk.SK_PARAM_LAST_CHUNK_ROWS))
    assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
    plan.close()
    return _bits(Y, rule), info


SHAPES = [
    # m, n, d, k, chunk rows, list capacity (0: automatic)
    (50001, 64, 4096, 8, 4096, 0),   # two column tiles, four groups of two blocks, 13 chunks
    (30011, 33, 2048, 4, 2048, 0),   # ragged second column tile (one column)
    (20000, 37, 3000, 3, 5000, 0),   # B = 1000: groups cut blocks; n % 4 != 0 (scalar reductions)
    (9000, 32, 8192, 2, 3000, 0),    # B = 4096: a group holds a quarter of a block
    (12000, 20, 256, 4, 4096, 0),    # d < 1024, B = 64 (long lists); n < 32
    (40000, 64, 4096, 8, 8192, 1),   # list capacity 1: most rows take the overflow path
    (40000, 48, 2048, 8, 2000, 3),   # capacity 3 at B = 256
    (60000, 64, 1024, 8, 8192, 0),   # B = 128: a group holds 8 blocks, long lists
]


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("shape", SHAPES)
def test_reg_exact_on_integer_data(sk, dev, rule, shape):
    m, n, d, k, R, cap = shape
    A = np.random.default_rng(m + n + d).integers(-3, 4, size=(m, n)).astype(np.float32)
    got, (kern, R_used) = _run(sk, _padded(A, dev), m, d, k, rule, 91 + k, chunk_rows=R, list_cap=cap)
    assert kern == sk.SK_KERNEL_REGISTER and R_used == R
    ref = oracle.sketch_canonical(A, d, k, 91 + k, rule, R)
    assert np.array_equal(got, ref), np.count_nonzero(got != ref)


@pytest.mark.parametrize("rule", RULES)
def test_reg_random_within_tolerance(sk, dev, rule):
    import torch
    m, n, d, k = 100003, 64, 4096, 8
    A = inputs.host_matrix(m, n, "incoherent", seed=21)
    got, (kern, _) = _run(sk, torch.from_numpy(A).to(dev), m, d, k, rule, 13)
    assert kern == sk.SK_KERNEL_REGISTER
    assert oracle.rel_fro(_as64(got, rule), oracle.sketch_f64(A, d, k, 13)) <= TOL[rule]


@pytest.mark.parametrize("family", ["coherent", "adversarial"])
@pytest.mark.parametrize("rule", [0, 1])
def test_reg_families_within_tolerance(sk, dev, family, rule):
    import torch
    m, n, d, k = 65536, 64, 2048, 8
    A = inputs.host_matrix(m, n, family, seed=5)
    got, _ = _run(sk, torch.from_numpy(A).to(dev), m, d, k, rule, 17)
    assert oracle.rel_fro(_as64(got, rule), oracle.sketch_f64(A, d, k, 17)) <= TOL[rule]


@pytest.mark.parametrize("rule", [0, 1, 2])
def test_reg_row_offset_and_stride(sk, dev, rule):
    # A is a column slice of a wider matrix (lda = 72) and its rows sit at global offset 77777, which
    # is not a multiple of the chunk length: S and the chunk grid follow the global row index.
    import torch
    m, n, lda, d, k, off, R = 30000, 64, 72, 2048, 4, 77777, 4096
    full = np.random.default_rng(3).integers(-3, 4, size=(m, lda)).astype(np.float32)
    A = torch.from_numpy(full).to(dev)[:, :n]
    got, (kern, _) = _run(sk, A, m, d, k, rule, 29, chunk_rows=R, row_offset=off)
    assert kern == sk.SK_KERNEL_REGISTER
    Af = np.zeros((off + m, n), dtype=np.float32)
    Af[off:] = full[:, :n]
    ref = oracle.sketch_canonical(Af, d, k, 29, rule, R)
    assert np.array_equal(got, ref), np.count_nonzero(got != ref)


def test_reg_matches_tile_kernel(sk, dev):
    # Same plan, two kernels: both within FP32 rounding of each other on random data.
    import torch
    m, n, d, k = 200000, 64, 4096, 8
    A = inputs.device_matrix(m, n, "incoherent", seed=8)
    outs = []
    for kern in (sk.SK_KERNEL_REGISTER, sk.SK_KERNEL_TILE):
        plan = sk.Plan(d, m, k, sk.SK_FP32, 3, kernel=kern)
        Y = plan.apply(A)
        torch.cuda.synchronize()
        assert plan.get(sk.SK_PARAM_LAST_KERNEL) == kern
        outs.append(Y.double().cpu().numpy())
        plan.close()
    assert oracle.rel_fro(outs[0], outs[1]) <= 2e-6


def test_reg_auto_choice(sk, dev):
    # AUTO takes the register kernel for FP32 A with k >= 2, n >= 32 and B <= 512, and not for k = 1,
    # n < 32 or taller blocks.
    import torch
    for (n, d, k, want) in ((64, 1024, 8, sk.SK_KERNEL_REGISTER), (64, 4096, 8, sk.SK_KERNEL_REGISTER),
                            (64, 1024, 1, None), (16, 1024, 4, None), (64, 4096, 2, None)):
        A = torch.zeros((5000, n), device=dev)
        plan = sk.Plan(d, 5000, k, 1, 0)
        plan.apply(A)
        torch.cuda.synchronize()
        got = plan.get(sk.SK_PARAM_LAST_KERNEL)
        assert (got == want) if want is not None else (got != sk.SK_KERNEL_REGISTER)
        plan.close()


def test_reg_unsupported_layouts(sk, dev):
    # Forced register kernel: 16-bit A and a row stride that is not a multiple of 16 bytes are refused.
    import torch
    plan = sk.Plan(1024, 1000, 4, 1, 0, kernel=sk.SK_KERNEL_REGISTER)
    A16 = torch.zeros((1000, 64), dtype=torch.float16, device=dev)
    with pytest.raises(sk.SkError) as e:
        plan.apply(A16)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    wide = torch.zeros((1000, 67), device=dev)
    with pytest.raises(sk.SkError) as e:
        plan.apply(wide[:, :64])
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    plan.close()
