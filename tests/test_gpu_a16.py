"""GPU parity of the 16-bit-A entry point (sk_apply_typed: binary16 or bfloat16 A, every value
converted exactly to FP32 as it is loaded) against the oracle run on the FP32 copy of A, through the
C ABI. The bars are those of the FP32 path: bit-exact in the deterministic and serial-tile modes and
on small-integer data in atomic mode; the FP32 path's tolerances otherwise."""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu

A_TYPES = ["fp16", "bf16"]
RULES5 = [0, 1, 2, 3, 4]
# bfloat16 (rule 4): the FP16 bar scaled by the ratio of unit roundoffs, 2^-9 / 2^-12 = 8 (reading 13)
TOL = {0: 1e-5, 1: 2e-3, 2: 2e-3, 3: 2e-3, 4: 1.6e-2}


def _to_np(Y, rule):
    import torch
    if rule == 0:
        return Y.cpu().numpy()
    return Y.view(torch.int16).cpu().numpy().view(np.uint16)


def _as64(Yn, rule):
    return Yn.astype(np.float64) if rule == 0 else oracle.bits16_to_f64(Yn, rule)


def _a16(A32, a_type, lda=None):
    """(16-bit device-ready host tensor with row stride lda, its exact FP32 values as numpy)."""
    import torch
    dt = torch.float16 if a_type == "fp16" else torch.bfloat16
    m, n = A32.shape
    lda = lda or n
    full = torch.zeros((m, lda), dtype=dt)
    full[:, :n] = torch.from_numpy(A32).to(dt)
    return full, full[:, :n].float().numpy()


def _apply16(sk, full16, n, d, k, rule, seed, dev, **params):
    import torch
    A = full16.to(dev)[:, :n]
    plan = sk.Plan(d, A.shape[0], k, rule, seed, **params)
    Y = plan.apply(A)
    torch.cuda.synchronize()
    out = _to_np(Y, rule)
    R = plan.get(sk.SK_PARAM_LAST_CHUNK_ROWS)
    kern = plan.get(sk.SK_PARAM_LAST_KERNEL)
    assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
    plan.close()
    return out, R, kern


@pytest.mark.parametrize("a_type", A_TYPES)
@pytest.mark.parametrize("rule", RULES5)
@pytest.mark.parametrize("lda", [13, 16])
def test_a16_deterministic_and_serial_bit_exact(sk, dev, a_type, rule, lda):
    # lda = 16: 32-byte rows, A staged through TMA in the serial tile kernel; lda = 13: direct loads.
    m, n, d, k, seed, R = 9000, 13, 256, 4, 5, 1000
    full, A32 = _a16(inputs.host_matrix(m, n, "incoherent", seed=1), a_type, lda)
    ref = oracle.sketch_canonical(A32, d, k, seed, rule, R)
    got, _, kern = _apply16(sk, full, n, d, k, rule, seed, dev, mode=sk.SK_MODE_DETERMINISTIC, chunk_rows=R)
    assert kern == 5 and np.array_equal(got, ref)
    for cols in (8, 16):
        got, _, kern = _apply16(sk, full, n, d, k, rule, seed, dev, mode=sk.SK_MODE_SERIAL_TILE, chunk_rows=R,
                                tile_cols=cols)
        assert kern == sk.SK_KERNEL_TILE and np.array_equal(got, ref), cols


# Small-integer data (exact in binary16 and bfloat16): chunk sums are exact, so atomic mode must equal
# the canonical order bit for bit (see the FP32 version of this test for the rule subsets).
@pytest.mark.parametrize("shape,R,rules,kernel", [
    ((50001, 64, 4096, 8), 50016, RULES5, "auto"),    # lane-row path, 16-bit TMA boxes of 8 columns
    ((50001, 64, 4096, 8), 50016, [0, 1], "global"),  # global-accumulator kernel (8-byte quad loads)
    ((50001, 12, 1024, 4), 0, [0, 1, 2], "auto"),     # lda 12: no 16-bit TMA (24-byte rows), direct loads
    ((50001, 16, 1024, 4), 0, [0, 1, 2], "auto"),
    ((30011, 24, 96, 3), 30016, RULES5, "auto"),      # odd k
    ((40000, 40, 512, 1), 0, [0, 1, 2], "auto"),      # CountSketch
    ((50001, 1, 1024, 4), 0, [0, 1, 2], "auto"),      # one column: the vector path
    ((20000, 8, 65536, 2), 0, [0, 1], "auto"),        # blocks too tall for shared memory: global kernel
])
@pytest.mark.parametrize("a_type", A_TYPES)
def test_a16_atomic_exact_on_integer_data(sk, dev, shape, R, rules, kernel, a_type):
    m, n, d, k = shape
    A = np.random.default_rng(m + k).integers(-3, 4, size=(m, n)).astype(np.float32)
    full, A32 = _a16(A, a_type)
    assert np.array_equal(A32, A)
    for rule in rules:
        params = {"chunk_rows": R} if R else {}
        if kernel == "global":
            params["kernel"] = sk.SK_KERNEL_GLOBAL
        got, Rg, kern = _apply16(sk, full, n, d, k, rule, 1234 + k, dev, **params)
        if kernel == "global" or d == 65536:
            assert kern == sk.SK_KERNEL_GLOBAL
        ref = oracle.sketch_canonical(A32, d, k, 1234 + k, rule, Rg)
        assert np.array_equal(got, ref), (rule, np.count_nonzero(got != ref))


@pytest.mark.parametrize("a_type", A_TYPES)
@pytest.mark.parametrize("rule", RULES5)
def test_a16_atomic_tolerance_and_fp32_path(sk, dev, a_type, rule):
    # Random values: atomic mode within the FP32 path's tolerance of the FP64 sketch of the FP32 copy,
    # and the deterministic mode equal to the FP32 entry point on that copy, bit for bit.
    import torch
    m, n, d, k, seed = 65537, 64, 4096, 8, 3
    full, A32 = _a16(inputs.host_matrix(m, n, "coherent", seed=7), a_type)
    got, R, _ = _apply16(sk, full, n, d, k, rule, seed, dev)
    Y64 = oracle.sketch_f64(A32, d, k, seed)
    assert oracle.rel_fro(_as64(got, rule), Y64) <= TOL[rule]
    det16, _, _ = _apply16(sk, full, n, d, k, rule, seed, dev, mode=sk.SK_MODE_DETERMINISTIC, chunk_rows=R)
    plan = sk.Plan(d, m, k, rule, seed, mode=sk.SK_MODE_DETERMINISTIC, chunk_rows=R)
    Y = plan.apply(torch.from_numpy(A32).to(dev))
    torch.cuda.synchronize()
    assert np.array_equal(det16, _to_np(Y, rule))
    plan.close()


@pytest.mark.parametrize("a_type", A_TYPES)
def test_a16_two_byte_aligned_view(sk, dev, a_type):
    # A view starting one element into a row: 2-byte aligned, not 4; accepted (direct loads).
    import torch
    m, n, d, k = 20000, 24, 512, 4
    full, _ = _a16(inputs.host_matrix(m, n + 1, "incoherent", seed=9), a_type)
    Ad = full.to(dev)[:, 1:]
    A32 = Ad.float().cpu().numpy()
    plan = sk.Plan(d, m, k, 0, 4)
    Y = plan.apply(Ad)
    torch.cuda.synchronize()
    assert oracle.rel_fro(Y.double().cpu().numpy(), oracle.sketch_f64(A32, d, k, 4)) <= TOL[0]
    plan.close()


def test_a16_rejections(sk, dev):
    import torch
    m, n, d, k = 4096, 32, 256, 2
    A = torch.zeros((m, n), dtype=torch.float16, device=dev)
    Y = torch.zeros((d, n), dtype=torch.float32, device=dev)
    plan = sk.Plan(d, m, k, 0, 1)
    with pytest.raises(sk.SkError) as e:
        sk.sk_apply_typed(plan.handle, A, 3, n, n, Y)
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    with pytest.raises(sk.SkError) as e:
        sk.sk_apply_typed(plan.handle, A.data_ptr() + 1, sk.SK_A_FP16, n, n, Y)
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    plan.set(sk.SK_PARAM_KERNEL, sk.SK_KERNEL_OWNER)
    with pytest.raises(sk.SkError) as e:
        plan.apply(A, Y)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    plan.close()
