"""sk_apply_noalloc, the sketch entry point for callers that cannot allocate device memory (code
running inside an allocator callback, services with a fixed device-memory footprint, applications
that own all device memory): its kernel's scratch is a fixed static device array of the library.

Checked through the C ABI against the regular sk_apply on the same plan, on two calls in a row,
within the tolerances the other tests use, and the device's free memory must not move across those
calls. This file is collected last so that a run stopping at the first failure has already run every
other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 2e-3, 2: 2e-3, 3: 2e-3}


def _as64(Y, rule):
    Yn = Y.cpu().numpy()
    return Yn.astype(np.float64) if rule == 0 else oracle.halfbits_to_f64(Yn.view(np.uint16))


@pytest.mark.parametrize("rule", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(16384, 16, 256, 4), (1 << 20, 64, 4096, 8), (50001, 13, 96, 3)])
def test_noalloc_matches_sk_apply_twice(sk, dev, rule, shape):
    import torch
    m, n, d, k = shape
    A_h = inputs.host_matrix(m, n, "incoherent", seed=m % 97)
    A = torch.from_numpy(A_h).to(dev)
    plan = sk.Plan(d, m, k, rule, 21)
    dt = torch.float32 if rule == 0 else torch.float16
    Y_ref = torch.empty((d, n), dtype=dt, device=dev)
    sk.sk_apply(plan.handle, A, n, n, Y_ref)
    torch.cuda.synchronize()
    apply_launches = plan.get(sk.SK_PARAM_LAST_LAUNCHES)
    ref = _as64(Y_ref, rule)
    Y64 = oracle.sketch_f64(A_h, d, k, 21)
    assert oracle.rel_fro(ref, Y64) <= TOL[rule]
    Y1 = torch.full((d, n), 5.0, dtype=dt, device=dev)
    Y2 = torch.full((d, n), -3.0, dtype=dt, device=dev)
    sk.sk_apply_noalloc(plan.handle, A, n, n, Y1)  # first call on the device: its code may load here
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info(dev)
    sk.sk_apply_noalloc(plan.handle, A, n, n, Y1)
    sk.sk_apply_noalloc(plan.handle, A, n, n, Y2)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info(dev)
    assert free_after == free_before, "sk_apply_noalloc changed the device's free memory"
    for Y in (Y1, Y2):
        got = _as64(Y, rule)
        # same kernel and chunking as sk_apply: equal up to the atomic summation order
        assert oracle.rel_fro(got, ref) <= TOL[rule]
        assert oracle.rel_fro(got, Y64) <= TOL[rule]
    assert plan.get(sk.SK_PARAM_LAST_LAUNCHES) == apply_launches
    # the no-allocation call's status word (in the static array) is readable and clear
    assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
    plan.close()


def test_noalloc_rejects_oversize_and_other_modes(sk, dev):
    import torch
    # chunks x d x n x 4 bytes of chunk totals (8 x 8192 x 64 x 4 = 16.8 MB) above the 16 MiB array:
    # rejected with a message, nothing enqueued
    m, n, d, k = 1 << 20, 64, 8192, 8
    plan = sk.Plan(d, m, k, 0, 1)
    A = torch.zeros((m, n), device=dev)
    Y = torch.zeros((d, n), device=dev)
    with pytest.raises(sk.SkError) as e:
        sk.sk_apply_noalloc(plan.handle, A, n, n, Y)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED and "static" in str(e.value)
    plan.close()
    plan = sk.Plan(256, 1000, 4, 0, 1, mode=sk.SK_MODE_DETERMINISTIC)
    A = torch.zeros((1000, 8), device=dev)
    Y = torch.zeros((256, 8), device=dev)
    with pytest.raises(sk.SkError):
        sk.sk_apply_noalloc(plan.handle, A, 8, 8, Y)
    plan.close()
    torch.cuda.synchronize()
