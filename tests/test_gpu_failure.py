"""Failure paths, made to happen without faulting, trapping or hanging the GPU.

- A bounded device wait that runs out: sk_solve's QR kernel synchronizes its CTAs with grid barriers
  whose waits are bounded (no asynchronous copies are in flight there). With the bound set to one
  SM clock cycle (SK_PARAM_SOLVE_WAIT_CYCLES) the first CTAs to arrive give up, the kernel ends, and
  sk_solve_status reports SK_ERR_TIMEOUT; the context stays usable and the next solve with the default
  bound is correct.
- A device allocation that is refused: with a scratch budget (SK_PARAM_SCRATCH_LIMIT) smaller than
  what the call needs, sk_apply returns SK_ERR_OOM before it enqueues anything (Y keeps its contents).
"""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_solve_barrier_timeout_is_reported_and_the_context_recovers(sk, dev):
    import torch
    m, n, d, k, seed = 1 << 16, 32, 2048, 8, 7
    A_h, b_h, _ = inputs.ls_problem_host(m, n, "incoherent", seed=3, noise=0.1)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    plan = sk.Plan(d, m, k, sk.SK_FP32, seed, solve_wait_cycles=1)
    x = plan.solve(A, b)
    status, _ = plan.solve_status()
    assert status == sk.SK_ERR_TIMEOUT
    assert "timed out" in sk.sk_last_error()
    # back to the default bound: the same plan solves correctly
    plan.set(sk.SK_PARAM_SOLVE_WAIT_CYCLES, 0)
    x = plan.solve(A, b)
    status, kappa = plan.solve_status()
    assert status == sk.SK_OK and kappa >= 1.0
    xo = oracle.sketch_solve(oracle.sketch_f64(A_h, d, k, seed), oracle.sketch_f64(b_h[:, None], d, k, seed)[:, 0])
    assert np.allclose(x.cpu().numpy(), xo, rtol=1e-3, atol=1e-4)
    plan.close()


def test_scratch_limit_refuses_before_enqueueing(sk, dev):
    import torch
    m, n, d, k = 1 << 18, 64, 4096, 8  # the register kernel: needs per-chunk totals in scratch
    A = inputs.device_matrix(m, n, "incoherent", seed=2)
    plan = sk.Plan(d, m, k, sk.SK_FP16_RN, 4, scratch_limit=64)
    Y = torch.full((d, n), 7.0, dtype=torch.float16, device=dev)
    with pytest.raises(sk.SkError) as e:
        plan.apply(A, Y)
    assert e.value.status == sk.SK_ERR_OOM and "limit" in str(e.value)
    torch.cuda.synchronize()
    assert bool((Y == 7.0).all()), "a refused call must leave Y untouched"
    assert plan.get(sk.SK_PARAM_SCRATCH_BYTES) <= 64
    # lifting the limit: the call goes through and the plan now holds the scratch it needed
    plan.set(sk.SK_PARAM_SCRATCH_LIMIT, 0)
    plan.apply(A, Y)
    torch.cuda.synchronize()
    assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
    assert plan.get(sk.SK_PARAM_SCRATCH_BYTES) > 64
    assert bool(torch.isfinite(Y.float()).all()) and float(Y.float().abs().max()) > 0
    plan.close()
