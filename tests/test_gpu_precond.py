"""Sketch-and-precondition least squares (sk_solve_precond): LSQR on A with the right preconditioner
R^{-1} from the FP64 QR of the sketch S A. The paper's discussion names this use of the sketch beside
sketch-and-solve (Sec. 5.1); the operator A R^{-1} is well conditioned whatever the sketch's rounding
rule, so the iteration reaches the FP64 least-squares solution of A itself.

Bars: residual ratio ||A x - b|| / ||A x* - b|| within 1e-6 of 1 against the oracle's FP64 TSQR
solution x*, ||x - x*|| / ||x*|| <= 1e-7, for every rule including the FP16 and BF16 sketches whose
sketch-and-solve ratio is far above 1 on the coherent problem; a handful of iterations.
"""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rule", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("family,noise", [("coherent", 1e-6), ("incoherent", 0.1)])
def test_precond_reaches_fp64_least_squares(sk, dev, rule, family, noise):
    import torch
    m, n, d, k = 1 << 18, 32, 512, 8
    A_h, b_h, _ = inputs.ls_problem_host(m, n, family, seed=21, noise=noise)
    x_opt, r_opt = oracle.lstsq_tall(A_h, b_h)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    plan = sk.Plan(d, m, k, rule, 5)
    x, it = plan.solve_precond(A, b, tol=1e-12)
    torch.cuda.synchronize()
    xg = x.cpu().numpy()
    ratio = oracle.residual_norm(A_h, b_h, xg) / r_opt
    assert abs(ratio - 1.0) <= 1e-6, (ratio, it)
    assert np.linalg.norm(xg - x_opt) <= 1e-7 * np.linalg.norm(x_opt), it
    assert 1 <= it <= 60
    # the sketch-and-solve starting point is much worse on the coherent problem with 16-bit rules
    x0 = plan.solve(A, b).cpu().numpy().astype(np.float64)
    assert oracle.residual_norm(A_h, b_h, x0) / r_opt >= ratio - 1e-12
    plan.close()


def test_precond_ragged_shapes(sk, dev):
    import torch
    for (m, n, d, k) in [(5000, 7, 64, 4), (70001, 100, 1026, 3)]:
        A_h, b_h, _ = inputs.ls_problem_host(m, n, "incoherent", seed=m, noise=0.5)
        x_opt, r_opt = oracle.lstsq_tall(A_h, b_h)
        plan = sk.Plan(d, m, k, 1, 9)
        x, it = plan.solve_precond(torch.from_numpy(A_h).to(dev), torch.from_numpy(b_h).to(dev), tol=1e-12)
        xg = x.cpu().numpy()
        assert abs(oracle.residual_norm(A_h, b_h, xg) / r_opt - 1.0) <= 1e-8
        assert np.linalg.norm(xg - x_opt) <= 1e-7 * np.linalg.norm(x_opt)
        plan.close()


def test_precond_rank_deficient_is_reported(sk, dev):
    import torch
    m, n, d, k = 4096, 8, 64, 4
    A = torch.zeros((m, n), device=dev)
    A[:, 0] = 1.0
    b = torch.ones(m, device=dev)
    plan = sk.Plan(d, m, k, 0, 1)
    with pytest.raises(sk.SkError) as e:
        plan.solve_precond(A, b)
    assert e.value.status == sk.SK_ERR_NUMERIC
    plan.close()
