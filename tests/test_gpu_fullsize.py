"""Parity at the benchmark's own sizes (paper Sec. 4.1-4.2 arithmetic; Sec. 5.1 sketch-and-solve).

1. The single-matrix sweep shape exactly as bench.py times it (m = 2^22, n = 64, d = 4096, k = 8, the
   kernel AUTO picks), for the three input families and seeds 0, 1, 2, every rule: relative Frobenius
   error against the FP64 sketch within 1e-5 (FP32), 2e-3 (FP16 rules), 1.6e-2 (bfloat16). The FP64
   sketch is built on the GPU from the plan's pattern (pinned against the oracle elsewhere); here its
   values are also checked against the CPU oracle itself on sampled outputs of every matrix.
2. Sketch-and-solve at the least-squares workload's shape with 2^23 rows (n = 128, d = 2048, k = 8,
   coherent family, b = A x* + 1e-6 N(0,1)): the deterministic mode's sketch is bit-identical to the
   oracle's canonical sketch, and the residual of the GPU's x is within 2 % of the residual of the x the
   oracle's FP64 QR gives from that sketch. 2^23 rows (4 GB of A) instead of 2^24 keeps the host-side
   generation and the oracle's canonical sketch within about a minute on the test host.
"""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu

RULES = [0, 1, 2, 3, 4]
TOL = {0: 1e-5, 1: 2e-3, 2: 2e-3, 3: 2e-3, 4: 1.6e-2}


@pytest.mark.parametrize("family", inputs.FAMILIES)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sweep_shape_every_rule_within_tolerance(sk, dev, family, seed):
    import torch
    import bench
    m, n, d, k = bench.WORKLOADS["sweep_m4M_n64_d4096_k8"]
    A_h = inputs.host_matrix(m, n, family, seed=seed)
    A = torch.from_numpy(A_h).to(dev)
    sk_seed = 1234 + seed
    plan = sk.Plan(d, m, k, sk.SK_FP32, sk_seed)
    Y64 = bench.sketch_f64_reference(plan.handle, A, d, k)
    plan.close()
    # the FP64 reference against the CPU oracle on sampled outputs (every row scan is m hashes)
    rng = np.random.default_rng(seed)
    rs = rng.integers(0, d, size=24)
    cs = rng.integers(0, n, size=24)
    o64, _ = oracle.sketch_sampled(A_h, d, k, sk_seed, 0, 1 << 19, rs, cs)
    assert np.allclose(Y64.cpu().numpy()[rs, cs], o64, rtol=1e-12, atol=1e-9)
    nrm = float(torch.linalg.norm(Y64))
    for rule in RULES:
        plan = sk.Plan(d, m, k, rule, sk_seed)
        Y = plan.apply(A)
        torch.cuda.synchronize()
        assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
        plan.close()
        err = float(torch.linalg.norm(Y.double() - Y64)) / nrm
        assert err <= TOL[rule], (family, seed, rule, err)


def test_sketch_and_solve_deterministic_at_2_23_rows(sk, dev):
    import torch
    m, n, d, k, seed, R = 1 << 23, 128, 2048, 8, 77, 1 << 20
    A_h, b_h, _ = inputs.ls_problem_host(m, n, "coherent", seed=9, noise=1e-6)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    rule = sk.SK_FP16_RN
    plan = sk.Plan(d, m, k, rule, seed, mode=sk.SK_MODE_DETERMINISTIC, chunk_rows=R)
    x = plan.solve(A, b)
    status, _ = plan.solve_status()
    assert status == sk.SK_OK
    # the same sketch of [A | b] as the oracle's canonical order, bit for bit
    Y = plan.apply(A)
    torch.cuda.synchronize()
    got = Y.view(torch.int16).cpu().numpy().view(np.uint16)
    Ab = np.empty((m, n + 1), dtype=np.float32)
    Ab[:, :n] = A_h
    Ab[:, n] = b_h
    canon = oracle.sketch_canonical(Ab, d, k, seed, rule, R)
    assert np.array_equal(got, canon[:, :n])
    plan.close()
    # the oracle's x from that sketch (FP64 QR), and both residuals on the full problem
    SAb = oracle.bits16_to_f64(canon, rule)
    x_or = oracle.sketch_solve(SAb[:, :n], SAb[:, n])
    r_gpu = oracle.residual_norm(A_h, b_h, x.cpu().numpy().astype(np.float64))
    r_or = oracle.residual_norm(A_h, b_h, x_or)
    assert abs(r_gpu / r_or - 1.0) <= 0.02, (r_gpu, r_or)
