"""Distortion parity (paper Sec. 5.1): for a general full-rank A = Q R_A, eta(S, Q) of the GPU sketch
(atomic mode) equals the oracle's FP64 eta for the same S within 2 %, and every 16-bit rule's eta is
within 2 % of the FP32 rule's (the paper's "equal distortion")."""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu

RULES5 = [0, 1, 2, 3, 4]


@pytest.mark.parametrize("family", ["incoherent", "coherent"])
def test_gpu_eta_matches_oracle_and_rules_agree(sk, dev, family):
    import torch
    m, n, d, k, seed = 1 << 17, 16, 512, 4, 21
    A = inputs.host_matrix(m, n, family, seed=3) * np.linspace(1.0, 20.0, n, dtype=np.float32)
    R_A = oracle.tall_r_factor(A)
    eta_or = oracle.distortion_of(oracle.sketch_f64(A, d, k, seed), R_A)
    At = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    etas = {}
    for rule in RULES5:
        plan = sk.Plan(d, m, k, rule, seed)
        Y = plan.apply(At)
        etas[rule] = oracle.distortion_of(Y.double().cpu().numpy(), R_A)
        plan.close()
    assert abs(etas[0] - eta_or) <= 0.02 * eta_or, (etas[0], eta_or)
    for rule in RULES5[1:]:
        assert abs(etas[rule] - etas[0]) <= 0.02 * etas[0], (rule, etas[rule], etas[0])
