"""GPU checks of bench.py's analysis helpers: the FP64 reference sketch it builds from the plan's
pattern (sk_materialize_S + torch index_add in FP64) equals the oracle's FP64 sketch, so the
relative errors the bench reports for each rule are against the right reference."""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [1, 3, 8])
def test_sketch_f64_reference_matches_oracle(sk, dev, k):
    import torch
    import bench
    m, n, d, seed = 50001, 24, 96 * k, 17
    A_h = inputs.host_matrix(m, n, "coherent", seed=5)
    plan = sk.Plan(d, m, k, 0, seed)
    Y64 = bench.sketch_f64_reference(plan.handle, torch.from_numpy(A_h).to(dev), d, k, chunk=1 << 14)
    plan.close()
    ref = oracle.sketch_f64(A_h, d, k, seed)
    assert np.allclose(Y64.cpu().numpy(), ref, rtol=1e-12, atol=1e-9)
