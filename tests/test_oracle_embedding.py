"""The sketch is a subspace embedding (paper Sec. 2.2): for an orthonormal basis Q of a 16-dimensional
subspace of R^16384, SparseStack with d = 256 and k = 4 keeps every singular value of S Q within
[1 - 0.5, 1 + 0.5] on at least 95 of 100 seeds, and its mean distortion is close to the Gaussian
sketch's sqrt(n / d) = 0.25. The accuracy parameter of the OSE bound is asymptotic in the paper; 0.5
is twice the Gaussian yardstick."""
import numpy as np

import oracle


def test_subspace_embedding_on_100_seeds():
    rng = np.random.default_rng(0)
    m, n, d, k = 16384, 16, 256, 4
    Q = np.linalg.qr(rng.standard_normal((m, n)))[0].astype(np.float32)
    # the float32 copy of Q is orthonormal to ~1e-7, far below the distortions measured here
    assert oracle.distortion(Q.astype(np.float64)) < 1e-5
    etas = np.array([oracle.distortion(oracle.sketch_f64(Q, d, k, seed)) for seed in range(100)])
    assert np.count_nonzero(etas <= 0.5) >= 95, np.sort(etas)[-10:]
    assert 0.15 <= etas.mean() <= 0.45, etas.mean()


def test_countsketch_collides_on_a_coordinate_basis():
    # k = 1 on the first n coordinate vectors: two of them share a target row with probability
    # 1 - prod(1 - i/d); then two columns of S Q coincide up to sign and sigma_min(SQ) = 0 (eta = 1).
    # SparseStack (k = 4) keeps sigma_min away from 0 on the same basis.
    m, n, d = 4096, 16, 64
    Q = np.zeros((m, n), dtype=np.float32)
    Q[np.arange(n), np.arange(n)] = 1.0
    eta_cs = [oracle.distortion(oracle.sketch_f64(Q, d, 1, s)) for s in range(50)]
    eta_ss = [oracle.distortion(oracle.sketch_f64(Q, d, 4, s)) for s in range(50)]
    p_collide = 1.0 - np.prod(1.0 - np.arange(n) / d)   # birthday bound, ~0.87 here
    assert np.mean(np.isclose(eta_cs, 1.0)) >= p_collide - 0.25
    assert max(eta_ss) < 1.0 - 1e-3
