"""Host-side checks of the measurement helpers of bench.py: the distortion eta(S, U) computed from
the Gram matrix (paper Sec. 5.1), directly or through the R factor of a general A, agrees with the
oracle's SVD-based distortion, and the coherence mu(U) (Sec. 5.2) has its closed-form extremes."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def test_eta_matches_oracle_svd():
    import bench
    rng = np.random.default_rng(1)
    m, n, d, k = 4000, 12, 96, 4
    U = np.linalg.qr(rng.standard_normal((m, n)))[0]
    S = oracle.dense_S(d, k, 3, m)
    SU = S @ U
    assert abs(bench.eta_of(torch.from_numpy(SU)) - oracle.distortion(SU)) <= 1e-12


def test_eta_general_matches_oracle():
    # eta of SA R^-1 for a general full-rank A, against the oracle's TSQR + solve + SVD
    import bench
    rng = np.random.default_rng(2)
    m, n, d, k = 5000, 10, 128, 4
    A = rng.standard_normal((m, n)) * np.linspace(1.0, 50.0, n)
    SA = oracle.dense_S(d, k, 5, m) @ A
    R_A = bench.r_factor_of(torch.from_numpy(A), chunk=1024)
    assert np.allclose(R_A.numpy(), oracle.tall_r_factor(A, chunk=1024), rtol=1e-10, atol=1e-10)
    got = bench.eta_general(torch.from_numpy(SA), R_A)
    assert abs(got - oracle.distortion_of(SA, oracle.tall_r_factor(A))) <= 1e-10


def test_coherence_extremes():
    import bench
    m, n = 1024, 8
    Qc = np.zeros((m, n))
    Qc[:n] = np.eye(n)
    assert bench.coherence_of(torch.from_numpy(Qc)) == pytest.approx(m / n)
    # a basis with every row of equal norm n/m has coherence 1
    H = np.kron(np.eye(n), np.ones((m // n, 1))) / np.sqrt(m // n)
    assert bench.coherence_of(torch.from_numpy(H)) == pytest.approx(1.0)
