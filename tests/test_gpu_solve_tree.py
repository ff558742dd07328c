"""GPU tests of sk_solve's tree factorization (groups of rows factored separately, their [R | c]
factors stacked in FP64 and factored again): forced small groups (several levels, uneven groups)
and n = 1024 with a sketch taller than one launch holds, checked against the oracle's FP64
sketch-and-solve on the canonical sketch (deterministic mode: the sketch is bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle_solve(A_h, b_h, d, k, seed, rule, R):
    n = A_h.shape[1]
    Ab = np.hstack([A_h, b_h[:, None]])
    SAb = oracle.sketch_canonical(Ab, d, k, seed, rule, R)
    SAb = SAb.astype(np.float64) if rule == 0 else oracle.bits16_to_f64(SAb, rule)
    return oracle.sketch_solve(SAb[:, :n], SAb[:, n]), SAb


def _solve(sk, A, b, d, k, rule, seed, group_rows):
    plan = sk.Plan(d, A.shape[0], k, rule, seed, mode=sk.SK_MODE_DETERMINISTIC)
    plan.set(sk.SK_PARAM_SOLVE_GROUP_ROWS, group_rows)
    x = plan.solve(A, b)
    status, kappa = plan.solve_status()
    out = (x.cpu().numpy().astype(np.float64), status, kappa, plan.get(sk.SK_PARAM_LAST_LAUNCHES),
           plan.get(sk.SK_PARAM_LAST_CHUNK_ROWS))
    plan.close()
    return out


@pytest.mark.parametrize("rule", [0, 1, 4])
def test_tree_levels_match_oracle(sk, dev, rule):
    import torch
    m, n, d, k, seed = 1 << 16, 24, 1024, 8, 5
    A_h, b_h, _ = inputs.ls_problem_host(m, n, "incoherent", seed=21, noise=0.1)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    x1, st1, kap1, l1, R = _solve(sk, A, b, d, k, rule, seed, 0)
    assert st1 == sk.SK_OK
    x_or, SAb = _oracle_solve(A_h, b_h, d, k, seed, rule, R)
    s = np.linalg.svd(SAb[:, :n], compute_uv=False)
    # group rows 48 (= 2n): 22 groups of 46-47 rows, then 12, 6, 3 and 2 groups before the last
    # launch; 100 and 333: uneven groups, fewer levels; 5: raised to 2n.
    for g in (48, 100, 333, 5):
        x, st, kap, launches, _ = _solve(sk, A, b, d, k, rule, seed, g)
        assert st == sk.SK_OK
        assert launches > l1, (g, launches, l1)
        # the same FP64 least-squares problem: x agrees with the oracle to FP32 rounding
        assert np.max(np.abs(x - x_or)) <= 1e-6 * np.max(np.abs(x_or)), g
        # |R_ii| of the tree's R equal the single launch's up to FP64 rounding
        assert abs(kap - kap1) <= 1e-9 * kap1, (g, kap, kap1)
        assert 1.0 <= kap <= 1.01 * s[0] / s[-1]
    assert np.max(np.abs(x1 - x_or)) <= 1e-6 * np.max(np.abs(x_or))


@pytest.mark.parametrize("rule", [0, 1])
def test_solve_n1024_tall_sketch(sk, dev, rule):
    # n = 1024 (the paper's least-squares width); d = 8192 rows of 1025 FP64 values exceed the
    # shared memory of one launch, so the automatic tree takes two groups and a final launch.
    import torch
    m, n, d, k, seed = 1 << 15, 1024, 8192, 8, 9
    A_h, b_h, _ = inputs.ls_problem_host(m, n, "incoherent", seed=23, noise=0.1)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    x, st, kap, _, R = _solve(sk, A, b, d, k, rule, seed, 0)
    assert st == sk.SK_OK
    x_or, SAb = _oracle_solve(A_h, b_h, d, k, seed, rule, R)
    assert np.max(np.abs(x - x_or)) <= 1e-5 * np.max(np.abs(x_or))
    s = np.linalg.svd(SAb[:, :n], compute_uv=False)
    assert 1.0 <= kap <= 1.01 * s[0] / s[-1]


def test_solve_rejects_n_above_1024(sk, dev):
    import torch
    m, n = 4096, 1025
    A = torch.zeros((m, n), device=dev)
    b = torch.zeros(m, device=dev)
    plan = sk.Plan(2 * n + 2, m, 2, 0, 1)
    with pytest.raises(sk.SkError) as e:
        plan.solve(A, b)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    plan.close()


@pytest.mark.parametrize("rule", [0, 1])
def test_solve_n256_serving_shape(sk, dev, rule):
    # The largest request of the serving mix (n = 256, d = 16 n = 4096): one QR launch.
    import torch
    m, n, d, k, seed = 1 << 16, 256, 4096, 4, 13
    A_h, b_h, _ = inputs.ls_problem_host(m, n, "incoherent", seed=29, noise=0.1)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    x, st, kap, _, R = _solve(sk, A, b, d, k, rule, seed, 0)
    assert st == sk.SK_OK
    x_or, SAb = _oracle_solve(A_h, b_h, d, k, seed, rule, R)
    assert np.max(np.abs(x - x_or)) <= 1e-6 * np.max(np.abs(x_or))
    s = np.linalg.svd(SAb[:, :n], compute_uv=False)
    assert 1.0 <= kap <= 1.01 * s[0] / s[-1]
