"""GPU tests of the host-buffer pipeline, FP64 sketch-and-solve (paper Sec. 5.1) and the batched
persistent launch with CUDA-graph replay, all through the C ABI, checked against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 2e-3, 2: 2e-3, 3: 2e-3}


def _as64(Y, rule):
    Yn = Y.cpu().numpy() if hasattr(Y, "cpu") else Y
    return Yn.astype(np.float64) if rule == 0 else oracle.halfbits_to_f64(Yn.view(np.uint16))


@pytest.mark.parametrize("rule", [0, 1, 2, 3])
@pytest.mark.parametrize("pinned", [True, False])
def test_apply_host_matches_device_path(sk, dev, rule, pinned):
    import torch
    m, n, d, k = 300_001, 24, 512, 8
    A_h = inputs.host_matrix(m, n, "incoherent", seed=5)
    A_t = torch.from_numpy(A_h)
    if pinned:
        A_t = A_t.pin_memory()
    dt = torch.float32 if rule == 0 else torch.float16
    Y_h = torch.empty((d, n), dtype=dt)
    if pinned:
        Y_h = Y_h.pin_memory()
    # deterministic mode: the tiled host pipeline gives the canonical result bit for bit
    plan = sk.Plan(d, m, k, rule, 3, mode=sk.SK_MODE_DETERMINISTIC, chunk_rows=65536)
    sk.sk_apply_host(plan.handle, A_t.data_ptr(), n, n, Y_h.data_ptr())
    ref = oracle.sketch_canonical(A_h, d, k, 3, rule, 65536)
    got = Y_h.numpy() if rule == 0 else Y_h.numpy().view(np.uint16)
    assert np.array_equal(got, ref)
    plan.close()
    # atomic mode: within tolerance of FP64
    plan = sk.Plan(d, m, k, rule, 3)
    sk.sk_apply_host(plan.handle, A_t.data_ptr(), n, n, Y_h.data_ptr())
    Y64 = oracle.sketch_f64(A_h, d, k, 3)
    assert oracle.rel_fro(_as64(Y_h, rule), Y64) <= TOL[rule]
    plan.close()


@pytest.mark.parametrize("rule", [0, 1, 2, 3, 4])
def test_sketch_and_solve_matches_oracle(sk, dev, rule):
    import torch
    m, n, d, k = 1 << 18, 32, 512, 8
    A_h, b_h, x_star = inputs.ls_problem_host(m, n, "coherent", seed=7, noise=1e-6)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    x_opt, r_opt = oracle.lstsq_tall(A_h, b_h)
    for mode in (sk.SK_MODE_DETERMINISTIC, sk.SK_MODE_ATOMIC):
        plan = sk.Plan(d, m, k, rule, 11, mode=mode)
        x = plan.solve(A, b)
        status, kappa = plan.solve_status()
        assert status == sk.SK_OK
        R = plan.get(sk.SK_PARAM_LAST_CHUNK_ROWS)
        x_gpu = x.cpu().numpy().astype(np.float64)
        # oracle sketch-and-solve from the canonical sketch of [A | b] with the same chunking
        Ab = np.hstack([A_h, b_h[:, None]])
        SAb = oracle.sketch_canonical(Ab, d, k, 11, rule, R)
        SAb = SAb.astype(np.float64) if rule == 0 else oracle.bits16_to_f64(SAb, rule)
        x_or = oracle.sketch_solve(SAb[:, :n], SAb[:, n])
        ratio_gpu = oracle.residual_norm(A_h, b_h, x_gpu) / r_opt
        ratio_or = oracle.residual_norm(A_h, b_h, x_or) / r_opt
        # Deterministic mode sketches bit for bit like the oracle: the 2% bar. In atomic mode the
        # rounding errors of SA (FP16 ~1e-3, FP32 ~6e-8 relative to entries of 1e3) dominate the
        # 1e-6 noise of b, so the ratio is a random variable of the summation order; that mode is
        # held to the 2% bar on the noisier problem below.
        if mode == sk.SK_MODE_DETERMINISTIC:
            assert abs(ratio_gpu - ratio_or) <= 0.02 * ratio_or, (mode, ratio_gpu, ratio_or)
        # kappa(SA): the diagonal estimate is a lower bound on the 2-norm condition number
        s = np.linalg.svd(SAb[:, :n], compute_uv=False)
        assert 1.0 <= kappa <= 1.01 * s[0] / s[-1]
        plan.close()


@pytest.mark.parametrize("rule", [0, 1, 2, 3, 4])
def test_sketch_and_solve_atomic_mode_noisy_problem(sk, dev, rule):
    # b = A x* + 0.1 N(0,1) with incoherent A: the residual ratio measures the sketch, not rounding.
    import torch
    m, n, d, k = 1 << 18, 32, 512, 8
    A_h, b_h, _ = inputs.ls_problem_host(m, n, "incoherent", seed=9, noise=0.1)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    _, r_opt = oracle.lstsq_tall(A_h, b_h)
    plan = sk.Plan(d, m, k, rule, 13)
    x = plan.solve(A, b)
    assert plan.solve_status()[0] == sk.SK_OK
    R = plan.get(sk.SK_PARAM_LAST_CHUNK_ROWS)
    Ab = np.hstack([A_h, b_h[:, None]])
    SAb = oracle.sketch_canonical(Ab, d, k, 13, rule, R)
    SAb = SAb.astype(np.float64) if rule == 0 else oracle.bits16_to_f64(SAb, rule)
    x_or = oracle.sketch_solve(SAb[:, :n], SAb[:, n])
    ratio_gpu = oracle.residual_norm(A_h, b_h, x.cpu().numpy().astype(np.float64)) / r_opt
    ratio_or = oracle.residual_norm(A_h, b_h, x_or) / r_opt
    assert abs(ratio_gpu - ratio_or) <= 0.02 * ratio_or, (ratio_gpu, ratio_or)
    assert 1.0 <= ratio_gpu < 1.2
    plan.close()


def test_solve_rank_deficient_reports_numeric(sk, dev):
    import torch
    m, n, d, k = 4096, 8, 64, 4
    A = torch.zeros((m, n), device=dev)
    A[:, 0] = 1.0
    b = torch.ones(m, device=dev)
    plan = sk.Plan(d, m, k, 0, 1)
    plan.solve(A, b)
    status, _ = plan.solve_status()
    assert status == sk.SK_ERR_NUMERIC
    plan.close()


def _batch_inputs(count, seed, dev):
    import torch
    shapes = inputs.batch_shapes(count, seed=seed, log2_lo=10, log2_hi=15, ns=(8, 16, 32, 64, 128))
    items, hosts = [], []
    for i, (m, n, fam) in enumerate(shapes):
        A_h = inputs.host_matrix(m, n, fam, seed=100 + i)
        A = torch.from_numpy(A_h).to(dev)
        d = 32 * n
        items.append({"A": A, "m": m, "n": n, "d": d, "k": 4, "seed": 1000 + i})
        hosts.append(A_h)
    return items, hosts


@pytest.mark.parametrize("rule", [0, 1])
def test_batch_matches_oracle_and_graph_replay(sk, dev, rule):
    import torch
    items, hosts = _batch_inputs(24, 3, dev)
    dt = torch.float32 if rule == 0 else torch.float16
    for it in items:
        it["Y"] = torch.full((it["d"], it["n"]), 7.0, dtype=dt, device=dev)  # launch must zero Y
    b = sk.sk_batch_create(items, rule)
    nwork, nbytes = sk.sk_batch_info(b)
    assert nwork >= len(items) and nbytes == sum(4 * it["m"] * it["n"] for it in items)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        sk.sk_batch_launch(b, stream)
    stream.synchronize()
    refs = [oracle.sketch_f64(h, it["d"], it["k"], it["seed"]) for h, it in zip(hosts, items)]
    for it, ref in zip(items, refs):
        assert oracle.rel_fro(_as64(it["Y"], rule), ref) <= TOL[rule]
    # capture the launch in a CUDA graph and replay it: same results (within tolerance)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        sk.sk_batch_launch(b, torch.cuda.current_stream(dev))
    for it in items:
        it["Y"].fill_(3.0)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for it, ref in zip(items, refs):
        assert oracle.rel_fro(_as64(it["Y"], rule), ref) <= TOL[rule]
    sk.sk_batch_destroy(b)


def test_batch_rejects_invalid_items(sk, dev):
    import torch
    A = torch.zeros((100, 8), device=dev)
    Y = torch.zeros((64, 8), device=dev)
    with pytest.raises(sk.SkError):
        sk.sk_batch_create([{"A": A, "Y": Y, "m": 100, "n": 8, "d": 63, "k": 4}], 0)
    with pytest.raises(sk.SkError):
        sk.sk_batch_create([{"A": A, "Y": Y, "m": 100, "n": 8, "lda": 4, "d": 64, "k": 4}], 0)
    with pytest.raises(sk.SkError):
        sk.sk_batch_create([], 0)
