"""GPU tests of the continuous-batching server (admission by slots and HBM budget, overlap on
streams, plan reuse) and of the autotuner, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2606_20195_gb300 import inputs

pytestmark = pytest.mark.gpu


def _stream(count, seed):
    from paper_2606_20195_gb300 import serve
    return serve.make_stream(count, rate_hz=2000.0, seed=seed, log2_m=(12, 16), ns=(16, 32), ks=(1, 4, 8))


def test_results_same_alone_and_in_the_mix(sk, dev):
    from paper_2606_20195_gb300 import serve
    reqs = _stream(16, seed=3)
    srv = serve.Server(slots=4, hbm_budget_bytes=2 * 10**9, deterministic=True)
    stats = srv.run(reqs)
    assert stats["ok"] == len(reqs)
    mixed = {r.rid: r.x.numpy().copy() for r in reqs}
    # each request again, alone, through the one-at-a-time path
    alone = _stream(16, seed=3)
    srv2 = serve.Server(slots=1, hbm_budget_bytes=2 * 10**9, deterministic=True)
    srv2.run_one_at_a_time(alone)
    for r in alone:
        a, b = mixed[r.rid], r.x.numpy()
        # deterministic sketches are bit-identical; the FP64 QR reduces with atomics, so x may
        # differ in the last bits only
        assert np.allclose(a, b, rtol=1e-6, atol=1e-7), r.rid
    srv.close()
    srv2.close()


def test_admission_respects_budget_and_slots(sk, dev):
    from paper_2606_20195_gb300 import serve
    reqs = _stream(24, seed=5)
    need = max(serve.footprint_bytes(r) + serve.plan_scratch_bytes(r) for r in reqs)
    budget = int(need * 2.5)  # at most two of the largest in flight
    srv = serve.Server(slots=8, hbm_budget_bytes=budget)
    stats = srv.run(reqs)
    assert stats["ok"] == len(reqs)
    assert srv.peak_bytes <= budget
    assert all(r.done >= r.admitted >= r.arrival for r in reqs)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    srv.close()


def test_server_solution_quality(sk, dev):
    # atomic mode: the served x solves the sketched problem as well as the oracle's sketch-and-solve
    import torch
    from paper_2606_20195_gb300 import serve
    r = serve.Request(rid=0, m=1 << 15, n=16, d=256, k=4, rule=0, family="incoherent", seed=42)
    srv = serve.Server(slots=2, hbm_budget_bytes=10**9)
    srv.run([r])
    assert r.status == sk.SK_OK
    A = inputs.device_matrix(r.m, r.n, r.family, seed=r.seed).cpu().numpy()
    g = torch.Generator(device="cuda:0")
    g.manual_seed(r.seed + 7)
    xs = torch.randn(r.n, generator=g, device="cuda:0")
    b = (torch.from_numpy(A).cuda() @ xs + 1e-6 * torch.randn(r.m, generator=g, device="cuda:0")).cpu().numpy()
    _, r_opt = oracle.lstsq_tall(A, b)
    ratio = oracle.residual_norm(A, b, r.x.numpy().astype(np.float64)) / r_opt
    assert 1.0 <= ratio < 2.0
    srv.close()


def test_autotune_plan_and_batch(sk, dev, tmp_path, monkeypatch):
    import torch
    from paper_2606_20195_gb300 import autotune
    monkeypatch.setenv("SK_TUNE_CACHE", str(tmp_path / "tune.json"))
    m, n, d, k = 1 << 16, 32, 512, 4
    A_h = inputs.host_matrix(m, n, "incoherent", seed=1)
    A = torch.from_numpy(A_h).to(dev)
    plan = sk.Plan(d, m, k, sk.SK_FP16_RN, 5)
    best = autotune.tune_plan(plan, A, reps=2)
    assert best["threads"] in autotune.THREADS
    Y = plan.apply(A)
    torch.cuda.synchronize()
    Y64 = oracle.sketch_f64(A_h, d, k, 5)
    assert oracle.rel_fro(oracle.halfbits_to_f64(Y.cpu().numpy().view(np.uint16)), Y64) <= 2e-3
    # cached on the second call
    assert autotune.tune_plan(plan, A)["ms"] == best["ms"]
    plan.close()
    items = []
    for i, (mm, nn, fam) in enumerate(inputs.batch_shapes(8, seed=2, log2_lo=10, log2_hi=14)):
        Ai = torch.from_numpy(inputs.host_matrix(mm, nn, fam, seed=i)).to(dev)
        items.append({"A": Ai, "Y": torch.empty((32 * nn, nn), dtype=torch.float16, device=dev), "m": mm, "n": nn,
                      "d": 32 * nn, "k": 4, "seed": i})
    b, params = autotune.tune_batch(items, sk.SK_FP16_RN, reps=1)
    sk.sk_batch_launch(b)
    torch.cuda.synchronize()
    for i, it in enumerate(items):
        ref = oracle.sketch_f64(it["A"].cpu().numpy(), it["d"], 4, i)
        assert oracle.rel_fro(oracle.halfbits_to_f64(it["Y"].cpu().numpy().view(np.uint16)), ref) <= 2e-3
    sk.sk_batch_destroy(b)
