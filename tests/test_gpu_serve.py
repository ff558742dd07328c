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
    srv = serve.Server(slots=4, hbm_budget_bytes=2 * 10**9, deterministic=True, keep_sketches=True)
    stats = srv.run(reqs)
    assert stats["ok"] == len(reqs)
    mixed = {r.rid: r.x.numpy().copy() for r in reqs}
    sketches = {r.rid: r.sketch for r in reqs}
    # each request again, alone, through the one-at-a-time path
    alone = _stream(16, seed=3)
    srv2 = serve.Server(slots=1, hbm_budget_bytes=2 * 10**9, deterministic=True, keep_sketches=True)
    srv2.run_one_at_a_time(alone)
    for r in alone:
        assert np.array_equal(sketches[r.rid], r.sketch), r.rid
        a, b = mixed[r.rid], r.x.numpy()
        # deterministic sketches are bit-identical; the FP64 QR reduces with atomics, so x may
        # differ in the last bits only
        assert np.allclose(a, b, rtol=1e-6, atol=1e-7), r.rid
    srv.close()
    srv2.close()


TOL = {0: 1e-5, 1: 2e-3, 2: 2e-3, 3: 2e-3}


def _sketch64(sk_host, rule):
    return sk_host.astype(np.float64) if rule == 0 else oracle.halfbits_to_f64(sk_host)


@pytest.mark.parametrize("batch_max_bytes", [1 << 40, 2 << 20])
def test_batched_results_same_alone_and_in_the_mix(sk, dev, batch_max_bytes):
    # Atomic mode, batched: the requests of a scheduling step are sketched by one batched launch per
    # rule. Each request's sketch [SA | Sb], in the mix and alone (a batch of one), is within the
    # atomic-mode tolerance of the FP64 sketch of its [A | b] (same S), the two sketches are within
    # that tolerance of each other, and each x is the least-squares solution of its own sketch (FP64
    # reference on the host, to FP32 output precision). The residual ||A x - b|| itself is not
    # compared: with b = A x* + 1e-6 noise the system is nearly consistent and the rounding of S b
    # (FP32 or binary16) already moves it by a few percent from one atomic order to another.
    # Run with every request batched, and with a 2 MiB limit, under which the larger requests take the
    # single-matrix path on streams of their own while the small ones are batched.
    from paper_2606_20195_gb300 import serve
    reqs = _stream(16, seed=4)
    for r in reqs:
        r.arrival = 0.0  # all at once: the first step batches as many as there are slots
    srv = serve.Server(slots=8, hbm_budget_bytes=2 * 10**9, keep_sketches=True)
    srv.BATCH_MAX_BYTES = batch_max_bytes
    big = [r for r in reqs if r.m * serve.ab_stride(r.n) * 4 > srv.BATCH_MAX_BYTES]
    assert (len(big) > 0) == (batch_max_bytes < (1 << 40))
    stats = srv.run(reqs)
    assert stats["ok"] == len(reqs)
    assert srv.launches < len(reqs) - len(big)  # some launch sketched several requests
    alone = _stream(16, seed=4)
    for r in alone:
        s1 = serve.Server(slots=1, hbm_budget_bytes=2 * 10**9, keep_sketches=True)
        s1.BATCH_MAX_BYTES = srv.BATCH_MAX_BYTES
        s1.run([r])
        assert r.status == sk.SK_OK and s1.launches == (0 if r.rid in {b.rid for b in big} else 1)
        s1.close()
    for rm, ra in zip(reqs, alone):
        A, b = srv.problem(rm)
        ref = oracle.sketch_f64(np.column_stack([A, b]).astype(np.float32), rm.d, rm.k,
                                serve.Server.sketch_seed(rm))
        ym, ya = _sketch64(rm.sketch, rm.rule), _sketch64(ra.sketch, ra.rule)
        assert oracle.rel_fro(ym, ref) <= TOL[rm.rule], rm.rid
        assert oracle.rel_fro(ya, ref) <= TOL[rm.rule], rm.rid
        assert oracle.rel_fro(ym, ya) <= TOL[rm.rule], rm.rid
        for r, y in ((rm, ym), (ra, ya)):
            xs = np.linalg.lstsq(y[:, :r.n], y[:, r.n], rcond=None)[0]
            assert np.allclose(r.x.numpy(), xs, rtol=1e-4, atol=1e-4 * np.abs(xs).max()), r.rid
    srv.close()


def test_solve_sketched_matches_solve(sk, dev):
    # sk_solve_sketched on the deterministic sketch [SA | Sb] gives the same x as sk_solve (the same
    # FP64 back end; the QR's reductions use atomics, so the last bits may differ).
    import torch
    m, n, d, k = 20000, 24, 384, 4
    A = inputs.host_matrix(m, n, "coherent", seed=3)
    b = inputs.host_vector(m, seed=4)
    Ad, bd = torch.from_numpy(A).to(dev), torch.from_numpy(b).to(dev)
    for rule in (0, 1):
        plan = sk.Plan(d, m, k, rule, 9, mode=sk.SK_MODE_DETERMINISTIC)
        x1 = plan.solve(Ad, bd)
        Ab = torch.from_numpy(np.column_stack([A, b]).astype(np.float32)).to(dev)
        Y = plan.apply(Ab)  # column n: S b with the rounding bits of column n, as sk_solve forms it
        x2 = torch.empty(n, dtype=torch.float32, device=dev)
        sk.sk_solve_sketched(plan.handle, Y, n + 1, n, x2)
        assert plan.solve_status()[0] == sk.SK_OK
        assert torch.allclose(x1, x2, rtol=1e-5, atol=1e-6)
        with pytest.raises(sk.SkError) as e:
            sk.sk_solve_sketched(plan.handle, Y, n, n, x2)  # ld < n + 1
        assert e.value.status == sk.SK_ERR_INVALID_ARG
        plan.close()


def test_batch_rebind_reuses_the_batch(sk, dev):
    # One batch object rebound to a second, larger set of items: results within tolerance of FP64
    # for both sets.
    import torch
    sets = [[(3000, 16), (5000, 32)], [(7000, 8), (2000, 64), (9000, 16)]]
    b = None
    for si, shapes in enumerate(sets):
        items = []
        for i, (mm, nn) in enumerate(shapes):
            Ai = torch.from_numpy(inputs.host_matrix(mm, nn, "incoherent", seed=10 * si + i)).to(dev)
            items.append({"A": Ai, "Y": torch.empty((16 * nn, nn), dtype=torch.float16, device=dev), "m": mm,
                          "n": nn, "d": 16 * nn, "k": 4, "seed": i})
        if b is None:
            b = sk.sk_batch_create(items, sk.SK_FP16_RN)
        else:
            sk.sk_batch_rebind(b, items)
            sk.sk_batch_set(b, sk.SK_PARAM_ITEM_CHUNKS, 2)
        sk.sk_batch_launch(b)
        torch.cuda.synchronize()
        for i, it in enumerate(items):
            ref = oracle.sketch_f64(it["A"].cpu().numpy(), it["d"], 4, i)
            assert oracle.rel_fro(oracle.halfbits_to_f64(it["Y"].cpu().numpy().view(np.uint16)), ref) <= 2e-3
    sk.sk_batch_destroy(b)


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
    A, b = srv.problem(r)
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


@pytest.mark.parametrize("rule", [0, 1, 2])
def test_batch_item_chunking_independent_of_the_batch(sk, dev, rule):
    # SK_PARAM_ITEM_CHUNKS: each item's chunk length comes from its own m, so on small-integer data
    # an item's sketch is the oracle's canonical sketch at that chunk length, bit for bit, alone and
    # beside other items. k is 1, 4 or 16, so the scale 1/sqrt(k) is a power of two: every chunk
    # total, its scaled value and every FP32 or binary16 sum of them is exact, whatever the order in
    # which the batched kernel's atomics add them. (Dither is left out: its noise, up to |x| 2^-11,
    # exceeds half an ulp for mantissas above 1, so it moves exact values off the integer grid and
    # the binary16 sums of the moved values then depend on the order of the atomics.)
    import torch
    shapes = [(50000, 24, 384, 4), (9000, 16, 256, 16), (130000, 8, 128, 1)]
    def run(which):
        items = []
        for i in which:
            m, n, d, k = shapes[i]
            A = np.random.default_rng(100 + i).integers(-3, 4, size=(m, n)).astype(np.float32)
            items.append((i, A, {"A": torch.from_numpy(A).to(dev), "m": m, "n": n, "d": d, "k": k, "seed": 40 + i,
                                 "Y": torch.empty((d, n), dtype=torch.float32 if rule == 0 else torch.float16,
                                                  device=dev)}))
        b = sk.sk_batch_create([it for _, _, it in items], rule)
        sk.sk_batch_set(b, sk.SK_PARAM_ITEM_CHUNKS, 8)
        sk.sk_batch_launch(b)
        torch.cuda.synchronize()
        out = {}
        for i, A, it in items:
            Yn = it["Y"].cpu().numpy()
            out[i] = (A, Yn if rule == 0 else Yn.view(np.uint16))
        sk.sk_batch_destroy(b)
        return out
    mixed = run([0, 1, 2])
    for i in range(3):
        alone = run([i])[i][1]
        A, got = mixed[i]
        m, n, d, k = shapes[i]
        R = max(4096, -(-m // 8))
        R = -(-R // 256) * 256
        ref = oracle.sketch_canonical(A, d, k, 40 + i, rule, R)
        assert np.array_equal(got, ref), (i, np.count_nonzero(got != ref))
        assert np.array_equal(alone, ref), i
