"""Benchmark of the SparseStack sketch Y = S A on GB300 (one JSON line on rank 0).

Workload (default): the single-matrix sweep configuration m = 2^22, n = 64, d = 4096, k = 8,
A FP32 iid N(0, 1) (the incoherent family), accumulation FP16 round-to-nearest (the headline rule);
FP32 / stochastic / dithered / bfloat16 variants are timed beside it. A is 1 GiB, larger than the 129 MB L2,
so no L2 flush is needed between steps. One step = one sk_apply (zero Y, the kernel AUTO picks: the
register kernel at this shape, and the chunk-finish kernel).

  value      device throughput, GB/s of (A read + Y written) with A resident in HBM
  e2e        the same metric through sk_apply_host with pinned host buffers (H2D of A and D2H of
             Y inside the timed region)
  roofline   the dominant kernel against the measured HBM copy bandwidth
  cpu_baseline  the CPU oracle (canonical FP16-RN sketch) on a bounded row sample, host cores

Extras (default: serve, solve, batch): the batched uneven launch (256 matrices, one CUDA-graph
replay), sketch-and-solve at 2^24 x 128, and the serving stream (reduced m range over 1000 requests,
the full m range up to 2^24 over 200, and a saturated run with every request arriving at once).

--impl reference times the oracle itself (the reference arm of this comparison) on the same
workload, each step a bounded row sample. Under torchrun (N > 1) every rank sketches its own
matrix (independent problems, weak scaling, no collective on the data path), or, with --shard rows,
the ranks share one matrix split by rows: each adds its FP32 chunk totals (sk_apply_partials), one
NCCL all-reduce sums them and every rank finishes Y (sk_finish_partials) (strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

WORKLOADS = {
    # name: (m, n, d, k)
    "sweep_m4M_n64_d4096_k8": (1 << 22, 64, 4096, 8),
    "small_m16384_n16_d256_k4": (16384, 16, 256, 4),
    # same kernel shape at a quarter of the rows: the ncu capture case (256 MiB of A, > L2)
    "profile_m1M_n64_d4096_k8": (1 << 20, 64, 4096, 8),
    # CountSketch at the sweep shape (k = 1: the tile kernel, one block per row)
    "countsketch_m4M_n64_d4096_k1": (1 << 22, 64, 4096, 1),
    # CountSketch on a wide matrix (the paper's n = 1024 at d/n = 2; AUTO: global-accumulator kernel)
    "countsketch_m2M_n1024_d2048_k1": (1 << 21, 1024, 2048, 1),
    # the same at an eighth of the rows (1 GiB of A): its ncu capture case
    "profile_m256K_n1024_d2048_k1": (1 << 18, 1024, 2048, 1),
}
DEFAULT_WORKLOAD = "sweep_m4M_n64_d4096_k8"
METRIC = "SA sketch HBM GB/s (% of peak) FP16 vs FP32 at equal distortion; p99 solve ms"
KERNEL_SOURCES = ["paper_2606_20195_gb300/csrc/sk_tile.cuh", "paper_2606_20195_gb300/csrc/sk_tile_kernel.cuh",
                  "paper_2606_20195_gb300/csrc/sk_kernels.cu",
                  "paper_2606_20195_gb300/csrc/sk_own.cu",
                  "paper_2606_20195_gb300/csrc/sk_reg.cu",
                  "paper_2606_20195_gb300/csrc/sk_device.cuh"]


def default_chunk_rows(m: int) -> int:
    """The library's default chunk length for an m-row matrix (at most 8 chunks, at least 4096 rows,
    a multiple of 32): the row shards of one matrix must all use it."""
    R = max(4096, (m + 7) // 8)
    return (R + 31) // 32 * 32


def y_dtype(rule: int):
    """torch dtype of Y for a rule: float32, binary16, or bfloat16 (rule 4)."""
    import torch
    return torch.float32 if rule == 0 else (torch.bfloat16 if rule == 4 else torch.float16)


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(HERE, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def traffic_record(kernel: str, workload: str, rule: str):
    """DRAM traffic per launch from the committed ncu summary, if it was taken on these sources."""
    p = os.path.join(HERE, "profiles", f"{kernel}_{workload}_{rule}_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    with open(p) as f:
        for ln in f:
            if "=" in ln and not ln.startswith("#"):
                a, b = ln.split("=", 1)
                kv[a.strip()] = b.strip()
    if kv.get("kernel_sources_sha256_16") != kernel_hash():
        return None
    try:
        return float(kv["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index: int = 0):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"sk_clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for ln in f:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    maxs.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_rate(m_total: int, n: int, d: int, k: int, budget_s: float, seed: int = 0):
    """Oracle canonical FP16-RN sketch on a row sample; returns (GB/s, cores, sample description)."""
    import oracle
    from paper_2606_20195_gb300 import inputs
    rows = min(m_total, 1 << 20)
    A = inputs.host_matrix(rows, n, "incoherent", seed=seed)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.sketch_canonical(A, d, k, seed, oracle.FP16_RN, max(1, rows // 32))
        reps += 1
        if time.perf_counter() - t0 >= budget_s or reps >= 20:
            break
    dt = (time.perf_counter() - t0) / reps
    gbps = (rows * n * 4 + d * n * 2) / dt / 1e9
    sample = f"{rows} of {m_total} rows (n={n}, d={d}, k={k}), canonical FP16-RN, {reps} reps"
    return gbps, oracle.num_threads(), sample


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    m, n, d, k = WORKLOADS[args.workload]
    import oracle
    from paper_2606_20195_gb300 import inputs
    rows = min(m, 1 << 20)
    A = inputs.host_matrix(rows, n, "incoherent", seed=0)
    R = max(1, rows // 32)
    for _ in range(args.warmup):
        oracle.sketch_canonical(A, d, k, 0, oracle.FP16_RN, R)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sketch_canonical(A, d, k, 0, oracle.FP16_RN, R)
    dt = (time.perf_counter() - t0) / args.steps
    gbps = (rows * n * 4 + d * n * 2) / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbps, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f16", "data": "synthetic",
        "config": {"workload": args.workload, "m": m, "n": n, "d": d, "k": k, "rule": "fp16_rn",
                   "sample_rows": rows},
        "cpu_baseline": {"value": gbps, "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{rows} of {m} rows per step, canonical FP16-RN"},
        "e2e": {"value": gbps, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_solve(dev, rules=(0, 1, 2, 3, 4), m=1 << 24, n=128, d=2048, k=8, reps=3):
    """Sketch-and-solve and sketch-and-precondition (LSQR with the sketch's R) at the coherent
    least-squares shape: phase times, iterations and residual ratios."""
    import torch
    from paper_2606_20195_gb300 import inputs, sk
    A = inputs.device_matrix(m, n, "coherent", seed=3, device=str(dev))
    g = torch.Generator(device=dev)
    g.manual_seed(4)
    xs = torch.randn(n, generator=g, device=dev, dtype=torch.float64)
    b = (A.double() @ xs + 1e-6 * torch.randn(m, generator=g, device=dev, dtype=torch.float64)).float()
    # FP64 least-squares optimum for the ratio (torch on the GPU, reporting only)
    Rr = torch.linalg.qr(torch.cat([A.double(), b.double()[:, None]], dim=1), mode="r").R
    r_opt = float(abs(Rr[n, n]))
    out = {}
    for rule in rules:
        plan = sk.Plan(d, m, k, rule, seed=11)
        x = torch.empty(n, dtype=torch.float32, device=dev)
        Y = torch.empty((d, n), dtype=plan.out_dtype(), device=dev)
        for _ in range(2):
            plan.solve(A, b, x)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ts, tk = [], []
        for _ in range(reps):
            ev[0].record()
            plan.solve(A, b, x)
            ev[1].record()
            plan.apply(A, Y)
            ev[2].record()
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
            tk.append(ev[1].elapsed_time(ev[2]))
        status, kappa = plan.solve_status()
        res = float(torch.linalg.vector_norm(A.double() @ x.double() - b.double()))
        # sketch-and-precondition on the same plan (one warm run, then timed)
        xp, its = plan.solve_precond(A, b, tol=1e-12)
        torch.cuda.synchronize()
        ev[0].record()
        xp, its = plan.solve_precond(A, b, tol=1e-12)
        ev[1].record()
        torch.cuda.synchronize()
        res_p = float(torch.linalg.vector_norm(A.double() @ xp - b.double()))
        out[list(sk.RULES)[rule]] = {"solve_ms": statistics.median(ts), "sketch_A_ms": statistics.median(tk),
                                     "qr_and_Sb_ms": statistics.median(ts) - statistics.median(tk),
                                     "residual_ratio": res / r_opt, "kappa_SA_diag_estimate": kappa,
                                     "status": status,
                                     "precond": {"ms": ev[0].elapsed_time(ev[1]), "iterations": its,
                                                 "residual_ratio": res_p / r_opt}}
        plan.close()
    del A, b
    torch.cuda.empty_cache()
    return {"workload": f"coherent LS m={m} n={n} d={d} k={k}", **out}


def eta_of(SU) -> float:
    """Distortion eta(S, U) = max(|sigma_max(SU) - 1|, |1 - sigma_min(SU)|) of a sketched orthonormal
    basis (paper Sec. 5.1), from the eigenvalues of the n x n Gram matrix (SU)^T (SU) in FP64."""
    import torch
    X = SU.double()
    ev = torch.linalg.eigvalsh(X.T @ X).clamp_min(0.0).sqrt()
    return float(max(abs(float(ev[-1]) - 1.0), abs(1.0 - float(ev[0]))))


def r_factor_of(A, chunk: int = 1 << 18):
    """R factor (n x n, FP64, diag > 0) of a tall matrix A = Q R by stacked chunk QRs (torch, on A's
    device)."""
    import torch
    Rs = [torch.linalg.qr(A[i0:i0 + chunk].double(), mode="r").R for i0 in range(0, A.shape[0], chunk)]
    R = torch.linalg.qr(torch.cat(Rs), mode="r").R
    sgn = torch.sign(torch.diagonal(R))
    sgn[sgn == 0] = 1.0
    return R * sgn[:, None]


def eta_general(SA, R_A) -> float:
    """eta(S, Q) for a full-rank A = Q R_A from its sketch: eta of SA R_A^-1 (paper Sec. 5.1)."""
    import torch
    SQ = torch.linalg.solve_triangular(R_A.T, SA.double().T, upper=False).T
    return eta_of(SQ)


def coherence_of(U) -> float:
    """mu(U) = (m/n) max_i ||U_i,:||^2 (paper Sec. 5.2, coherence sweep)."""
    m, n = U.shape
    return float((U.double() ** 2).sum(dim=1).max()) * m / n


# nonzeros per column of SparseStack in the paper's experiments (Sec. 5, "unless otherwise stated")
ZETA = 4


def bench_paper(dev, m=1 << 21, n=1024, ratios=(2, 4, 8, 16, 32, 64, 128, 256),
                sweep_ratios=(2, 4, 8, 16), alphas=(0.0, 0.3, 0.6, 0.8, 0.9, 0.95, 1.0), reps=3):
    """The paper's sketching experiments on synthetic inputs (Sec. 5.1-5.2): distortion eta and
    throughput over the sketch ratio d/n for a Gaussian and an identity-like orthonormal basis
    U (m x n), and the coherence sweep U(alpha) = orth((1 - alpha) Q_rand + alpha [I; 0]).
    SparseStack (k = 4, the paper's default) with every rounding rule and CountSketch (k = 1); U itself
    is the sketched matrix (its GB/s is the throughput); throughput also at m = 2^19 and 2^20. Inputs
    are built with torch (FP32 QR), not by the library."""
    import torch
    from paper_2606_20195_gb300 import sk
    torch.backends.cuda.matmul.allow_tf32 = False
    g = torch.Generator(device=dev)
    g.manual_seed(2606)
    methods = [("sparsestack", ZETA, r) for r in ("fp32", "fp16_rn", "fp16_sr", "fp16_dither", "bf16_rn")]
    methods += [("countsketch", 1, "fp32"), ("countsketch", 1, "fp16_rn")]

    def sketch(U, d, k, rule_name, timed=False):
        rv = sk.RULES[rule_name]
        plan = sk.Plan(d, U.shape[0], k, rv, seed=77)
        Y = torch.empty((d, U.shape[1]), dtype=y_dtype(rv), device=dev)
        ms = None
        if timed:
            for _ in range(2):
                plan.apply(U, Y)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                plan.apply(U, Y)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        else:
            plan.apply(U, Y)
        plan.close()
        return Y.float(), ms

    out = {"workload": f"n={n} m={m}, d/n in {list(ratios)}; SparseStack k={ZETA}, CountSketch k=1", "extremes": {}}
    Qg = torch.linalg.qr(torch.randn((m, n), generator=g, device=dev)).Q.contiguous()
    Qc = torch.zeros((m, n), device=dev)
    Qc[:n] = torch.eye(n, device=dev)
    for fam, U in (("gaussian", Qg), ("identity", Qc)):
        res = {}
        for name, k, rname in methods:
            key = f"{name}_{rname}"
            etas, gbs = [], []
            for r in ratios:
                d = r * n
                Y, ms = sketch(U, d, k, rname, timed=(fam == "gaussian"))
                etas.append(eta_of(Y))
                es = 4 if rname == "fp32" else 2
                gbs.append((m * n * 4 + d * n * es) / (ms * 1e-3) / 1e9 if ms else None)
                del Y
            res[key] = {"eta": etas, "GB/s": gbs} if fam == "gaussian" else {"eta": etas}
        res["gaussian_reference_sqrt_n_over_d"] = [float(np.sqrt(1.0 / r)) for r in ratios]
        out["extremes"][fam] = res
    # coherence sweep
    sweep = {"alpha": list(alphas), "mu": [], "d_over_n": list(sweep_ratios)}
    sweep_methods = [mt for mt in methods if mt[2] in ("fp32", "fp16_rn", "fp16_sr", "fp16_dither") and
                     (mt[0] == "sparsestack" or mt[2] == "fp32")]
    for name, k, rname in sweep_methods:
        sweep[f"{name}_{rname}"] = {str(r): [] for r in sweep_ratios}
    for a in alphas:
        U = torch.linalg.qr((1.0 - a) * Qg + a * Qc).Q.contiguous()
        sweep["mu"].append(coherence_of(U))
        for name, k, rname in sweep_methods:
            for r in sweep_ratios:
                Y, _ = sketch(U, r * n, k, rname)
                sweep[f"{name}_{rname}"][str(r)].append(eta_of(Y))
                del Y
        del U
    out["coherence_sweep"] = sweep
    # throughput at the paper's other leading dimensions (rows of the Gaussian basis)
    tp = {}
    for mm in (1 << 19, 1 << 20):
        Um = Qg[:mm].contiguous()
        row = {}
        for name, k, rname in methods:
            if rname not in ("fp32", "fp16_rn"):
                continue
            gbs = []
            for r in ratios:
                d = r * n
                plan = sk.Plan(d, mm, k, sk.RULES[rname], seed=77)
                Y = torch.empty((d, n), dtype=y_dtype(sk.RULES[rname]), device=dev)
                for _ in range(2):
                    plan.apply(Um, Y)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(reps):
                    plan.apply(Um, Y)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                es = 4 if rname == "fp32" else 2
                gbs.append((mm * n * 4 + d * n * es) / (ms * 1e-3) / 1e9)
                plan.close()
                del Y
            row[f"{name}_{rname}"] = gbs
        tp[str(mm)] = row
        del Um
    out["throughput_GBps_by_m"] = tp
    del Qg, Qc
    torch.cuda.empty_cache()
    return out


def bench_paper_ls(dev, m=1 << 21, n=1024, ratios=(2, 4, 8, 16, 24), reps=2):
    """The paper's sketch-and-solve least-squares families (Sec. 5.3) on synthetic inputs: dense
    A = U Sigma V^T (singular values 100 -> 1, b = A 1 + noise; "easy": noise 1e-3 N(0,1), "hard":
    noise 1e-1 N(0,1) plus an offset of 1e-1) and the coherent permuted [I_n; tau G / sqrt(m-n)]
    (tau = 1e-3, noise 0.5 on the identity block). Per sketch ratio and method: sk_solve time,
    relative residual ||Ax - b|| / ||b|| and kappa(SA) (FP64 Gram eigenvalues of the sketch).
    The least-squares optimum (FP64 QR of [A | b] by torch) is the normal-equations reference.
    On the coherent problem the paper's per-element FP16 scheme (R = 1, literal kernel) also runs."""
    import torch
    from paper_2606_20195_gb300 import inputs, sk
    methods = [("sparsestack", ZETA, r) for r in ("fp32", "fp16_rn", "fp16_sr", "fp16_dither", "bf16_rn")]
    methods += [("countsketch", 1, "fp32"), ("countsketch", 1, "fp16_rn")]
    step = 1 << 18

    def rel_res(A, b, x):
        x64 = x.double()
        acc = 0.0
        for i0 in range(0, A.shape[0], step):
            r = A[i0:i0 + step].double() @ x64 - b[i0:i0 + step].double()
            acc += float(r @ r)
        return (acc ** 0.5) / float(torch.linalg.vector_norm(b.double()))

    def optimum(A, b):
        Rs = []
        for i0 in range(0, A.shape[0], step):
            blk = torch.cat([A[i0:i0 + step].double(), b[i0:i0 + step].double()[:, None]], dim=1)
            Rs.append(torch.linalg.qr(blk, mode="r").R)
        R = torch.linalg.qr(torch.cat(Rs), mode="r").R
        return float(abs(R[n, n])) / float(torch.linalg.vector_norm(b.double()))

    def problems():
        torch.backends.cuda.matmul.allow_tf32 = False
        for fam in ("dense_easy", "dense_hard", "coherent_permuted"):
            A, b = inputs.paper_ls_problem(fam, m, n, seed=5303, device=str(dev))
            yield fam, A, b
            del A, b

    out = {"workload": f"m={m} n={n}, d/n in {list(ratios)}; SparseStack k={ZETA}, CountSketch k=1", "families": {}}
    for name, A, b in problems():
        fam = {"optimum_rel_res": optimum(A, b)}
        for r in ratios:
            d = r * n
            row = {}
            # the paper's per-element scheme (R = 1, one FP16 atomic per contribution) beside the
            # chunked one, on the coherent problem at the two smallest ratios
            # and the whole column pre-combined in FP32 before one binary16 rounding (one chunk)
            extra = ([("sparsestack_literal", ZETA, "fp16_rn"), ("sparsestack_onechunk", ZETA, "fp16_rn")]
                     if name.startswith("coherent") and r <= 4 else [])
            for meth, k, rname in methods + extra:
                params = ({"kernel": sk.SK_KERNEL_LITERAL, "chunk_rows": 1} if meth.endswith("literal")
                          else {"chunk_rows": m} if meth.endswith("onechunk") else {})
                plan = sk.Plan(d, m, k, sk.RULES[rname], seed=31, **params)
                x = plan.solve(A, b)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ts = []
                for _ in range(reps):
                    e0.record()
                    plan.solve(A, b, x)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                status, kd = plan.solve_status()
                launches = plan.get(sk.SK_PARAM_LAST_LAUNCHES)
                Y = torch.empty((d, n), dtype=y_dtype(sk.RULES[rname]), device=dev)
                e0.record()
                plan.apply(A, Y)
                e1.record()
                torch.cuda.synchronize()
                X = Y.double()
                ev = torch.linalg.eigvalsh(X.T @ X).clamp_min(0.0)
                kap = float((ev[-1] / ev[0]) ** 0.5) if float(ev[0]) > 0 else float("inf")
                row[f"{meth}_{rname}"] = {"ms": statistics.median(ts), "sketch_A_ms": e0.elapsed_time(e1),
                                          "rel_res": rel_res(A, b, x), "kappa_SA": kap, "kappa_diag_estimate": kd,
                                          "status": status, "solve_launches": launches}
                del Y, X
                plan.close()
            fam[str(r)] = row
        out["families"][name] = fam
        del A, b
        torch.cuda.empty_cache()
    return out


def sketch_f64_reference(plan_h, A, d: int, k: int, chunk: int = 1 << 17):
    """FP64 S A from the plan's nonzero pattern (sk_materialize_S, pinned bit-exact against the
    oracle by the tests) and torch index_add in FP64: the reference for the relative error."""
    import torch
    from paper_2606_20195_gb300 import sk
    m, n = A.shape
    Y = torch.zeros((d, n), dtype=torch.float64, device=A.device)
    rows = torch.empty(chunk * k, dtype=torch.int32, device=A.device)
    signs = torch.empty(chunk * k, dtype=torch.int8, device=A.device)
    scale = 1.0 / float(np.sqrt(k))
    for i0 in range(0, m, chunk):
        c = min(chunk, m - i0)
        sk.sk_materialize_S(plan_h, i0, c, rows, signs)
        r = rows[:c * k].long()
        v = A[i0:i0 + c].double().repeat_interleave(k, dim=0) * (signs[:c * k].double() * scale)[:, None]
        Y.index_add_(0, r, v)
    return Y


def bench_families(dev, m, n, d, k, seed=1234):
    """The sweep shape on the three input families (iid N(0,1), coherent 1e3 I block over an N(0, 1e-6)
    tail, adversarial row i = g_i e_(i mod n)): FP16-RN and FP32 GB/s, relative Frobenius error of
    every rule against the FP64 sketch, and eta of FP16-RN against FP32 (same S)."""
    import torch
    from paper_2606_20195_gb300 import inputs, sk
    out = {}
    for fam in ("incoherent", "coherent", "adversarial"):
        A = inputs.device_matrix(m, n, fam, seed=7, device=str(dev))
        row = {}
        ys = {}
        for name, rv in sk.RULES.items():
            plan = sk.Plan(d, m, k, rv, seed=seed)
            Y = torch.empty((d, n), dtype=y_dtype(rv), device=dev)
            plan.apply(A, Y)
            if name in ("fp32", "fp16_rn"):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(3):
                    plan.apply(A, Y)
                e1.record()
                torch.cuda.synchronize()
                es = 4 if rv == 0 else 2
                row[f"GB/s_{name}"] = (m * n * 4 + d * n * es) / (e0.elapsed_time(e1) / 3 * 1e-3) / 1e9
            if name == "fp32":
                Y64 = sketch_f64_reference(plan.handle, A, d, k)
            ys[name] = Y.double()
            plan.close()
        nrm = float(torch.linalg.norm(Y64))
        row["rel_fro_vs_fp64"] = {nm: float(torch.linalg.norm(Yv - Y64)) / nrm for nm, Yv in ys.items()}
        try:
            R_A = r_factor_of(A)
            ef = eta_general(ys["fp32"], R_A)
            eh = eta_general(ys["fp16_rn"], R_A)
            row["eta_fp32"], row["eta_fp16_rn"] = ef, eh
        except RuntimeError:
            row["eta_fp32"] = row["eta_fp16_rn"] = None  # rank-deficient A (adversarial with few rows)
        out[fam] = row
        del A, Y64, ys
        torch.cuda.empty_cache()
    return out


def bench_batch(dev, rule_name="fp16_rn", count=256, reps=5):
    """256 uneven matrices in one persistent launch, captured in a CUDA graph and replayed."""
    import torch
    from paper_2606_20195_gb300 import autotune, inputs, sk
    rule = sk.RULES[rule_name]
    items = []
    total = 0
    for i, (m, n, fam) in enumerate(inputs.batch_shapes(count, seed=0)):
        A = inputs.device_matrix(m, n, fam, seed=100 + i, device=str(dev))
        Y = torch.empty((32 * n, n), dtype=y_dtype(rule), device=dev)
        items.append({"A": A, "Y": Y, "m": m, "n": n, "d": 32 * n, "k": 4, "seed": i})
        total += m * n * 4 + 32 * n * n * (4 if rule == 0 else 2)
    b, params = autotune.tune_batch(items, rule, reps=2)
    nwork, bytes_a = sk.sk_batch_info(b)
    stream = torch.cuda.Stream(device=dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        sk.sk_batch_launch(b, stream)
    stream.synchronize()
    with torch.cuda.graph(graph, stream=stream):
        sk.sk_batch_launch(b, torch.cuda.current_stream(dev))
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        graph.replay()
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / reps
    sk.sk_batch_destroy(b)
    del items
    torch.cuda.empty_cache()
    return {"workload": f"{count} uneven matrices, m log-uniform [2^12,2^20], n in 8..128, d=32n, k=4, {rule_name}",
            "GB/s": total / (ms * 1e-3) / 1e9, "ms": ms, "work_items": nwork, "bytes_A": bytes_a,
            "tuned": params, "graph": True}


def bench_serve(dev, count=1000, warm=200, log2_m=(14, 20), seed=0, rates=(0.5, 0.8, 0.95)):
    """Poisson stream of sketch-and-solve requests: continuous batching vs one at a time. Each
    measured run serves `count` requests after a warm-up run of `warm` requests of the same mix; the
    saturated run submits every request at t = 0 (throughput of the continuous path beside the
    one-at-a-time path's back-to-back throughput)."""
    from paper_2606_20195_gb300 import serve
    one = serve.Server(slots=1, hbm_budget_bytes=120 * 10**9, device=str(dev), keep_results=False)
    one.run_one_at_a_time(serve.make_stream(warm, rate_hz=0.0, seed=seed + 1, log2_m=log2_m))
    cap = one.run_one_at_a_time(serve.make_stream(count, rate_hz=0.0, seed=seed, log2_m=log2_m))
    capacity = cap["solves_per_s"]
    one.close()
    out = {"workload": f"Poisson sketch-and-solve requests, m log-uniform [2^{log2_m[0]},2^{log2_m[1]}], "
                       f"n in 16..256, d=16n, k in {{1,4,8}}, 4 rules, 120 GB budget, 8 slots; continuous path: one batched "
                       f"sketch launch per rule and scheduling step, then per-request FP64 QR; "
                       f"{count} requests per run after {warm} warm-up requests",
           "one_at_a_time_back_to_back": cap}
    srv = serve.Server(slots=8, hbm_budget_bytes=120 * 10**9, device=str(dev), keep_results=False)
    srv.run(serve.make_stream(warm, rate_hz=0.0, seed=seed + 1, log2_m=log2_m))
    l0 = srv.launches
    out["saturated_continuous"] = srv.run(serve.make_stream(count, rate_hz=0.0, seed=seed, log2_m=log2_m))
    out["saturated_continuous"]["batched_launches"] = srv.launches - l0
    srv.close()
    # the same loop with batching off (every request through the single-matrix path on its own
    # stream): what overlapping requests alone gives, beside what batching their sketches adds
    srv = serve.Server(slots=8, hbm_budget_bytes=120 * 10**9, device=str(dev), keep_results=False)
    srv.BATCH_MAX_BYTES = 0
    srv.run(serve.make_stream(warm, rate_hz=0.0, seed=seed + 1, log2_m=log2_m))
    out["saturated_continuous_no_batching"] = srv.run(serve.make_stream(count, rate_hz=0.0, seed=seed, log2_m=log2_m))
    srv.close()
    # more slots: larger batches per scheduling step when every request is already waiting
    srv = serve.Server(slots=32, hbm_budget_bytes=120 * 10**9, device=str(dev), keep_results=False)
    srv.run(serve.make_stream(warm, rate_hz=0.0, seed=seed + 1, log2_m=log2_m))
    out["saturated_continuous_32_slots"] = srv.run(serve.make_stream(count, rate_hz=0.0, seed=seed, log2_m=log2_m))
    srv.close()
    for frac in rates:
        srv = serve.Server(slots=8, hbm_budget_bytes=120 * 10**9, device=str(dev), keep_results=False)
        # warm-up pass over the same mix (plan scratch and per-stream allocator pools)
        srv.run(serve.make_stream(warm, rate_hz=frac * capacity, seed=seed + 1, log2_m=log2_m))
        cb = srv.run(serve.make_stream(count, rate_hz=frac * capacity, seed=seed, log2_m=log2_m))
        srv.close()
        s1 = serve.Server(slots=1, hbm_budget_bytes=120 * 10**9, device=str(dev), keep_results=False)
        s1.run_one_at_a_time(serve.make_stream(warm, rate_hz=0.0, seed=seed + 1, log2_m=log2_m))
        fifo = s1.run_one_at_a_time(serve.make_stream(count, rate_hz=frac * capacity, seed=seed, log2_m=log2_m))
        s1.close()
        out[f"rate_{int(frac * 100)}pct"] = {"rate_hz": frac * capacity, "continuous": cb, "fifo": fifo}
    return out


def run_sharded(args, world, rank, dev, sk, inputs) -> int:
    """One matrix split by rows over the ranks (strong scaling): per step every rank adds its rows'
    FP32 chunk totals (sk_apply_partials), one NCCL all-reduce sums them, and every rank finishes Y
    (sk_finish_partials)."""
    import torch
    import torch.distributed as dist
    m, n, d, k = WORKLOADS[args.workload]
    rule = sk.RULES[args.rule]
    R = default_chunk_rows(m)
    nchunks = (m + R - 1) // R
    lo, hi = rank * m // world, (rank + 1) * m // world
    A_pin = torch.from_numpy(inputs.host_matrix(hi - lo, n, "incoherent", seed=rank)).pin_memory()
    A = A_pin.to(dev)
    plan = sk.Plan(d, hi - lo, k, rule, seed=1234, row_offset=lo, chunk_rows=R)
    full = sk.Plan(d, m, k, rule, seed=1234, chunk_rows=R)
    P = torch.zeros((nchunks, d, n), dtype=torch.float32, device=dev)
    Y = torch.empty((d, n), dtype=y_dtype(rule), device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(Ad):
        sk.sk_apply_partials(plan.handle, Ad, n, n, P, 0, nchunks, stream)
        if world > 1:
            dist.all_reduce(P, op=dist.ReduceOp.SUM)
        sk.sk_finish_partials(full.handle, P, 0, nchunks, n, Y, stream)

    for _ in range(args.warmup):
        step(A)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        torch.cuda.synchronize()
        evs[0].record(stream)
        for _ in range(args.steps):
            step(A)
        evs[1].record(stream)
        torch.cuda.synchronize()
    clocks = clk.summary()
    t = torch.tensor([evs[0].elapsed_time(evs[1])], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    es = 4 if rule == 0 else 2
    bytes_step = m * n * 4 + d * n * es
    value = bytes_step * args.steps / (max_ms * 1e-3) / 1e9
    assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
    launches = plan.get(sk.SK_PARAM_LAST_LAUNCHES) + full.get(sk.SK_PARAM_LAST_LAUNCHES)
    # e2e: this rank's rows copied in from pinned host memory every step, Y copied out
    Y_pin = torch.empty((d, n), dtype=y_dtype(rule)).pin_memory()
    A_in = torch.empty_like(A)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        A_in.copy_(A_pin, non_blocking=True)
        step(A_in)
        Y_pin.copy_(Y, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    te = torch.tensor([e2e_s], device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") or 6800.0
    achieved = bytes_step / world / (max_ms / args.steps * 1e-3) / 1e9  # per-GPU share of the bytes
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32+f16" if rule != 0 else "f32",
            "data": "synthetic (seeded iid N(0,1) rows, one matrix split by rows over the ranks)",
            "config": {"workload": args.workload, "m": m, "n": n, "d": d, "k": k, "rule": args.rule,
                       "chunk_rows": R, "l2": "inputs larger than L2, no flush" if m * n * 4 > 129e6 else "inputs below L2",
                       "parallelism": f"rows{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "note": "per-GPU share of the step (partials + all-reduce + finish)"},
            "cpu_baseline": None,
            "e2e": {"value": bytes_step / float(te.item()) / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": (hi - lo) * n * 4, "d2h_bytes_per_step": d * n * es},
            "gpu_launches": launches * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    full.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--rule", default="fp16_rn", choices=["fp32", "fp16_rn", "fp16_sr", "fp16_dither", "bf16_rn"])
    ap.add_argument("--no-extras", action="store_true", help="skip variants, distortion, cpu baseline, serving")
    ap.add_argument("--extras", default="serve,solve,batch",
                    help="comma list of extra measurements: serve, solve, batch (the default), paper, all")
    ap.add_argument("--shard", default="none", choices=["none", "rows"],
                    help="rows: the ranks share one matrix split by rows (partials, NCCL all-reduce, finish)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_2606_20195_gb300 import _build, inputs, sk
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    sk.load()
    if args.shard == "rows":
        return run_sharded(args, world, rank, dev, sk, inputs)

    m, n, d, k = WORKLOADS[args.workload]
    rule = sk.RULES[args.rule]
    # Host matrix (pinned) for e2e; a device copy for the resident measurement. Each rank gets its
    # own independent matrix (seed = rank).
    A_h = inputs.host_matrix(m, n, "incoherent", seed=rank)
    A_pin = torch.from_numpy(A_h).pin_memory()
    A = A_pin.to(dev)
    Yb = torch.empty((d, n), dtype=y_dtype(rule), device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(plan_h, rule_v, steps, warmup):
        Y = torch.empty((d, n), dtype=y_dtype(rule_v), device=dev)
        for _ in range(warmup):
            sk.sk_apply(plan_h, A, n, n, Y, stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        torch.cuda.synchronize()
        evs[0].record(stream)
        for s in range(steps):
            sk.sk_apply(plan_h, A, n, n, Y, stream)
            evs[s + 1].record(stream)
        torch.cuda.synchronize()
        per = [evs[s].elapsed_time(evs[s + 1]) for s in range(steps)]
        total = evs[0].elapsed_time(evs[-1])
        return total, per, Y

    plan = sk.Plan(d, m, k, rule, seed=1234 + rank)
    with ClockSampler(local) as clk:
        total_ms, per_ms, Y = timed(plan.handle, rule, args.steps, args.warmup)
    clocks = clk.summary()
    launches_per_step = plan.get(sk.SK_PARAM_LAST_LAUNCHES)
    R_used = plan.get(sk.SK_PARAM_LAST_CHUNK_ROWS)
    kernel_name = {sk.SK_KERNEL_TILE: "tile_kernel", sk.SK_KERNEL_OWNER: "own_kernel",
                   sk.SK_KERNEL_LITERAL: "literal_kernel", sk.SK_KERNEL_GLOBAL: "global_kernel",
                   sk.SK_KERNEL_REGISTER: "reg_kernel"}.get(plan.get(sk.SK_PARAM_LAST_KERNEL), "det_kernel")
    t = torch.tensor([total_ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    es = 4 if rule == 0 else 2
    bytes_step = m * n * 4 + d * n * es
    value = world * bytes_step * args.steps / (max_ms * 1e-3) / 1e9

    # e2e through the host-buffer entry point (pinned A in, pinned Y out)
    Y_pin = torch.empty((d, n), dtype=y_dtype(rule)).pin_memory()
    for _ in range(max(3, args.warmup)):
        sk.sk_apply_host(plan.handle, A_pin.data_ptr(), n, n, Y_pin.data_ptr(), stream)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    # Three repetitions of e2e_steps calls; the median repetition's time per call is reported (a
    # single host-side stall of tens of milliseconds, seen in a few runs, would otherwise dominate).
    call_s, rep_s = [], []
    for _ in range(3):
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            tc = time.perf_counter()
            sk.sk_apply_host(plan.handle, A_pin.data_ptr(), n, n, Y_pin.data_ptr(), stream)
            call_s.append(time.perf_counter() - tc)
        rep_s.append((time.perf_counter() - t0) / e2e_steps)
    e2e_s = statistics.median(rep_s)
    e2e_launches = plan.get(sk.SK_PARAM_LAST_LAUNCHES)
    te = torch.tensor([e2e_s], device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * bytes_step / float(te.item()) / 1e9
    # context for e2e: plain pinned host -> device copy bandwidth of A
    A_scratch = torch.empty_like(A)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    A_scratch.copy_(A_pin, non_blocking=True)
    h0.record(stream)
    for _ in range(3):
        A_scratch.copy_(A_pin, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    h2d_gbps = 3 * m * n * 4 / (h0.elapsed_time(h1) * 1e-3) / 1e9
    del A_scratch

    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_note = "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if peak else "fallback 6800 GB/s"
    peak = peak or 6800.0
    avg_launch_ms = statistics.mean(per_ms)
    achieved = bytes_step / (avg_launch_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_record(kernel_name, args.workload, args.rule), "peak_source": peak_note,
                "kernel": f"sk::{kernel_name}<{args.rule}>",
                "algorithmic_bytes_per_launch": bytes_step}
    # The second ceiling of this path: signed FP32 updates (m n k per launch, k/4 per byte of A); in
    # the register kernel every update is a packed FMA on a row staged in shared memory, so the rate of
    # shared-memory row reads bounds it. Reported per SM clock beside the HBM fraction.
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    upd_s = m * n * k / (avg_launch_ms * 1e-3)
    sm_hz = (clocks.get("sm_mhz") or 0) * 1e6
    roofline["updates"] = {"per_launch": m * n * k, "per_s": upd_s,
                           "per_clk_per_sm": upd_s / (sms * sm_hz) if sm_hz else None,
                           "per_byte_of_A": k / 4.0}

    extras = {}
    cpu_baseline = None
    if rank == 0 and not args.no_extras:
        # Variants at the same workload (a few steps each).
        variants = {}
        etas = {}
        for name, rv in sk.RULES.items():
            p2 = sk.Plan(d, m, k, rv, seed=1234)
            tot, per, Yv = timed(p2.handle, rv, 5, 3)
            es2 = 4 if rv == 0 else 2
            variants[name] = {"GB/s": (m * n * 4 + d * n * es2) / (statistics.mean(per) * 1e-3) / 1e9,
                              "ms": statistics.mean(per)}
            etas[name] = Yv.double()
            p2.close()
        # 16-bit A (sk_apply_typed): the same rows, half the bytes of A read; GB/s of its own
        # algorithmic bytes (2 bytes per element of A).
        for a_name, a_dt, a_code in (("fp16_rn_a_fp16", torch.float16, sk.SK_A_FP16),
                                     ("fp16_rn_a_bf16", torch.bfloat16, sk.SK_A_BF16)):
            A16 = A.to(a_dt)
            p2 = sk.Plan(d, m, k, sk.SK_FP16_RN, seed=1234)
            Y16 = torch.empty((d, n), dtype=torch.float16, device=dev)
            for _ in range(3):
                sk.sk_apply_typed(p2.handle, A16, a_code, n, n, Y16, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(5):
                sk.sk_apply_typed(p2.handle, A16, a_code, n, n, Y16, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms16 = e0.elapsed_time(e1) / 5
            variants[a_name] = {"GB/s": (m * n * 2 + d * n * 2) / (ms16 * 1e-3) / 1e9, "ms": ms16,
                                "rows_per_s_vs_fp32_A": variants["fp16_rn"]["ms"] / ms16}
            p2.close()
            del A16, Y16
        # Distortion eta(S, Q) of the column space of A (A = Q R_A) for every rule (same S).
        R_A = r_factor_of(A)
        eta = {nm: eta_general(Yv, R_A) for nm, Yv in etas.items()}
        extras["variants"] = variants
        extras["distortion"] = {"eta_fp32": eta["fp32"], "eta_fp16_rn": eta["fp16_rn"],
                                "rel_diff": abs(eta["fp16_rn"] - eta["fp32"]) / eta["fp32"],
                                "eta_fp16_sr": eta["fp16_sr"], "eta_fp16_dither": eta["fp16_dither"],
                                "eta_bf16_rn": eta["bf16_rn"],
                                "rel_diff_bf16": abs(eta["bf16_rn"] - eta["fp32"]) / eta["fp32"],
                                "gaussian_reference_sqrt_n_over_d": float(np.sqrt(n / d))}
        extras["fp16_vs_fp32_speedup"] = variants["fp16_rn"]["GB/s"] / variants["fp32"]["GB/s"]
        extras["families"] = bench_families(dev, m, n, d, k)
        gb, cores, sample = cpu_oracle_rate(m, n, d, k, budget_s=10.0)
        cpu_baseline = {"value": gb, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample}
        want = set(args.extras.split(",")) if args.extras else set()
        if "all" in want:
            want = {"serve", "solve", "batch"}  # "paper" (minutes) only when asked for by name
        del A_pin
        if "serve" in want:
            extras["serving"] = bench_serve(dev)
            extras["p99_solve_ms"] = extras["serving"]["rate_80pct"]["continuous"]["p99_ms"]
            # the serving configuration's full m range (up to 2^24 rows: up to 16 GB of A per request)
            extras["serving_full_m_range"] = bench_serve(dev, count=200, warm=40, log2_m=(14, 24), rates=(0.8,))
        if "solve" in want:
            extras["sketch_and_solve"] = bench_solve(dev)
        if "batch" in want:
            extras["batched"] = bench_batch(dev)
        if "paper" in want:
            extras["paper_experiments"] = bench_paper(dev)
            extras["paper_least_squares"] = bench_paper_ls(dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f16" if rule != 0 else "f32",
            "data": "synthetic (seeded iid N(0,1) matrix per rank; paper publishes no number for this workload)",
            "config": {"workload": args.workload, "m": m, "n": n, "d": d, "k": k, "rule": args.rule,
                       "chunk_rows": R_used, "l2": (f"inputs larger than L2 ({m * n * 4 / 2**30:.2f} GiB of A), no flush" if m * n * 4 > 129e6
                              else "inputs smaller than L2: a cached-input number, not a headline"),
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "roofline": roofline,
            "cpu_baseline": cpu_baseline,
            "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": m * n * 4,
                    "d2h_bytes_per_step": d * n * es, "launches_per_step": e2e_launches,
                    "pinned_h2d_copy_GBps": h2d_gbps,
                    "repetitions_GBps": [bytes_step / r / 1e9 for r in rep_s],
                    "per_call_GBps_min_median_max": [bytes_step / max(call_s) / 1e9,
                                                     bytes_step / statistics.median(call_s) / 1e9,
                                                     bytes_step / min(call_s) / 1e9]},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            **extras,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
