"""The paper's coherent least-squares experiment (Sec. 5.3) at its size, m = 2^21, n = 1024 and
SparseStack with zeta = 4, through sk_solve, against the values the paper prints for it
(tests/golden/coherent_ls_table.txt). The instance is a fresh draw of the paper's construction, so
the bars leave room for sampling variation; what they hold is the paper's result: FP32 SparseStack
within a few percent of the printed residual and kappa(SA), CountSketch's residual and kappa two to
three orders of magnitude above SparseStack's, the FP16 rounding rules close to one another, and, with
the whole column pre-combined in FP32 before its one binary16 rounding, FP16 closer to FP32 than with
the default chunking (RN within 15 %, SR and dither within 30 %; the paper's "within 1 %" is not
reproduced)."""
import math
import os

import numpy as np
import pytest

from paper_2606_20195_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _table():
    out = {}
    with open(os.path.join(HERE, "golden", "coherent_ls_table.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            r, meth, res, kap = line.split()
            out[(int(r), meth)] = (float(res), float(kap))
    return out


def _rel_res(A, b, x, step=1 << 18):
    import torch
    acc = 0.0
    x64 = x.double()
    for i0 in range(0, A.shape[0], step):
        r = A[i0:i0 + step].double() @ x64 - b[i0:i0 + step].double()
        acc += float(r @ r)
    return math.sqrt(acc) / float(torch.linalg.vector_norm(b.double()))


def _kappa(Y):
    import torch
    X = Y.double()
    ev = torch.linalg.eigvalsh(X.T @ X)
    return float((ev[-1] / ev[0]).sqrt())


def test_golden_table_parses():
    t = _table()
    assert t[(2, "SparseStack")] == (6.09e-4, 6.70)
    assert t[(24, "CountSketch")] == (5.98e-2, 1.48e3)
    assert len(t) == 35


@pytest.mark.gpu
def test_coherent_least_squares_matches_paper_table(sk, dev):
    import torch
    m, n = 1 << 21, 1024
    A, b = inputs.paper_ls_problem("coherent_permuted", m, n, seed=5303, device=str(dev))
    tab = _table()
    # the least-squares optimum of the construction (normal-equations row of the table)
    Rs = []
    for i0 in range(0, m, 1 << 18):
        blk = torch.cat([A[i0:i0 + (1 << 18)].double(), b[i0:i0 + (1 << 18)].double()[:, None]], dim=1)
        Rs.append(torch.linalg.qr(blk, mode="r").R)
    r_opt = float(abs(torch.linalg.qr(torch.cat(Rs), mode="r").R[n, n])) / float(torch.linalg.vector_norm(b.double()))
    assert abs(r_opt - tab[(2, "NormalEq")][0]) <= 0.02 * tab[(2, "NormalEq")][0], r_opt
    for ratio in (2, 4):
        d = ratio * n
        got = {}
        for name, k, rule in (("SparseStack", 4, "fp32"), ("SparseStack-detm", 4, "fp16_rn"),
                              ("SparseStack-stoch", 4, "fp16_sr"), ("SparseStack-dither", 4, "fp16_dither"),
                              ("CountSketch", 1, "fp32")):
            plan = sk.Plan(d, m, k, rule, seed=31)
            x = plan.solve(A, b)
            status, _ = plan.solve_status()
            assert status == sk.SK_OK
            Y = plan.apply(A)
            got[name] = (_rel_res(A, b, x), _kappa(Y))
            plan.close()
            del Y
        res_ss, kap_ss = got["SparseStack"]
        p_res, p_kap = tab[(ratio, "SparseStack")]
        assert abs(res_ss - p_res) <= 0.08 * p_res, (ratio, res_ss, p_res)
        assert abs(kap_ss - p_kap) <= 0.15 * p_kap, (ratio, kap_ss, p_kap)
        res_cs, kap_cs = got["CountSketch"]
        p_res, p_kap = tab[(ratio, "CountSketch")]
        assert abs(res_cs - p_res) <= 0.2 * p_res, (ratio, res_cs, p_res)
        assert abs(kap_cs - p_kap) <= 0.15 * p_kap, (ratio, kap_cs, p_kap)
        assert res_cs > 100 * res_ss and kap_cs > 100 * kap_ss
        # FP16 rules: the same sketch geometry (kappa) as FP32, residuals close to one another and
        # within 2x of the FP32 residual
        fp16 = [got[nm] for nm in ("SparseStack-detm", "SparseStack-stoch", "SparseStack-dither")]
        for res, kap in fp16:
            assert abs(kap - kap_ss) <= 1e-2 * kap_ss
            assert 0.9 * res_ss <= res <= 2.0 * res_ss, (ratio, res, res_ss)
        rs = np.array([r for r, _ in fp16])
        assert rs.max() <= 1.25 * rs.min(), rs
        # One chunk (R = m: the whole column pre-combined in FP32, one binary16 rounding per output)
        # removes most of the FP16 excess of the default 8 chunks (measured at d/n = 2: +9 % over FP32
        # against +28 %), but not all of it: the rounding of S b is comparable to the tail rows' share
        # of S b in this construction, so the paper's "within 1 %" is not reached (see the design notes).
        for rule in ("fp16_rn", "fp16_sr", "fp16_dither"):
            plan = sk.Plan(d, m, 4, rule, seed=31, chunk_rows=m)
            x = plan.solve(A, b)
            assert plan.solve_status()[0] == sk.SK_OK
            res1 = _rel_res(A, b, x)
            plan.close()
            res8 = got[{"fp16_rn": "SparseStack-detm", "fp16_sr": "SparseStack-stoch",
                        "fp16_dither": "SparseStack-dither"}[rule]][0]
            # RN: +9 % measured at d/n = 2; SR and dither draw their noise from a wider distribution
            # (+18 % for SR)
            bar = 1.15 if rule == "fp16_rn" else 1.30
            assert res_ss <= res1 <= bar * res_ss, (ratio, rule, res1, res_ss)
            assert res1 <= 1.01 * res8, (ratio, rule, res1, res8)
    del A, b
    torch.cuda.empty_cache()
