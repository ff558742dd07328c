"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the sketching method: only the matrix families the
workloads are built from. Host generation uses numpy's PCG64 (default_rng(seed)); device
generation (for sizes the host should not produce) uses torch's CUDA generator with the seed.

Families (matching the workload definitions):
  incoherent   iid N(0, 1)
  coherent     first min(m, n) rows = 1e3 * I, remaining rows iid N(0, variance 1e-6)
  adversarial  row i = g_i * e_(i mod n), g_i iid N(0, 1)
"""
from __future__ import annotations

import numpy as np

FAMILIES = ("incoherent", "coherent", "adversarial")


def host_matrix(m: int, n: int, family: str = "incoherent", seed: int = 0, chunk: int = 1 << 22) -> np.ndarray:
    """m x n float32 matrix of the given family, generated on the host in row chunks."""
    rng = np.random.default_rng(seed)
    A = np.empty((m, n), dtype=np.float32)
    if family == "incoherent":
        for i0 in range(0, m, max(1, chunk // max(n, 1))):
            i1 = min(m, i0 + max(1, chunk // max(n, 1)))
            A[i0:i1] = rng.standard_normal((i1 - i0, n), dtype=np.float32)
    elif family == "coherent":
        for i0 in range(0, m, max(1, chunk // max(n, 1))):
            i1 = min(m, i0 + max(1, chunk // max(n, 1)))
            A[i0:i1] = rng.standard_normal((i1 - i0, n), dtype=np.float32) * np.float32(1e-3)
        q = min(m, n)
        A[:q, :] = 0.0
        A[np.arange(q), np.arange(q)] = np.float32(1e3)
    elif family == "adversarial":
        g = rng.standard_normal(m, dtype=np.float32)
        A[:] = 0.0
        A[np.arange(m), np.arange(m) % n] = g
    else:
        raise ValueError(f"unknown family {family!r}")
    return A


def host_vector(m: int, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(m, dtype=np.float32)


def device_matrix(m: int, n: int, family: str = "incoherent", seed: int = 0, device: str = "cuda:0"):
    """The same families generated on the GPU with torch (values differ from host_matrix)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    if family == "incoherent":
        return torch.randn((m, n), generator=g, device=device, dtype=torch.float32)
    if family == "coherent":
        A = torch.randn((m, n), generator=g, device=device, dtype=torch.float32).mul_(1e-3)
        q = min(m, n)
        A[:q, :] = 0.0
        idx = torch.arange(q, device=device)
        A[idx, idx] = 1e3
        return A
    if family == "adversarial":
        gv = torch.randn(m, generator=g, device=device, dtype=torch.float32)
        A = torch.zeros((m, n), device=device, dtype=torch.float32)
        r = torch.arange(m, device=device)
        A[r, r % n] = gv
        return A
    raise ValueError(f"unknown family {family!r}")


_GENERATORS: dict = {}


def device_generator(device, seed: int):
    """A torch generator of `device` seeded with `seed`: one object per device, re-seeded on every
    call, so it yields what a fresh generator with that seed would, without creating one per call."""
    import torch
    key = str(device)
    g = _GENERATORS.get(key)
    if g is None:
        g = _GENERATORS[key] = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def fill_device_matrix(out, family: str = "incoherent", seed: int = 0):
    """device_matrix written into an existing float32 CUDA tensor (same values for the same seed and
    shape): no device allocation, for callers that place matrices in their own memory."""
    import torch
    g = device_generator(out.device, seed)
    m, n = out.shape
    if family == "incoherent":
        torch.randn((m, n), generator=g, out=out)
        return out
    if family == "coherent":
        torch.randn((m, n), generator=g, out=out)
        out.mul_(1e-3)
        q = min(m, n)
        out[:q, :] = 0.0
        # fill kernels with the value as an argument: an indexed assignment of a Python scalar would
        # copy it from pageable host memory, which waits for the stream's earlier work
        out.diagonal().fill_(1e3)
        return out
    raise ValueError(f"unknown family {family!r} for an in-place fill")


def ls_problem_host(m: int, n: int, family: str = "coherent", seed: int = 0, noise: float = 1e-6):
    """(A, b, x_star) with b = A x_star + noise * N(0, 1), float32 (sketch-and-solve workload)."""
    A = host_matrix(m, n, family, seed)
    rng = np.random.default_rng(seed + 1)
    x_star = rng.standard_normal(n)
    b = np.empty(m, dtype=np.float32)
    step = 1 << 20
    for i0 in range(0, m, step):
        i1 = min(m, i0 + step)
        b[i0:i1] = (A[i0:i1].astype(np.float64) @ x_star + noise * rng.standard_normal(i1 - i0)).astype(np.float32)
    return A, b, x_star


def paper_ls_problem(family: str, m: int = 1 << 21, n: int = 1024, seed: int = 5303, device: str = "cuda:0"):
    """(A, b) of the paper's least-squares families (Sec. 5.3), float32 on the device.

    dense_easy / dense_hard: A = U diag(sigma) V^T, U and V the Q factors of Gaussian matrices,
    sigma linear from 100 to 1; b = A 1 + noise, with noise 1e-3 N(0,1) (easy) or 1e-1 N(0,1) + 1e-1
    (hard). coherent_permuted: A = [I_n; tau G / sqrt(m - n)], tau = 1e-3, b = [x* + eta;
    (tau G / sqrt(m - n)) x*], x* ~ N(0,1), eta ~ 0.5 N(0,1), rows permuted at random."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    if family in ("dense_easy", "dense_hard"):
        U = torch.linalg.qr(torch.randn((m, n), generator=g, device=device)).Q
        V = torch.linalg.qr(torch.randn((n, n), generator=g, device=device)).Q
        sig = torch.linspace(100.0, 1.0, n, device=device)
        A = ((U * sig) @ V.T).contiguous()
        del U
        b = A.sum(dim=1)
        if family == "dense_easy":
            b += 1e-3 * torch.randn(m, generator=g, device=device)
        else:
            b += 1e-1 * torch.randn(m, generator=g, device=device) + 1e-1
        return A, b.contiguous()
    if family == "coherent_permuted":
        tau = 1e-3
        G = torch.randn((m - n, n), generator=g, device=device) * (tau / (m - n) ** 0.5)
        xs = torch.randn(n, generator=g, device=device)
        A = torch.cat([torch.eye(n, device=device), G])
        b = torch.cat([xs + 0.5 * torch.randn(n, generator=g, device=device), G @ xs])
        del G
        perm = torch.randperm(m, generator=g, device=device)
        return A[perm].contiguous(), b[perm].contiguous()
    raise ValueError(f"unknown least-squares family {family!r}")


def batch_shapes(count: int = 256, seed: int = 0, log2_lo: float = 12.0, log2_hi: float = 20.0,
                 ns=(8, 16, 32, 64, 128)):
    """(m_i, n_i, family_i) for the batched workload: m log-uniform in [2^lo, 2^hi], n uniform in ns,
    even index incoherent, odd index coherent."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(2.0 ** rng.uniform(log2_lo, log2_hi))
        n = int(rng.choice(ns))
        out.append((m, n, "incoherent" if i % 2 == 0 else "coherent"))
    return out
