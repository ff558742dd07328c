"""Row-sharded sketching across ranks (gloo, world size 2).

S is a pure function of (seed, global row, block), so rank r sketches its contiguous row range with
the global row indices (sk's SK_PARAM_ROW_OFFSET) and the partial sketches add up to the sketch of
the whole matrix; the one exchange step is an all-reduce (sum) of the partials, in FP32 chunk totals
before any 16-bit rounding.

Two forms: on CPU (no GPU needed), the ranks compute FP64 partials with the oracle, which checks the
sharding arithmetic and the collective; on the GPU, both ranks call libsk (sk_apply_partials) on the
one GPU, all-reduce their FP32 chunk totals over gloo on the host, and rank 0 finishes them
(sk_finish_partials): bit-exact with the oracle's canonical order on small-integer data. The ranks'
kernels never wait on each other; the only exchange is the host all-reduce.
"""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2606_20195_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, n, d, k, seed = 10_007, 6, 96, 4, 5
    A = inputs.host_matrix(m, n, "coherent", seed=1)
    # contiguous shard; the partial sketch uses global row indices: rows before the shard are zero
    lo, hi = rank * m // world, (rank + 1) * m // world
    Ashard = np.zeros_like(A)
    Ashard[lo:hi] = A[lo:hi]
    part = torch.from_numpy(oracle.sketch_f64(Ashard[:hi], d, k, seed))
    dist.all_reduce(part, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, part.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_sketch_allreduce_equals_full(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_2606_20195_gb300 import inputs
    port = _free_port()
    out = str(tmp_path / "y.npy")
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    Y = np.load(out)
    A = inputs.host_matrix(10_007, 6, "coherent", seed=1)
    ref = oracle.sketch_f64(A, 96, 4, 5)
    assert np.allclose(Y, ref, rtol=1e-12, atol=1e-9)


def _gpu_worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2606_20195_gb300 import sk
    sk.load()  # built by the parent before the ranks start
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, n, d, k, seed, R, rule = 40_009, 64, 2048, 8, 19, 4096, 1
    A = np.random.default_rng(7).integers(-3, 4, size=(m, n)).astype(np.float32)
    lo, hi = rank * m // world + 5, (rank + 1) * m // world + 5  # shard edges off the chunk grid
    lo, hi = (0 if rank == 0 else lo), (m if rank == world - 1 else hi)
    nchunks = (m + R - 1) // R
    dev = torch.device("cuda:0")
    plan = sk.Plan(d, hi - lo, k, rule, seed, row_offset=lo, chunk_rows=R)
    P = torch.zeros((nchunks, d, n), dtype=torch.float32, device=dev)
    Ad = torch.from_numpy(A[lo:hi]).to(dev)
    sk.sk_apply_partials(plan.handle, Ad, n, n, P, 0, nchunks)
    torch.cuda.synchronize()
    assert plan.get(sk.SK_PARAM_DEVICE_STATUS) == 0
    plan.close()
    Ph = P.cpu()
    dist.all_reduce(Ph, op=dist.ReduceOp.SUM)
    if rank == 0:
        full = sk.Plan(d, m, k, rule, seed, chunk_rows=R)
        Pd = Ph.to(dev)
        Y = torch.empty((d, n), dtype=torch.float16, device=dev)
        sk.sk_finish_partials(full.handle, Pd, 0, nchunks, n, Y)
        torch.cuda.synchronize()
        np.save(out_path, Y.view(torch.int16).cpu().numpy().view(np.uint16))
        full.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_two_ranks_libsk_partials_allreduce_bit_exact(tmp_path):
    import torch
    import torch.multiprocessing as mp

    import oracle
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_20195_gb300 import _build
    _build.build()
    port = _free_port()
    out = str(tmp_path / "y16.npy")
    mp.start_processes(_gpu_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    A = np.random.default_rng(7).integers(-3, 4, size=(40_009, 64)).astype(np.float32)
    ref = oracle.sketch_canonical(A, 2048, 8, 19, 1, 4096)
    assert np.array_equal(got, ref), np.count_nonzero(got != ref)
