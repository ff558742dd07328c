"""Row-sharded sketching across ranks (CPU, gloo, world size 2).

S is a pure function of (seed, global row, block), so rank r sketches its contiguous row range with
the global row indices (sk's SK_PARAM_ROW_OFFSET) and the partial sketches add up to the sketch of
the whole matrix; the one exchange step is an all-reduce (sum) of the FP32/FP64 partials. The ranks
here compute their partials with the CPU oracle; the test checks the sharding arithmetic and the
collective, not a GPU kernel.
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
