"""Exhaustive pins of the oracle's 16-bit arithmetic against CUDA's (through PyTorch on the GPU):
every binary32 pattern rounded to binary16 and to bfloat16 (round to nearest, ties to even), and
every pair of binary16 and of bfloat16 patterns added. PyTorch's CUDA conversions are the hardware
ones; its 16-bit additions round the binary32 sum, which is the correctly rounded 16-bit sum because
binary32 carries at least 2p + 2 significant bits for p = 11 and p = 8 (double rounding is then
innocuous). NaN results are compared as NaN (payloads are not specified)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

CHUNK = 1 << 28


def _nan16(h, bf16):
    h = np.asarray(h, dtype=np.uint16)
    if bf16:
        return ((h & 0x7F80) == 0x7F80) & ((h & 0x7F) != 0)
    return ((h & 0x7C00) == 0x7C00) & ((h & 0x3FF) != 0)


def _check(got, ref, bf16):
    ng, nr = _nan16(got, bf16), _nan16(ref, bf16)
    assert np.array_equal(ng, nr), int(np.count_nonzero(ng != nr))
    ok = ~nr
    bad = np.count_nonzero(got[ok] != ref[ok])
    assert bad == 0, bad


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_every_fp32_pattern_rounds_like_cuda(dev, fmt):
    import torch
    dt = torch.float16 if fmt == "fp16" else torch.bfloat16
    for c in range((1 << 32) // CHUNK):
        x = np.arange(c * CHUNK, (c + 1) * CHUNK, dtype=np.uint64).astype(np.uint32).view(np.float32)
        ref = oracle.round_to_half_array(x, 0) if fmt == "fp16" else oracle.round_to_bf16_array(x)
        got = torch.from_numpy(x).to(dev).to(dt).view(torch.int16).cpu().numpy().view(np.uint16)
        _check(got, ref, fmt == "bf16")


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_every_16bit_pair_adds_like_cuda(dev, fmt):
    import torch
    dt = torch.float16 if fmt == "fp16" else torch.bfloat16
    for c in range((1 << 32) // CHUNK):
        idx = np.arange(c * CHUNK, (c + 1) * CHUNK, dtype=np.uint64)
        a = (idx >> 16).astype(np.uint16)
        b = (idx & 0xFFFF).astype(np.uint16)
        ref = oracle.half_add_array(a, b) if fmt == "fp16" else oracle.bf16_add_array(a, b)
        ta = torch.from_numpy(a.view(np.int16)).to(dev).view(dt)
        tb = torch.from_numpy(b.view(np.int16)).to(dev).view(dt)
        got = (ta + tb).view(torch.int16).cpu().numpy().view(np.uint16)
        _check(got, ref, fmt == "bf16")
