"""CPU oracle for the SparseStack sketch (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import this package. The CUDA product path never imports it, and it
imports nothing from the CUDA package: the two share only the seeded input generators.

The arithmetic lives in ``sk_oracle.c`` (built with ``-ffp-contract=off``) and is exposed
here through ctypes with numpy-friendly wrappers. The least-squares and distortion helpers
at the bottom use numpy's FP64 QR/SVD as library steps.

Sources restated (see the C file for the per-function citations):
  * SparseStack operator, paper Sec. 2.2 (Definition of SparseStack) and Sec. 4.1.
  * FP16 quantizers, paper Sec. 4.2 (round-to-nearest, exact stochastic, dithered), and the
    bfloat16 round-to-nearest rule (Sec. 4.2 names BF16 beside FP16 as a 16-bit reduction target).
  * Distortion eta(S, U), paper Sec. 2.2 / Sec. 5.1.
  * Sketch-and-solve least squares, paper Sec. 5.1 (min ||SAx - Sb||).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libsk_oracle.so")
_lock = threading.Lock()
_lib = None

FP32, FP16_RN, FP16_SR, FP16_DITHER, BF16_RN = 0, 1, 2, 3, 4
RULES = {"fp32": FP32, "fp16_rn": FP16_RN, "fp16_sr": FP16_SR, "fp16_dither": FP16_DITHER, "bf16_rn": BF16_RN}


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            u64, i64, i32, u32, u16 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint16
            P = ctypes.c_void_p
            L.sko_splitmix64_mix.restype = u64
            L.sko_splitmix64_mix.argtypes = [u64]
            L.sko_splitmix64_nth.restype = u64
            L.sko_splitmix64_nth.argtypes = [u64, u64]
            L.sko_philox4x32_10.restype = None
            L.sko_philox4x32_10.argtypes = [P, P, P]
            L.sko_uniform.restype = ctypes.c_float
            L.sko_uniform.argtypes = [u64, i64, i64, i64]
            L.sko_s_pattern.restype = None
            L.sko_s_pattern.argtypes = [i64, i32, u64, i64, i64, P, P]
            L.sko_half_to_double.restype = ctypes.c_double
            L.sko_half_to_double.argtypes = [u16]
            L.sko_round_to_half.restype = u16
            L.sko_round_to_half.argtypes = [ctypes.c_double, ctypes.c_int]
            L.sko_half_add.restype = u16
            L.sko_half_add.argtypes = [u16, u16]
            L.sko_bf16_to_double.restype = ctypes.c_double
            L.sko_bf16_to_double.argtypes = [u16]
            L.sko_round_to_bf16.restype = u16
            L.sko_round_to_bf16.argtypes = [ctypes.c_double]
            L.sko_bf16_add.restype = u16
            L.sko_bf16_add.argtypes = [u16, u16]
            L.sko_quantize.restype = u16
            L.sko_quantize.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int]
            L.sko_sketch_f64.restype = None
            L.sko_sketch_f64.argtypes = [P, i64, i64, i64, i64, i32, u64, P]
            L.sko_sketch_canonical.restype = None
            L.sko_sketch_canonical.argtypes = [P, i64, i64, i64, i64, i32, u64, ctypes.c_int, i64, P]
            L.sko_sketch_sampled.restype = None
            L.sko_sketch_sampled.argtypes = [P, i64, i64, i64, i64, i32, u64, ctypes.c_int, i64, i64, P, P, P, P]
            L.sko_num_threads.restype = ctypes.c_int
            L.sko_num_threads.argtypes = []
            L.sko_round_to_half_f32_array.restype = None
            L.sko_round_to_half_f32_array.argtypes = [P, i64, ctypes.c_int, P]
            L.sko_half_add_array.restype = None
            L.sko_half_add_array.argtypes = [P, P, i64, P]
            L.sko_round_to_bf16_f32_array.restype = None
            L.sko_round_to_bf16_f32_array.argtypes = [P, i64, P]
            L.sko_bf16_add_array.restype = None
            L.sko_bf16_add_array.argtypes = [P, P, i64, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as_f32_rows(A: np.ndarray) -> tuple[np.ndarray, int]:
    """A as float32 with unit column stride; returns (array, lda)."""
    A = np.asarray(A, dtype=np.float32)
    if A.ndim != 2:
        raise ValueError("A must be 2-D")
    if A.strides[1] != 4 or A.strides[0] % 4 != 0:
        A = np.ascontiguousarray(A)
    return A, A.strides[0] // 4


# ----------------------------------------------------------------------------- generators
def splitmix64_mix(z: int) -> int:
    return int(lib().sko_splitmix64_mix(z & (2**64 - 1)))


def splitmix64_nth(seed: int, n: int) -> int:
    return int(lib().sko_splitmix64_nth(seed & (2**64 - 1), n & (2**64 - 1)))


def philox4x32_10(ctr, key) -> tuple[int, int, int, int]:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().sko_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return tuple(int(x) for x in out)


def uniform(seed: int, r: int, c: int, t: int) -> float:
    return float(lib().sko_uniform(seed, r, c, t))


def s_pattern(d: int, k: int, seed: int, m: int, i0: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(rows[m, k] int64, signs[m, k] int8) of the SparseStack operator for rows i0..i0+m-1."""
    rows = np.zeros((m, k), dtype=np.int64)
    signs = np.zeros((m, k), dtype=np.int8)
    lib().sko_s_pattern(d, k, seed, i0, m, _ptr(rows), _ptr(signs))
    return rows, signs


def dense_S(d: int, k: int, seed: int, m: int) -> np.ndarray:
    """The d x m SparseStack matrix in float64 (tiny sizes only)."""
    rows, signs = s_pattern(d, k, seed, m)
    S = np.zeros((d, m), dtype=np.float64)
    v = 1.0 / np.sqrt(k)
    for i in range(m):
        for j in range(k):
            S[rows[i, j], i] += signs[i, j] * v
    return S


# ----------------------------------------------------------------------------- binary16
def half_to_double(h: int) -> float:
    return float(lib().sko_half_to_double(h & 0xFFFF))


def round_to_half(x: float, mode: int = 0) -> int:
    return int(lib().sko_round_to_half(float(x), mode))


def half_add(a: int, b: int) -> int:
    return int(lib().sko_half_add(a & 0xFFFF, b & 0xFFFF))


def bf16_to_double(h: int) -> float:
    return float(lib().sko_bf16_to_double(h & 0xFFFF))


def round_to_bf16(x: float) -> int:
    return int(lib().sko_round_to_bf16(float(x)))


def bf16_add(a: int, b: int) -> int:
    return int(lib().sko_bf16_add(a & 0xFFFF, b & 0xFFFF))


def round_to_half_array(x: np.ndarray, mode: int = 0) -> np.ndarray:
    """binary16 bit patterns of float32 values (element-wise round_to_half)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib().sko_round_to_half_f32_array(_ptr(x), x.size, mode, _ptr(out))
    return out


def half_add_array(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Element-wise binary16 sums (bit patterns in, bit patterns out)."""
    a = np.ascontiguousarray(a, dtype=np.uint16)
    b = np.ascontiguousarray(b, dtype=np.uint16)
    out = np.empty(a.shape, dtype=np.uint16)
    lib().sko_half_add_array(_ptr(a), _ptr(b), a.size, _ptr(out))
    return out


def round_to_bf16_array(x: np.ndarray) -> np.ndarray:
    """bfloat16 bit patterns of float32 values (element-wise round_to_bf16)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib().sko_round_to_bf16_f32_array(_ptr(x), x.size, _ptr(out))
    return out


def bf16_add_array(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Element-wise bfloat16 sums (bit patterns in, bit patterns out)."""
    a = np.ascontiguousarray(a, dtype=np.uint16)
    b = np.ascontiguousarray(b, dtype=np.uint16)
    out = np.empty(a.shape, dtype=np.uint16)
    lib().sko_bf16_add_array(_ptr(a), _ptr(b), a.size, _ptr(out))
    return out


def bf16bits_to_f64(h: np.ndarray) -> np.ndarray:
    """bfloat16 bit patterns (uint16) to float64, exactly."""
    return (np.asarray(h, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bits16_to_f64(h: np.ndarray, rule: int) -> np.ndarray:
    """16-bit results of an FP16 or BF16 rule to float64."""
    return bf16bits_to_f64(h) if rule == BF16_RN else halfbits_to_f64(h)


def quantize(x: float, u: float, rule: int) -> int:
    return int(lib().sko_quantize(np.float32(x), np.float32(u), rule))


def halfbits_to_f64(h: np.ndarray) -> np.ndarray:
    return np.asarray(h, dtype=np.uint16).view(np.float16).astype(np.float64)


# ----------------------------------------------------------------------------- sketches
def sketch_f64(A: np.ndarray, d: int, k: int, seed: int) -> np.ndarray:
    A, lda = _as_f32_rows(A)
    m, n = A.shape
    Y = np.zeros((d, n), dtype=np.float64)
    lib().sko_sketch_f64(_ptr(A), lda, m, n, d, k, seed, _ptr(Y))
    return Y


def sketch_canonical(A: np.ndarray, d: int, k: int, seed: int, rule: int, R: int) -> np.ndarray:
    """Canonical-order result: float32 (rule FP32) or the 16-bit patterns (binary16 or bfloat16) as uint16."""
    if d % k != 0 or R < 1:
        raise ValueError("need d % k == 0 and R >= 1")
    A, lda = _as_f32_rows(A)
    m, n = A.shape
    Y = np.zeros((d, n), dtype=np.float32 if rule == FP32 else np.uint16)
    lib().sko_sketch_canonical(_ptr(A), lda, m, n, d, k, seed, rule, R, _ptr(Y))
    return Y


def sketch_sampled(A: np.ndarray, d: int, k: int, seed: int, rule: int, R: int, rs, cs):
    """(FP64 values, canonical values as float64) at outputs (rs[q], cs[q])."""
    A, lda = _as_f32_rows(A)
    m, n = A.shape
    rs = np.ascontiguousarray(rs, dtype=np.int64)
    cs = np.ascontiguousarray(cs, dtype=np.int64)
    out64 = np.zeros(len(rs), dtype=np.float64)
    outc = np.zeros(len(rs), dtype=np.uint32)
    lib().sko_sketch_sampled(_ptr(A), lda, m, n, d, k, seed, rule, R, len(rs), _ptr(rs), _ptr(cs),
                             _ptr(out64), _ptr(outc))
    if rule == FP32:
        canon = outc.view(np.float32).astype(np.float64)
    else:
        canon = bits16_to_f64(outc.astype(np.uint16), rule)
    return out64, canon


def num_threads() -> int:
    return int(lib().sko_num_threads())


# ----------------------------------------------------------------------------- FP64 helpers
def rel_fro(X: np.ndarray, Ref: np.ndarray) -> float:
    """||X - Ref||_F / ||Ref||_F in float64."""
    X = np.asarray(X, dtype=np.float64)
    Ref = np.asarray(Ref, dtype=np.float64)
    den = np.linalg.norm(Ref)
    return float(np.linalg.norm(X - Ref) / den) if den > 0 else float(np.linalg.norm(X))


def distortion(SU: np.ndarray) -> float:
    """eta = max(|sigma_max(SU) - 1|, |1 - sigma_min(SU)|) (paper Sec. 2.2), U orthonormal."""
    s = np.linalg.svd(np.asarray(SU, dtype=np.float64), compute_uv=False)
    return float(max(abs(s[0] - 1.0), abs(1.0 - s[-1])))


def distortion_of(SA: np.ndarray, R_A: np.ndarray) -> float:
    """Distortion of the sketch of a general full-rank A with A = Q R_A: eta(S, Q) = eta of SA R_A^-1."""
    SQ = np.linalg.solve(np.asarray(R_A, dtype=np.float64).T, np.asarray(SA, dtype=np.float64).T).T
    return distortion(SQ)


def tall_r_factor(A: np.ndarray, chunk: int = 1 << 18) -> np.ndarray:
    """R factor (n x n, FP64) of a tall matrix by stacking chunk R factors (TSQR, one level)."""
    m, n = A.shape
    Rs = []
    for i0 in range(0, m, chunk):
        blk = np.asarray(A[i0:i0 + chunk], dtype=np.float64)
        Rs.append(np.linalg.qr(blk, mode="r"))
    R = np.linalg.qr(np.vstack(Rs), mode="r")
    # sign-normalise so that diag(R) > 0
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return R * sgn[:, None]


def lstsq_tall(A: np.ndarray, b: np.ndarray, chunk: int = 1 << 18):
    """FP64 least squares for a tall A via TSQR of [A | b]: returns (x_opt, ||A x_opt - b||)."""
    m, n = A.shape
    Rs = []
    for i0 in range(0, m, chunk):
        blk = np.hstack([np.asarray(A[i0:i0 + chunk], dtype=np.float64),
                         np.asarray(b[i0:i0 + chunk], dtype=np.float64).reshape(-1, 1)])
        Rs.append(np.linalg.qr(blk, mode="r"))
    R = np.linalg.qr(np.vstack(Rs), mode="r")
    x = np.linalg.solve(R[:n, :n], R[:n, n])
    return x, float(abs(R[n, n]))


def sketch_solve(SA: np.ndarray, Sb: np.ndarray):
    """x = argmin ||SA x - Sb|| by FP64 Householder QR (numpy) and a triangular solve."""
    SA = np.asarray(SA, dtype=np.float64)
    Sb = np.asarray(Sb, dtype=np.float64).reshape(-1)
    Q, R = np.linalg.qr(SA, mode="reduced")
    c = Q.T @ Sb
    return np.linalg.solve(R, c)


def residual_norm(A: np.ndarray, b: np.ndarray, x: np.ndarray, chunk: int = 1 << 20) -> float:
    """||A x - b|| in FP64, chunked over rows."""
    x = np.asarray(x, dtype=np.float64)
    acc = 0.0
    for i0 in range(0, A.shape[0], chunk):
        r = np.asarray(A[i0:i0 + chunk], dtype=np.float64) @ x - np.asarray(b[i0:i0 + chunk], dtype=np.float64)
        acc += float(r @ r)
    return float(np.sqrt(acc))
