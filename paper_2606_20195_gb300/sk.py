"""Thin ctypes binding of libsk (include/sk.h): the same entry points, argument marshalling only.

Every step of the sketch runs in the CUDA kernels of libsk.so. Importing this module loads the
library and fails loudly if it is missing; there is no CPU fallback. PyTorch tensors are accepted
for device buffers and streams (plumbing only).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsk.so")

SK_OK, SK_ERR_INVALID_ARG, SK_ERR_UNSUPPORTED, SK_ERR_OOM, SK_ERR_CUDA, SK_ERR_TIMEOUT, SK_ERR_NUMERIC = range(7)
SK_FP32, SK_FP16_RN, SK_FP16_SR, SK_FP16_DITHER, SK_BF16_RN = range(5)
RULES = {"fp32": SK_FP32, "fp16_rn": SK_FP16_RN, "fp16_sr": SK_FP16_SR, "fp16_dither": SK_FP16_DITHER,
         "bf16_rn": SK_BF16_RN}
SK_PARAM_CHUNK_ROWS, SK_PARAM_MODE, SK_PARAM_ROW_OFFSET, SK_PARAM_KERNEL = 1, 2, 3, 4
SK_PARAM_TILE_COLS, SK_PARAM_THREADS, SK_PARAM_LAST_LAUNCHES, SK_PARAM_LAST_CHUNK_ROWS = 5, 6, 7, 8
SK_PARAM_DEVICE_STATUS, SK_PARAM_LAST_KERNEL, SK_PARAM_SOLVE_GROUP_ROWS, SK_PARAM_LIST_CAP = 9, 10, 11, 12
SK_PARAM_SCRATCH_LIMIT, SK_PARAM_SOLVE_WAIT_CYCLES, SK_PARAM_SCRATCH_BYTES, SK_PARAM_ROWS = 13, 14, 15, 16
SK_PARAM_ITEM_CHUNKS = 17
SK_MODE_ATOMIC, SK_MODE_DETERMINISTIC, SK_MODE_SERIAL_TILE = 0, 1, 2
SK_KERNEL_AUTO, SK_KERNEL_TILE, SK_KERNEL_LITERAL, SK_KERNEL_OWNER, SK_KERNEL_GLOBAL = 0, 1, 2, 3, 4
SK_KERNEL_REGISTER = 6
SK_A_FP32, SK_A_FP16, SK_A_BF16 = 0, 1, 2

# Every symbol include/sk.h declares.
EXPORTS = [
    "sk_version", "sk_last_error", "sk_plan_create", "sk_plan_set", "sk_plan_get", "sk_apply",
    "sk_apply_host", "sk_solve", "sk_solve_status", "sk_solve_precond", "sk_materialize_S", "sk_batch_create",
    "sk_batch_set", "sk_batch_launch", "sk_batch_info", "sk_batch_destroy", "sk_destroy",
    "sk_apply_noalloc", "sk_apply_typed", "sk_apply_partials", "sk_finish_partials", "sk_solve_sketched",
    "sk_batch_rebind",
]


class SkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sk status {status}: {msg}")
        self.status = status


class sk_batch_item(ctypes.Structure):
    _fields_ = [("A_dev", ctypes.c_void_p), ("Y_dev", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("lda", ctypes.c_int64), ("d", ctypes.c_int64), ("k", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("seed", ctypes.c_uint64)]


_lib = None


def load(path: str | None = None):
    """Load libsk.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libsk.so not found at {p}: run __graft_entry__.build() (nvcc) first")
    L = ctypes.CDLL(p)
    i64, i32, u64, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p
    st = ctypes.c_int
    L.sk_version.restype = i32
    L.sk_version.argtypes = []
    L.sk_last_error.restype = ctypes.c_char_p
    L.sk_last_error.argtypes = []
    L.sk_plan_create.restype = st
    L.sk_plan_create.argtypes = [i64, i64, i32, i32, u64, ctypes.POINTER(vp)]
    L.sk_plan_set.restype = st
    L.sk_plan_set.argtypes = [vp, i32, i64]
    L.sk_plan_get.restype = st
    L.sk_plan_get.argtypes = [vp, i32, ctypes.POINTER(i64)]
    L.sk_apply.restype = st
    L.sk_apply.argtypes = [vp, vp, i64, i64, vp, vp]
    L.sk_apply_host.restype = st
    L.sk_apply_host.argtypes = [vp, vp, i64, i64, vp, vp]
    L.sk_solve.restype = st
    L.sk_solve.argtypes = [vp, vp, i64, i64, vp, vp, vp]
    L.sk_solve_status.restype = st
    L.sk_solve_status.argtypes = [vp, ctypes.POINTER(ctypes.c_double), vp]
    L.sk_solve_precond.restype = st
    L.sk_solve_precond.argtypes = [vp, vp, i64, i64, vp, vp, ctypes.c_int32, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_int32), vp]
    L.sk_materialize_S.restype = st
    L.sk_materialize_S.argtypes = [vp, i64, i64, vp, vp, vp]
    L.sk_batch_create.restype = st
    L.sk_batch_create.argtypes = [ctypes.POINTER(sk_batch_item), i32, i32, ctypes.POINTER(vp)]
    L.sk_batch_set.restype = st
    L.sk_batch_set.argtypes = [vp, i32, i64]
    L.sk_batch_rebind.restype = st
    L.sk_batch_rebind.argtypes = [vp, ctypes.POINTER(sk_batch_item), i32]
    L.sk_solve_sketched.restype = st
    L.sk_solve_sketched.argtypes = [vp, vp, i64, i64, vp, vp]
    L.sk_batch_launch.restype = st
    L.sk_batch_launch.argtypes = [vp, vp]
    L.sk_batch_info.restype = st
    L.sk_batch_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.sk_batch_destroy.restype = None
    L.sk_batch_destroy.argtypes = [vp]
    L.sk_destroy.restype = None
    L.sk_destroy.argtypes = [vp]
    L.sk_apply_noalloc.restype = st
    L.sk_apply_noalloc.argtypes = [vp, vp, i64, i64, vp, vp]
    L.sk_apply_typed.restype = st
    L.sk_apply_typed.argtypes = [vp, vp, i32, i64, i64, vp, vp]
    L.sk_apply_partials.restype = st
    L.sk_apply_partials.argtypes = [vp, vp, i64, i64, vp, i64, i64, vp]
    L.sk_finish_partials.restype = st
    L.sk_finish_partials.argtypes = [vp, vp, i64, i64, i64, vp, vp]
    _lib = L
    return L


def check(status: int) -> None:
    if status != SK_OK:
        raise SkError(status, load().sk_last_error().decode(errors="replace"))


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


# ----------------------------------------------------------------------------- raw C-ABI mirrors
def sk_version() -> int:
    return load().sk_version()


def sk_last_error() -> str:
    return load().sk_last_error().decode(errors="replace")


def sk_plan_create(d: int, m: int, k: int, rule: int, seed: int) -> int:
    out = ctypes.c_void_p()
    check(load().sk_plan_create(d, m, k, rule, seed & (2**64 - 1), ctypes.byref(out)))
    return out.value


def sk_plan_set(plan: int, key: int, value: int) -> None:
    check(load().sk_plan_set(plan, key, value))


def sk_plan_get(plan: int, key: int) -> int:
    v = ctypes.c_int64()
    check(load().sk_plan_get(plan, key, ctypes.byref(v)))
    return v.value


def sk_apply(plan: int, A, lda: int, n: int, Y, stream=None) -> None:
    check(load().sk_apply(plan, _ptr(A), lda, n, _ptr(Y), _stream_handle(stream)))


def sk_apply_typed(plan: int, A, a_type: int, lda: int, n: int, Y, stream=None) -> None:
    check(load().sk_apply_typed(plan, _ptr(A), a_type, lda, n, _ptr(Y), _stream_handle(stream)))


def sk_apply_host(plan: int, A_host_ptr: int, lda: int, n: int, Y_host_ptr: int, stream=None) -> None:
    check(load().sk_apply_host(plan, A_host_ptr, lda, n, Y_host_ptr, _stream_handle(stream)))


def sk_solve(plan: int, A, lda: int, n: int, b, x, stream=None) -> None:
    check(load().sk_solve(plan, _ptr(A), lda, n, _ptr(b), _ptr(x), _stream_handle(stream)))


def sk_solve_sketched(plan: int, SAb, ld: int, n: int, x, stream=None) -> None:
    check(load().sk_solve_sketched(plan, _ptr(SAb), ld, n, _ptr(x), _stream_handle(stream)))


def sk_solve_status(plan: int, stream=None) -> tuple[int, float]:
    kap = ctypes.c_double()
    s = load().sk_solve_status(plan, ctypes.byref(kap), _stream_handle(stream))
    return s, kap.value


def sk_solve_precond(plan: int, A, lda: int, n: int, b, x, max_iters: int = 0, tol: float = 0.0,
                     stream=None) -> int:
    """Sketch-and-precondition least squares into x (n doubles); returns the iterations used."""
    it = ctypes.c_int32(0)
    check(load().sk_solve_precond(plan, _ptr(A), lda, n, _ptr(b), _ptr(x), int(max_iters), float(tol),
                                  ctypes.byref(it), _stream_handle(stream)))
    return it.value


def sk_materialize_S(plan: int, i0: int, cnt: int, rows, signs, stream=None) -> None:
    check(load().sk_materialize_S(plan, i0, cnt, _ptr(rows), _ptr(signs), _stream_handle(stream)))


def _batch_items(items: list[dict]):
    arr = (sk_batch_item * len(items))()
    for q, it in enumerate(items):
        arr[q].A_dev = _ptr(it["A"])
        arr[q].Y_dev = _ptr(it["Y"])
        arr[q].m = it["m"]
        arr[q].n = it["n"]
        arr[q].lda = it.get("lda", it["n"])
        arr[q].d = it["d"]
        arr[q].k = it["k"]
        arr[q].pad_ = 0
        arr[q].seed = it.get("seed", 0) & (2**64 - 1)
    return arr


def sk_batch_create(items: list[dict], rule: int) -> int:
    arr = _batch_items(items)
    out = ctypes.c_void_p()
    check(load().sk_batch_create(arr, len(items), rule, ctypes.byref(out)))
    return out.value


def sk_batch_rebind(batch: int, items: list[dict]) -> None:
    check(load().sk_batch_rebind(batch, _batch_items(items), len(items)))


def sk_batch_set(batch: int, key: int, value: int) -> None:
    check(load().sk_batch_set(batch, key, value))


def sk_batch_launch(batch: int, stream=None) -> None:
    check(load().sk_batch_launch(batch, _stream_handle(stream)))


def sk_batch_info(batch: int) -> tuple[int, int]:
    w, b = ctypes.c_int64(), ctypes.c_int64()
    check(load().sk_batch_info(batch, ctypes.byref(w), ctypes.byref(b)))
    return w.value, b.value


def sk_batch_destroy(batch: int) -> None:
    load().sk_batch_destroy(batch)


def sk_destroy(plan: int) -> None:
    load().sk_destroy(plan)


def sk_apply_noalloc(plan: int, A, lda: int, n: int, Y, stream=None) -> None:
    """sk_apply for callers that cannot allocate device memory: the kernel's scratch is a fixed
    16 MiB static device array of the library (see include/sk.h for the limits and the rule that
    calls overlapping on the GPU race)."""
    check(load().sk_apply_noalloc(plan, _ptr(A), lda, n, _ptr(Y), _stream_handle(stream)))


def sk_apply_partials(plan: int, A, lda: int, n: int, P, t0: int, nchunks: int, stream=None) -> None:
    check(load().sk_apply_partials(plan, _ptr(A), lda, n, _ptr(P), t0, nchunks, _stream_handle(stream)))


def sk_finish_partials(plan: int, P, t0: int, nchunks: int, n: int, Y, stream=None) -> None:
    check(load().sk_finish_partials(plan, _ptr(P), t0, nchunks, n, _ptr(Y), _stream_handle(stream)))


# ----------------------------------------------------------------------------- convenience wrapper
class Plan:
    """Owns an sk_plan handle; methods take torch CUDA tensors (marshalling only)."""

    def __init__(self, d: int, m: int, k: int, rule: int | str = SK_FP32, seed: int = 0, **params):
        if isinstance(rule, str):
            rule = RULES[rule]
        self.d, self.m, self.k, self.rule, self.seed = d, m, k, rule, seed
        self.handle = sk_plan_create(d, m, k, rule, seed)
        keys = {"chunk_rows": SK_PARAM_CHUNK_ROWS, "mode": SK_PARAM_MODE, "row_offset": SK_PARAM_ROW_OFFSET,
                "kernel": SK_PARAM_KERNEL, "tile_cols": SK_PARAM_TILE_COLS, "threads": SK_PARAM_THREADS,
                "solve_group_rows": SK_PARAM_SOLVE_GROUP_ROWS, "list_cap": SK_PARAM_LIST_CAP,
                "scratch_limit": SK_PARAM_SCRATCH_LIMIT, "solve_wait_cycles": SK_PARAM_SOLVE_WAIT_CYCLES}
        for name, v in params.items():
            sk_plan_set(self.handle, keys[name], int(v))

    def set(self, key: int, value: int) -> None:
        sk_plan_set(self.handle, key, value)

    def get(self, key: int) -> int:
        return sk_plan_get(self.handle, key)

    def out_dtype(self):
        import torch
        if self.rule == SK_FP32:
            return torch.float32
        return torch.bfloat16 if self.rule == SK_BF16_RN else torch.float16

    def apply(self, A, Y=None, stream=None):
        """Y = S A for a CUDA matrix A of float32, float16 or bfloat16 (16-bit A: sk_apply_typed)."""
        import torch
        a_types = {torch.float32: SK_A_FP32, torch.float16: SK_A_FP16, torch.bfloat16: SK_A_BF16}
        if A.dtype not in a_types or not A.is_cuda or A.dim() != 2 or A.stride(1) != 1:
            raise ValueError("A must be a CUDA float32, float16 or bfloat16 matrix with unit column stride")
        n = A.shape[1]
        if Y is None:
            Y = torch.empty((self.d, n), dtype=self.out_dtype(), device=A.device)
        if A.dtype == torch.float32:
            sk_apply(self.handle, A, A.stride(0), n, Y, stream)
        else:
            sk_apply_typed(self.handle, A, a_types[A.dtype], A.stride(0), n, Y, stream)
        return Y

    def solve(self, A, b, x=None, stream=None):
        import torch
        n = A.shape[1]
        if x is None:
            x = torch.empty(n, dtype=torch.float32, device=A.device)
        sk_solve(self.handle, A, A.stride(0), n, b, x, stream)
        return x

    def solve_precond(self, A, b, x=None, max_iters: int = 0, tol: float = 0.0, stream=None):
        """(x as float64, iterations) of the sketch-and-precondition least-squares solve."""
        import torch
        n = A.shape[1]
        if x is None:
            x = torch.empty(n, dtype=torch.float64, device=A.device)
        it = sk_solve_precond(self.handle, A, A.stride(0), n, b, x, max_iters, tol, stream)
        return x, it

    def solve_status(self, stream=None):
        return sk_solve_status(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            sk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
