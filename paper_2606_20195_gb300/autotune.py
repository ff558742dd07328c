"""Autotuner for the tile kernels: threads per CTA, columns per work item and chunk length.

For a single-matrix plan it tries the candidate (threads, tile columns) pairs on the caller's data;
for a batch it tries (threads, tile columns, chunk-length scale) on the batch itself. Each candidate
is timed with CUDA events over a few launches after a warm-up, and the fastest is kept. Results are
cached in a JSON file keyed by the shape signature, so later runs of the same shapes skip the search.
The cache path is $SK_TUNE_CACHE or ~/.cache/sk_tune.json.

Chunk length is part of the result's definition for the FP16 rules (it sets how many rounded
contributions each output receives), so the single-matrix tuner keeps it fixed at the plan's value
and tunes only the launch shape; the batch tuner may scale it within the accuracy limit of at most
32 chunks per matrix.
"""
from __future__ import annotations

import json
import os
import threading

from . import sk as skb

_lock = threading.Lock()
THREADS = (256, 512, 1024)
TILE_COLS = (0, 4, 8, 16, 32)


def cache_path() -> str:
    return os.environ.get("SK_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sk_tune.json"))


def _load() -> dict:
    p = cache_path()
    if os.path.exists(p):
        try:
            with open(p) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _store(key: str, value: dict) -> None:
    with _lock:
        db = _load()
        db[key] = value
        p = cache_path()
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, p)


def _time_ms(fn, reps: int = 5, warmup: int = 2) -> float:
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune_plan(plan: "skb.Plan", A, reps: int = 5, use_cache: bool = True) -> dict:
    """Pick threads and tile columns for `plan` on matrix A (torch CUDA tensor); applies them."""
    import torch
    n = A.shape[1]
    key = f"plan:d{plan.d}:m{plan.m}:k{plan.k}:n{n}:r{plan.rule}:R{plan.get(skb.SK_PARAM_CHUNK_ROWS)}"
    if use_cache:
        hit = _load().get(key)
        if hit:
            plan.set(skb.SK_PARAM_THREADS, hit["threads"])
            plan.set(skb.SK_PARAM_TILE_COLS, hit["tile_cols"])
            return hit
    Y = torch.empty((plan.d, n), dtype=plan.out_dtype(), device=A.device)
    best = None
    for thr in THREADS:
        for cols in TILE_COLS:
            try:
                plan.set(skb.SK_PARAM_THREADS, thr)
                plan.set(skb.SK_PARAM_TILE_COLS, cols)
                ms = _time_ms(lambda: plan.apply(A, Y), reps=reps)
            except skb.SkError:
                continue
            if best is None or ms < best["ms"]:
                best = {"threads": thr, "tile_cols": cols, "ms": ms}
    if best is None:
        raise RuntimeError("no tile configuration ran")
    plan.set(skb.SK_PARAM_THREADS, best["threads"])
    plan.set(skb.SK_PARAM_TILE_COLS, best["tile_cols"])
    _store(key, best)
    return best


def batch_signature(items: list[dict], rule: int) -> str:
    parts = sorted((it["m"], it["n"], it["d"], it["k"]) for it in items)
    h = 0
    for p in parts:
        h = (h * 1000003 + hash(p)) & 0xFFFFFFFFFFFF
    return f"batch:{len(items)}:r{rule}:{h:x}"


def tune_batch(items: list[dict], rule: int, reps: int = 3, use_cache: bool = True,
               scales=(1.0, 2.0, 4.0)) -> tuple[int, dict]:
    """Build the best batch for `items`: returns (batch handle, chosen parameters)."""
    key = batch_signature(items, rule)
    cand = []
    if use_cache and _load().get(key):
        c = _load()[key]
        cand = [(c["threads"], c["tile_cols"], c["chunk_rows"])]
    else:
        base = max(it["m"] for it in items)
        for thr in THREADS:
            for cols in (0, 8, 16):
                for sc in scales:
                    # chunk rows relative to the automatic choice (0 keeps it)
                    R = 0 if sc == 1.0 else max(256, int(sc * base / 32) // 256 * 256)
                    cand.append((thr, cols, R))
    best, best_b = None, None
    for thr, cols, R in cand:
        b = skb.sk_batch_create(items, rule)
        try:
            skb.sk_batch_set(b, skb.SK_PARAM_THREADS, thr)
            skb.sk_batch_set(b, skb.SK_PARAM_TILE_COLS, cols)
            skb.sk_batch_set(b, skb.SK_PARAM_CHUNK_ROWS, R)
            ms = _time_ms(lambda: skb.sk_batch_launch(b), reps=reps, warmup=1)
        except skb.SkError:
            skb.sk_batch_destroy(b)
            continue
        if best is None or ms < best["ms"]:
            if best_b is not None:
                skb.sk_batch_destroy(best_b)
            best, best_b = {"threads": thr, "tile_cols": cols, "chunk_rows": R, "ms": ms}, b
        else:
            skb.sk_batch_destroy(b)
    if best is None:
        raise RuntimeError("no batch configuration ran")
    _store(key, best)
    return best_b, best
