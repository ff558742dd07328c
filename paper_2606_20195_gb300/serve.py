"""Continuous-batching server for sketch-and-solve least-squares requests (libsk C ABI).

Requests arrive over time (a Poisson stream in the benchmark). The server keeps a fixed number of
slots, each a CUDA stream, and an HBM budget. A waiting request is admitted as soon as a slot is free
and its device footprint fits the budget; admitted requests run concurrently on their streams, so
requests that arrive while others are on the GPU overlap with them. Plans (and the device scratch
they own: sketches, FP64 QR workspace, chunk buffers) are cached per (d, k, rule) and reused by later
requests of any height (SK_PARAM_ROWS sets a request's m on the cached plan), so once the scratch has
grown to the largest request seen, serving allocates no device memory: a cudaMalloc in the middle of
the stream would synchronize every slot's stream. Latency is measured from arrival to the moment x is
ready.

Device memory for requests comes from one arena: a buffer the size of the HBM budget, allocated when
the server starts, in which every admitted request's A, b and x get a range (first fit, freed when
the request completes). Admission needs both a free slot and a range; serving itself never calls the
CUDA allocator, whose cudaMalloc / cudaFree of multi-GB blocks would synchronize every slot's stream.

Each request's matrix is materialized on the device by a seeded generator when it is admitted
(synthetic workloads; the same families the tests and benchmarks use). That generation stands in for
the client's data arriving and is part of the request's service time; a host-to-device upload is not
modelled (at the host link's ~210 GB/s it would dominate every request larger than a few MB).
"""
from __future__ import annotations

import dataclasses
import heapq
import math
import time
from typing import Callable

import numpy as np

from . import inputs
from . import sk as skb


@dataclasses.dataclass
class Request:
    rid: int
    m: int
    n: int
    d: int
    k: int
    rule: int
    family: str
    seed: int
    arrival: float = 0.0          # seconds from the start of the stream
    # filled by the server
    admitted: float = math.nan
    done: float = math.nan
    x: object = None
    status: int = -1
    kappa: float = math.nan

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def footprint_bytes(req: Request) -> int:
    """Device bytes a request holds while admitted: A, b and x."""
    return req.m * req.n * 4 + req.m * 4 + req.n * 4


def plan_scratch_bytes(req: Request) -> int:
    """Estimate of the device scratch a plan needs for a request (before it has run): sketches, FP64
    QR workspace, chunk totals. After a request the server reads the plan's actual scratch instead."""
    es = 4 if req.rule == skb.SK_FP32 else 2
    sketches = req.d * (req.n + 1) * es
    qr = 8 * (2 * req.n * (req.n + 1) + 2 * req.n) + 4096
    chunks = 9 * req.d * (req.n + 1) * 4 + 4096
    return sketches + qr + chunks


def make_stream(count: int, rate_hz: float, seed: int = 0, log2_m=(14, 24), ns=(16, 32, 64, 128, 256),
                ks=(1, 4, 8), rules=(0, 1, 2, 3), families=("incoherent", "coherent"), d_per_n: int = 16):
    """Poisson arrivals at `rate_hz` of requests with m log-uniform in [2^lo, 2^hi], n, k, rule and the
    matrix family uniform over the given sets, d = d_per_n * n."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate_hz) if rate_hz > 0 else 0.0
        m = int(2.0 ** rng.uniform(*log2_m))
        n = int(rng.choice(ns))
        m = max(m, 2 * d_per_n * n)
        k = int(rng.choice(ks))
        d = d_per_n * n
        d = ((d + k - 1) // k) * k
        out.append(Request(rid=i, m=m, n=n, d=d, k=k, rule=int(rng.choice(rules)),
                           family=str(rng.choice(families)), seed=1000 + i, arrival=t))
    return out


class Arena:
    """First-fit ranges of one float32 device buffer, 256-byte aligned, coalesced on release."""

    ALIGN = 64  # floats

    def __init__(self, floats: int, device):
        import torch
        self.size = max(int(floats) // self.ALIGN * self.ALIGN, self.ALIGN)
        self.buf = torch.empty(self.size, dtype=torch.float32, device=device)
        self.free = [(0, self.size)]  # (offset, length), sorted by offset, disjoint, not adjacent

    def _round(self, n: int) -> int:
        return max((int(n) + self.ALIGN - 1) // self.ALIGN * self.ALIGN, self.ALIGN)

    def alloc(self, n: int):
        """Offset of a range of n floats, or None if no free range is long enough."""
        n = self._round(n)
        for i, (o, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    del self.free[i]
                else:
                    self.free[i] = (o + n, ln - n)
                return o
        return None

    def release(self, o: int, n: int) -> None:
        n = self._round(n)
        i = 0
        while i < len(self.free) and self.free[i][0] < o:
            i += 1
        self.free.insert(i, (o, n))
        # merge with the next and the previous range when they touch
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (o, self.free[i][1] + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]

    def view(self, o: int, shape):
        numel = 1
        for v in shape:
            numel *= v
        return self.buf[o:o + numel].view(*shape)

    def free_floats(self) -> int:
        return sum(ln for _, ln in self.free)


class Server:
    def __init__(self, slots: int = 8, hbm_budget_bytes: int = 120 * 10**9, device: str = "cuda:0",
                 deterministic: bool = False, keep_results: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.slots = slots
        self.budget = int(hbm_budget_bytes)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.used_bytes = 0
        self.plans: dict = {}        # (d, k, rule) -> list of [Plan, busy, scratch bytes]
        self.resident_bytes = 0      # device scratch kept by cached plans
        self.deterministic = deterministic
        self.keep_results = keep_results
        self.peak_bytes = 0
        self.arena = Arena(self.budget // 4, self.device)

    # ------------------------------------------------------------------ plans
    def _plan(self, req: Request):
        key = (req.d, req.k, req.rule)
        pool = self.plans.setdefault(key, [])
        for idx, entry in enumerate(pool):
            if not entry[1]:
                entry[1] = True
                entry[0].set(skb.SK_PARAM_ROWS, req.m)
                return entry[0], (key, idx)
        mode = skb.SK_MODE_DETERMINISTIC if self.deterministic else skb.SK_MODE_ATOMIC
        # The sketch seed is derived from (d, k, rule), so a cached plan serves every request of them.
        seed = (req.d * 1000003 + req.k * 13 + req.rule) & 0xFFFFFFFF
        plan = skb.Plan(req.d, req.m, req.k, req.rule, seed=seed, mode=mode)
        est = plan_scratch_bytes(req)
        pool.append([plan, True, est])
        self.resident_bytes += est
        return plan, (key, len(pool) - 1)

    def _release_plan(self, key):
        entry = self.plans[key[0]][key[1]]
        entry[1] = False
        actual = entry[0].get(skb.SK_PARAM_SCRATCH_BYTES)  # what the plan holds now
        self.resident_bytes += actual - entry[2]
        entry[2] = actual

    # ------------------------------------------------------------------ one request
    @staticmethod
    def _xs_offset(n: int) -> int:
        """Offset of x* within the x range: x, then x* at the next aligned position."""
        return Arena.ALIGN * ((n + Arena.ALIGN - 1) // Arena.ALIGN)

    def _place(self, req: Request):
        """Arena ranges for A (m x n), b (m) and x followed by x* (each at an aligned start); None if
        they do not all fit."""
        got = []
        for numel in (req.m * req.n, req.m, self._xs_offset(req.n) + req.n):
            o = self.arena.alloc(numel)
            if o is None:
                for o2, n2 in got:
                    self.arena.release(o2, n2)
                return None
            got.append((o, numel))
        return got

    def _launch(self, req: Request, slot: int, ranges):
        torch = self.torch
        st = self.streams[slot]
        (oa, _), (ob, _), (ox, _) = ranges
        A = self.arena.view(oa, (req.m, req.n))
        b = self.arena.view(ob, (req.m,))
        x = self.arena.view(ox, (req.n,))
        xs = self.arena.view(ox + self._xs_offset(req.n), (req.n,))
        with torch.cuda.stream(st):
            inputs.fill_device_matrix(A, req.family, seed=req.seed)
            g = torch.Generator(device=self.device)
            g.manual_seed(req.seed + 7)
            torch.randn(req.n, generator=g, out=xs)
            torch.randn(req.m, generator=g, out=b)
            b.mul_(1e-6).addmv_(A, xs)  # b = A x* + 1e-6 N(0, 1)
            plan, key = self._plan(req)
            skb.sk_solve(plan.handle, A, req.n, req.n, b, x, st)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"req": req, "slot": slot, "ranges": ranges, "x": x, "plan": plan, "key": key, "event": ev}

    def _finish(self, job, now: float):
        req = job["req"]
        req.done = now
        status, kappa = job["plan"].solve_status(self.streams[job["slot"]])
        req.status, req.kappa = status, kappa
        if self.keep_results:
            req.x = job["x"].cpu()
        for o, numel in job["ranges"]:
            self.arena.release(o, numel)
        self._release_plan(job["key"])
        self.free_slots.append(job["slot"])
        self.used_bytes -= footprint_bytes(req)

    # ------------------------------------------------------------------ serving loops
    def run(self, requests: list[Request], clock: Callable[[], float] = time.perf_counter,
            poll_s: float = 2e-5) -> dict:
        """Continuous batching: admit as slots and budget free up, overlap admitted requests."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            if footprint_bytes(r) + plan_scratch_bytes(r) > self.budget:
                raise ValueError(f"request {r.rid} needs {footprint_bytes(r)} B, above the HBM budget")
        waiting: list = []
        running: list = []
        i = 0
        t0 = clock()
        while i < len(pending) or waiting or running:
            now = clock() - t0
            while i < len(pending) and pending[i].arrival <= now:
                heapq.heappush(waiting, (pending[i].arrival, pending[i].rid, pending[i]))
                i += 1
            # completions
            still = []
            for job in running:
                if job["event"].query():
                    self._finish(job, clock() - t0)
                else:
                    still.append(job)
            running = still
            # admissions (FIFO by arrival; a request that does not fit waits for memory)
            while waiting and self.free_slots:
                req = waiting[0][2]
                fb = footprint_bytes(req)
                if self.used_bytes + self.resident_bytes + fb + plan_scratch_bytes(req) > self.budget:
                    if running:
                        break
                    self._evict_idle_plans()
                    if self.used_bytes + self.resident_bytes + fb + plan_scratch_bytes(req) > self.budget:
                        break
                ranges = self._place(req)
                if ranges is None:  # no contiguous range in the arena yet: wait for completions
                    break
                heapq.heappop(waiting)
                slot = self.free_slots.pop(0)
                self.used_bytes += fb
                self.peak_bytes = max(self.peak_bytes, self.used_bytes + self.resident_bytes)
                req.admitted = clock() - t0
                running.append(self._launch(req, slot, ranges))
            if not running and not waiting and i < len(pending):
                # idle until the next arrival
                delay = pending[i].arrival - (clock() - t0)
                if delay > 0:
                    time.sleep(min(delay, 0.01))
            elif running:
                time.sleep(poll_s)
        torch.cuda.synchronize(self.device)
        return summarize(requests, clock() - t0)

    def run_one_at_a_time(self, requests: list[Request], clock: Callable[[], float] = time.perf_counter) -> dict:
        """Baseline: FIFO, one request on the GPU at a time, on one stream."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        for req in pending:
            now = clock() - t0
            if req.arrival > now:
                time.sleep(req.arrival - now)
            self.used_bytes += footprint_bytes(req)
            req.admitted = clock() - t0
            ranges = self._place(req)
            if ranges is None:
                raise ValueError(f"request {req.rid} does not fit in the arena")
            job = self._launch(req, self.free_slots.pop(0), ranges)
            job["event"].synchronize()
            self._finish(job, clock() - t0)
        return summarize(requests, clock() - t0)

    def _evict_idle_plans(self):
        """Release the scratch of cached plans that no running request uses."""
        for key in list(self.plans):
            keep = []
            for entry in self.plans[key]:
                if entry[1]:
                    keep.append(entry)
                else:
                    entry[0].close()
                    self.resident_bytes -= entry[2]
            self.plans[key] = keep
        self.resident_bytes = max(self.resident_bytes, 0)

    def close(self):
        for pool in self.plans.values():
            for entry in pool:
                entry[0].close()
        self.plans.clear()
        self.resident_bytes = 0
        self.arena = None


def summarize(requests: list[Request], wall_s: float) -> dict:
    lat = np.array([r.latency for r in requests], dtype=np.float64) * 1e3
    ok = sum(1 for r in requests if r.status == skb.SK_OK)
    return {"requests": len(requests), "ok": ok, "wall_s": wall_s,
            "solves_per_s": len(requests) / wall_s if wall_s > 0 else float("nan"),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
