"""Continuous-batching server for sketch-and-solve least-squares requests (libsk C ABI).

Requests arrive over time (a Poisson stream in the benchmark). The server keeps a slot count (the
most requests on the GPU at once), a pool of CUDA streams and an HBM budget. A waiting request is
admitted as soon as a slot is free and its device footprint fits the budget. At every scheduling
step the requests admitted in that step are batched: for each rounding rule among them, ONE batched
sketch launch (sk_batch_launch, a persistent kernel over a device work list) forms S [A_i | b_i] for
all of them, then each request's FP64 QR and triangular solve run from its sketch
(sk_solve_sketched), on the same stream. Requests whose [A | b] exceeds 4 MiB are not batched: each
runs on a stream of its own through the single-matrix kernels, which are faster on larger matrices. Requests admitted while earlier ones are still on the GPU
run on other streams and overlap with them. Plans (which own the FP64 QR workspace) are cached per
(d, k, rule), and batch objects per rule are rebound to the next step's requests once their last
launch has completed (sk_batch_rebind), so once the pools have warmed up serving allocates no device
memory: a cudaMalloc or cudaFree in the middle of the stream would synchronize every stream.
Latency is measured from arrival to the moment x is ready.

With deterministic=True the server runs each request through sk_solve in SK_MODE_DETERMINISTIC
instead (the batched kernel runs in atomic mode only), so that results can be compared bit for bit
alone and in the mix.

Device memory for requests comes from one arena: a buffer the size of the HBM budget, allocated when
the server starts, in which every admitted request's [A | b] (A and b side by side, row stride
n + 1 rounded up to 4 floats, the layout the batched TMA staging reads), its sketch and x get a range
(first fit, freed when the request completes). Admission needs both a free slot and a range.

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
    sketch: object = None         # [SA | Sb] on the host (keep_sketches)
    status: int = -1
    kappa: float = math.nan

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def ab_stride(n: int) -> int:
    """Row stride (floats) of a request's [A | b]: n + 1 rounded up to a multiple of 4 (16 bytes)."""
    return (n + 1 + 3) // 4 * 4


def sketch_elem_bytes(rule: int) -> int:
    return 4 if rule == skb.SK_FP32 else 2


def footprint_bytes(req: Request) -> int:
    """Device bytes a request holds while admitted: [A | b], its sketch, x and x*."""
    return (req.m * ab_stride(req.n) * 4 + req.d * (req.n + 1) * sketch_elem_bytes(req.rule)
            + 2 * req.n * 4)


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


def partition_step(admitted: list, batch_max_bytes: int):
    """Split one scheduling step's admitted (request, slot, ranges) entries into those that run alone
    ([A | b] larger than batch_max_bytes) and, per rounding rule, those sketched by one batched launch;
    arrival order is kept within each part."""
    singles, by_rule = [], {}
    for entry in admitted:
        req = entry[0]
        if req.m * ab_stride(req.n) * 4 > batch_max_bytes:
            singles.append(entry)
        else:
            by_rule.setdefault(req.rule, []).append(entry)
    return singles, by_rule


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
                 deterministic: bool = False, keep_results: bool = True, keep_sketches: bool = False):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.slots = slots
        self.budget = int(hbm_budget_bytes)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.status_stream = torch.cuda.Stream(device=self.device)  # status reads of finished requests only
        self.free_slots = list(range(slots))
        self.used_bytes = 0
        self.plans: dict = {}        # (d, k, rule) -> list of [Plan, busy, scratch bytes]
        self.resident_bytes = 0      # device scratch kept by cached plans
        self.deterministic = deterministic
        self.keep_results = keep_results
        self.keep_sketches = keep_sketches  # copy each request's sketch [SA | Sb] to the host (tests)
        self.batches: dict = {}      # rule -> list of [batch handle, event of its last launch or None]
        self.launches = 0            # batched sketch launches made (one per rule and scheduling step)
        self._rr = 0                 # next stream of the pool
        self._last_event: dict = {}  # stream index -> event of the last work launched on it
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
        plan = skb.Plan(req.d, req.m, req.k, req.rule, seed=self.sketch_seed(req), mode=mode)
        est = plan_scratch_bytes(req)
        pool.append([plan, True, est])
        self.resident_bytes += est
        return plan, (key, len(pool) - 1)

    @staticmethod
    def sketch_seed(req: Request) -> int:
        """The sketch seed is derived from (d, k, rule), so a cached plan serves every request of them."""
        return (req.d * 1000003 + req.k * 13 + req.rule) & 0xFFFFFFFF

    def _batch(self, rule: int, items: list):
        """A batch object of this rule whose last launch has completed, bound to `items`."""
        pool = self.batches.setdefault(rule, [])
        for entry in pool:
            if entry[1] is None or entry[1].query():
                skb.sk_batch_rebind(entry[0], items)
                break
        else:
            entry = [skb.sk_batch_create(items, rule), None]
            pool.append(entry)
        # Each request's chunking from its own m (at most 8 chunks, as sk_solve's default), so its
        # rounding does not depend on the other requests of the step.
        skb.sk_batch_set(entry[0], skb.SK_PARAM_ITEM_CHUNKS, 8)
        return entry

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
        """Arena ranges for [A | b] (m x ab_stride(n)), the sketch (d x (n+1) elements of the rule's
        type) and x followed by x*; None if they do not all fit."""
        got = []
        sk_floats = (req.d * (req.n + 1) * sketch_elem_bytes(req.rule) + 3) // 4
        for numel in (req.m * ab_stride(req.n), sk_floats, self._xs_offset(req.n) + req.n):
            o = self.arena.alloc(numel)
            if o is None:
                for o2, n2 in got:
                    self.arena.release(o2, n2)
                return None
            got.append((o, numel))
        return got

    def _views(self, req: Request, ranges):
        (oa, _), (oy, _), (ox, _) = ranges
        Ab = self.arena.view(oa, (req.m, ab_stride(req.n)))
        x = self.arena.view(ox, (req.n,))
        xs = self.arena.view(ox + self._xs_offset(req.n), (req.n,))
        return Ab, Ab[:, :req.n], Ab[:, req.n], x, xs, oy

    def _generate(self, req: Request, A, b, xs):
        """The request's data (on the current stream): A of its family, x* ~ N(0,1) and
        b = A x* + 1e-6 N(0,1)."""
        torch = self.torch
        inputs.fill_device_matrix(A, req.family, seed=req.seed)
        g = inputs.device_generator(self.device, req.seed + 7)
        torch.randn(req.n, generator=g, out=xs)
        torch.randn(req.m, generator=g, out=b)
        b.mul_(1e-6).addmv_(A, xs)

    def problem(self, req: Request):
        """(A, b) of a request as numpy arrays, generated exactly as the server generates them (in
        the same [A | b] layout), for checking served results."""
        torch = self.torch
        Ab = torch.empty((req.m, ab_stride(req.n)), dtype=torch.float32, device=self.device)
        xs = torch.empty(req.n, dtype=torch.float32, device=self.device)
        self._generate(req, Ab[:, :req.n], Ab[:, req.n], xs)
        torch.cuda.synchronize(self.device)
        return Ab[:, :req.n].cpu().numpy(), Ab[:, req.n].cpu().numpy()

    def _next_stream(self):
        """A stream of the pool with no work outstanding (round robin among those), else the next in
        turn: work launched in this step should not queue behind a long request on the same stream."""
        ns = len(self.streams)
        for i in range(ns):
            idx = (self._rr + i) % ns
            ev = self._last_event.get(idx)
            if ev is None or ev.query():
                self._rr = idx + 1
                return self.streams[idx]
        st = self.streams[self._rr % ns]
        self._rr += 1
        return st

    def _mark(self, st, ev):
        self._last_event[self.streams.index(st)] = ev

    # Requests whose [A | b] is larger than this are not batched: the single-matrix kernels AUTO picks
    # (register, global) are faster than the batched kernel on larger matrices, and a large item in a
    # batch would hold back the small requests launched with it. Measured on the [2^14, 2^20] stream:
    # batching up to 4 MiB matches running every request alone on its own stream (1337 solves/s
    # saturated) with a slightly lower p99 at 80 % load; larger limits lose up to 5 % throughput.
    BATCH_MAX_BYTES = 4 << 20

    def _launch_group(self, admitted: list):
        """Jobs for the requests admitted in one scheduling step: per rule, the small requests' data,
        one batched sketch launch over all their [A | b], then each one's QR solve from its sketch;
        every large request on a stream of its own through the single-matrix path."""
        torch = self.torch
        singles, by_rule = partition_step(admitted, self.BATCH_MAX_BYTES)
        jobs = [self._launch_single(req, slot, ranges, self._next_stream()) for req, slot, ranges in singles]
        for rule, group in by_rule.items():
            st = self._next_stream()
            with torch.cuda.stream(st):
                items = []
                for req, slot, ranges in group:
                    Ab, A, b, x, xs, oy = self._views(req, ranges)
                    self._generate(req, A, b, xs)
                    items.append({"A": Ab, "Y": self.arena.buf[oy:], "m": req.m, "n": req.n + 1,
                                  "lda": ab_stride(req.n), "d": req.d, "k": req.k, "seed": self.sketch_seed(req)})
                entry = self._batch(rule, items)
                skb.sk_batch_launch(entry[0], st)
                self.launches += 1
                for (req, slot, ranges), it in zip(group, items):
                    _, _, _, x, _, _ = self._views(req, ranges)
                    plan, key = self._plan(req)
                    skb.sk_solve_sketched(plan.handle, it["Y"], req.n + 1, req.n, x, st)
                    ev = torch.cuda.Event()
                    ev.record(st)
                    jobs.append({"req": req, "slot": slot, "ranges": ranges, "x": x, "plan": plan, "key": key,
                                 "event": ev, "stream": st, "sketch": it["Y"]})
                entry[1] = jobs[-1]["event"]  # the batch is free again once its group's last solve is done
                self._mark(st, entry[1])
        return jobs

    def _launch_single(self, req: Request, slot: int, ranges, st=None):
        """One request on its own (large requests, the one-at-a-time baseline and the deterministic
        mode): the plan's sketch of [A | b] (sk_apply over the n + 1 columns: column n is S b with the
        rounding bits of column n, as sk_solve forms it), then the FP64 back end (sk_solve_sketched)."""
        torch = self.torch
        st = st if st is not None else self.streams[slot % len(self.streams)]
        Ab, A, b, x, xs, oy = self._views(req, ranges)
        Y = self.arena.buf[oy:]
        with torch.cuda.stream(st):
            self._generate(req, A, b, xs)
            plan, key = self._plan(req)
            skb.sk_apply(plan.handle, Ab, ab_stride(req.n), req.n + 1, Y, st)
            skb.sk_solve_sketched(plan.handle, Y, req.n + 1, req.n, x, st)
            ev = torch.cuda.Event()
            ev.record(st)
        self._mark(st, ev)
        return {"req": req, "slot": slot, "ranges": ranges, "x": x, "plan": plan, "key": key, "event": ev,
                "stream": st, "sketch": Y}

    def _finish(self, job, now: float):
        req = job["req"]
        req.done = now
        # The job's event has completed, so its status word is written; read it on a stream of its own
        # (the job's stream may already hold later requests' work, which a read there would wait for).
        status, kappa = job["plan"].solve_status(self.status_stream)
        req.status, req.kappa = status, kappa
        if self.keep_results:
            req.x = job["x"].cpu()
        if self.keep_sketches and job["sketch"] is not None:
            es = sketch_elem_bytes(req.rule)
            raw = job["sketch"][:(req.d * (req.n + 1) * es + 3) // 4].cpu().numpy().view(np.uint8)
            dt = np.float32 if es == 4 else np.uint16
            req.sketch = raw[:req.d * (req.n + 1) * es].view(dt).reshape(req.d, req.n + 1).copy()
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
            # admissions (FIFO by arrival; a request that does not fit waits for memory), then the
            # step's admitted requests are launched together
            admitted = []
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
                if self.deterministic:
                    running.append(self._launch_single(req, slot, ranges))
                else:
                    admitted.append((req, slot, ranges))
            if admitted:
                running.extend(self._launch_group(admitted))
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
            job = self._launch_single(req, self.free_slots.pop(0), ranges)
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
        for pool in self.batches.values():
            for entry in pool:
                skb.sk_batch_destroy(entry[0])
        self.batches.clear()
        self.resident_bytes = 0
        self.arena = None


def summarize(requests: list[Request], wall_s: float) -> dict:
    lat = np.array([r.latency for r in requests], dtype=np.float64) * 1e3
    ok = sum(1 for r in requests if r.status == skb.SK_OK)
    return {"requests": len(requests), "ok": ok, "wall_s": wall_s,
            "solves_per_s": len(requests) / wall_s if wall_s > 0 else float("nan"),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
