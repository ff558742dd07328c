"""The server's HBM arena (first-fit ranges of one buffer), exercised on a CPU buffer: allocation,
alignment, exhaustion, release with coalescing, and reuse of a coalesced range."""
from paper_2606_20195_gb300 import serve


def test_arena_first_fit_alignment_and_coalescing():
    U = serve.Arena.ALIGN
    ar = serve.Arena(U * 10, "cpu")
    a = ar.alloc(1)        # rounded up to one unit
    b = ar.alloc(2 * U + 2)  # three units
    c = ar.alloc(U)
    assert (a, b, c) == (0, U, 4 * U)
    assert ar.free == [(5 * U, 5 * U)]
    assert ar.alloc(6 * U) is None           # more than what is left
    ar.release(b, 2 * U + 2)                 # a three-unit hole between a and c
    assert ar.free == [(U, 3 * U), (5 * U, 5 * U)]
    d = ar.alloc(4 * U)                      # first fit skips the hole, takes the tail
    assert d == 5 * U
    ar.release(a, 1)                         # the hole grows to four units at offset 0
    assert ar.free == [(0, 4 * U), (9 * U, U)]
    e = ar.alloc(4 * U)
    assert e == 0
    for o, n in ((e, 4 * U), (c, U), (d, 4 * U)):
        ar.release(o, n)
    assert ar.free == [(0, 10 * U)]          # everything merged back into one range
    assert ar.free_floats() == 10 * U
    v = ar.view(ar.alloc(12), (3, 4))
    assert tuple(v.shape) == (3, 4)


def test_x_and_xstar_stay_inside_their_range():
    # A request's x and x* share one arena range: x at its start, x* at the next aligned offset. The
    # range must hold both, or x* would overwrite whatever the arena placed after it (another
    # request's A or b while both run).
    srv = object.__new__(serve.Server)  # placement only: no streams, no device
    srv.arena = serve.Arena(serve.Arena.ALIGN * 40000, "cpu")
    for n in (1, 16, 32, 63, 64, 65, 100, 256):
        req = serve.Request(rid=0, m=128, n=n, d=16 * n, k=4, rule=0, family="incoherent", seed=0)
        ranges = srv._place(req)
        (ox, nx) = ranges[2]
        assert srv._xs_offset(n) >= n                        # x* starts after x
        assert srv._xs_offset(n) + n <= srv.arena._round(nx)  # and ends inside the range
        for o, numel in ranges:
            srv.arena.release(o, numel)


def test_partition_step_by_size_and_rule():
    # One scheduling step: requests whose [A | b] exceeds the limit run alone; the others are grouped
    # by rounding rule (one batched launch each), in arrival order.
    def req(rid, m, n, rule):
        return serve.Request(rid=rid, m=m, n=n, d=16 * n, k=4, rule=rule, family="incoherent", seed=rid)
    reqs = [req(0, 1 << 20, 64, 1), req(1, 4096, 16, 1), req(2, 8192, 32, 0), req(3, 2048, 16, 1),
            req(4, 1 << 22, 16, 0), req(5, 4096, 256, 3)]
    limit = 64 << 20  # bytes of [A | b]
    admitted = [(r, r.rid, None) for r in reqs]
    singles, by_rule = serve.partition_step(admitted, limit)
    assert [e[0].rid for e in singles] == [0, 4]  # 2^20 x 68 and 2^22 x 20 floats exceed 64 MiB
    assert {rule: [e[0].rid for e in g] for rule, g in by_rule.items()} == {1: [1, 3], 0: [2], 3: [5]}
    assert serve.ab_stride(16) == 20 and serve.ab_stride(15) == 16 and serve.ab_stride(64) == 68
    singles, by_rule = serve.partition_step(admitted, 1 << 40)  # nothing too large: all batched
    assert singles == [] and sum(len(g) for g in by_rule.values()) == len(reqs)


def test_next_stream_prefers_idle_streams():
    # New work goes to a stream whose last work has completed, round robin among those; only when all
    # are busy does it queue behind one (the next in turn).
    class Ev:
        def __init__(self, done):
            self.done = done

        def query(self):
            return self.done

    srv = object.__new__(serve.Server)
    srv.streams = ["s0", "s1", "s2"]
    srv._rr = 0
    srv._last_event = {0: Ev(False), 1: Ev(True)}
    assert srv._next_stream() == "s1"          # s0 busy, s1 idle
    assert srv._next_stream() == "s2"          # never used: idle
    srv._mark("s2", Ev(False))
    srv._last_event[1] = Ev(False)
    assert srv._next_stream() == "s0"          # all busy: the next in turn (after s2 comes s0)
