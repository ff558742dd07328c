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
