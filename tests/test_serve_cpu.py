"""Host logic of the continuous-batching server, on CPU: the arrival ring
never hands out space that an event still held occupies; the rule that
forms the next batch (the longest run of pending events in arrival order
within the slot's capacity, or the oldest event's size class first); and the
arrival process."""
from collections import deque

import numpy as np
import pytest


@pytest.fixture(scope="module")
def serve():
    # the server module loads the library: build it first (host compile only)
    from paper_2402_14670_gb300 import build
    build.build()
    from paper_2402_14670_gb300 import serve as m
    return m


def test_ring_never_overlaps_held_events(serve):
    rng = np.random.default_rng(3)
    ring = serve._Ring(1000, 300, "cpu")
    held = deque()            # (virtual hit start, n hits, virtual track start, n tracks)
    placed = refused = 0
    for step in range(5000):
        if held and (rng.random() < 0.45 or len(held) > 40):
            held.popleft()    # the oldest event completes
            continue
        nh, nt = int(rng.integers(0, 120)), int(rng.integers(0, 40))
        tail = (held[0][0], held[0][2]) if held else None
        pos = ring.place(nh, nt, tail)
        if pos is None:
            assert held       # an empty ring takes any run that fits its arrays
            refused += 1
            continue
        vh, vt = pos
        ph, pt = vh % ring.cap_h, vt % ring.cap_t
        assert ph + nh <= ring.cap_h and pt + nt <= ring.cap_t        # contiguous in the arrays
        for (h0, n0, t0, m0) in held:
            a0 = h0 % ring.cap_h
            assert a0 + n0 <= ph or ph + nh <= a0 or nh == 0 or n0 == 0     # hit ranges disjoint
            c0 = t0 % ring.cap_t
            assert c0 + m0 <= pt or pt + nt <= c0 or nt == 0 or m0 == 0     # track ranges disjoint
        ring.vh, ring.vt = vh + nh, vt + nt
        held.append((vh, nh, vt, nt))
        placed += 1
    assert placed > 1000 and refused > 0


def _server(serve, nh, nt, max_events, max_hits, max_tracks, group=False):
    s = serve.Server.__new__(serve.Server)
    s.nh, s.nt = np.asarray(nh, dtype=np.int64), np.asarray(nt, dtype=np.int64)
    s.size_class = np.searchsorted(np.asarray(serve.TRACK_EDGES), s.nt, side="left")
    s.max_events, s.max_hits, s.max_tracks = max_events, max_hits, max_tracks
    s.group_by_size = group
    return s


def _pending(serve, s, events):
    p = [deque() for _ in range(len(serve.TRACK_EDGES) + 1)]
    for e in events:
        p[s._class(e)].append(e)
    return p


def _brute(nh, nt, head, avail, max_events, max_hits, max_tracks):
    """Longest run head..head+k-1 within every capacity, by trying each k."""
    best = 0
    for k in range(1, min(avail, max_events) + 1):
        if nh[head:head + k].sum() <= max_hits and nt[head:head + k].sum() <= max_tracks:
            best = k
        else:
            break
    return best


def test_take_is_the_longest_run_within_capacity(serve):
    rng = np.random.default_rng(11)
    nh = rng.integers(0, 5000, 400)
    nt = rng.integers(0, 90, 400)
    for max_events, max_hits, max_tracks in ((8, 10 ** 9, 10 ** 9), (10 ** 6, 20000, 10 ** 9),
                                             (10 ** 6, 10 ** 9, 300), (50, 40000, 700)):
        s = _server(serve, nh, nt, max_events, max(max_hits, int(nh.max())), max(max_tracks, int(nt.max())))
        for head in (0, 1, 17, 200, 399):
            for avail in sorted({1, min(3, 400 - head), 400 - head}):
                ev, taken, nbytes = s._take(_pending(serve, s, range(head, head + avail)))
                k = _brute(nh, nt, head, avail, s.max_events, s.max_hits, s.max_tracks)
                assert ev == list(range(head, head + k))
                assert nbytes == (int(nh[ev].sum()) * serve.SLOT_BYTES_PER_HIT +
                                  int(nt[ev].sum()) * serve.SLOT_BYTES_PER_TRACK)


def test_take_counts_empty_events_and_refuses_an_event_above_capacity(serve):
    # empty events cost nothing, so they ride along up to the event capacity
    s = _server(serve, [0, 0, 0, 10, 0], [0, 2, 0, 1, 0], 4, 10, 3)
    assert s._take(_pending(serve, s, range(5)))[0] == [0, 1, 2, 3]
    s = _server(serve, [5, 11, 1], [1, 1, 1], 10, 10, 10)
    assert s._take(_pending(serve, s, range(3)))[0] == [0]
    with pytest.raises(RuntimeError):
        s._take(_pending(serve, s, [1, 2]))      # event 1 alone exceeds the hit capacity


def test_take_by_size_class_oldest_first(serve):
    rng = np.random.default_rng(7)
    n = 400
    nt = rng.integers(1, 400, n)
    nh = nt * 120
    s = _server(serve, nh, nt, 64, 10 ** 9, 10 ** 9, group=True)
    pending = _pending(serve, s, range(n))
    seen = []
    while any(pending):
        oldest = min(q[0] for q in pending if q)
        ev, taken, nbytes = s._take(pending)
        for c, k in enumerate(taken):
            for _ in range(k):
                pending[c].popleft()
        assert oldest in ev and len(ev) <= 64
        c0 = s.size_class[oldest]
        main = [e for e in ev if s.size_class[e] == c0]
        assert main == sorted(main)             # the oldest event's class, in arrival order
        if len(main) < len(ev):                 # other classes only top up a slot below a quarter
            assert len(main) < 64 // 4
        seen += ev
    assert sorted(seen) == list(range(n))


def test_poisson_arrivals_rate_and_order(serve):
    t = serve.poisson_arrivals(200_000, 5000.0, seed=3)
    assert np.all(np.diff(t) >= 0) and t[0] >= 0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 5000.0 - 1.0) < 0.01
    # exponential gaps: the coefficient of variation is 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.02
    assert np.array_equal(t, serve.poisson_arrivals(200_000, 5000.0, seed=3))
