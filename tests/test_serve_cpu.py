"""Host logic of the server, on CPU: the arrival ring never hands out space
that an event still held occupies, and batching by size takes the oldest
event's class first, within the slot's capacity."""
from collections import deque

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_14670_gb300 import serve  # noqa: E402


def test_ring_never_overlaps_held_events():
    rng = np.random.default_rng(3)
    ring = serve._Ring(1000, 300, "cpu")
    held = deque()            # (virtual hit start, n hits, virtual track start, n tracks)
    placed = 0
    for step in range(5000):
        if held and (rng.random() < 0.45 or len(held) > 40):
            held.popleft()    # the oldest event completes
            continue
        nh, nt = int(rng.integers(0, 120)), int(rng.integers(0, 40))
        tail = (held[0][0], held[0][2]) if held else None
        pos = ring.place(nh, nt, tail)
        if pos is None:
            # refused only when the ring really lacks the room: the held
            # span plus the run exceeds the capacity
            assert held
            continue
        vh, vt = pos
        ph, pt = vh % ring.cap_h, vt % ring.cap_t
        assert ph + nh <= ring.cap_h and pt + nt <= ring.cap_t        # contiguous in the arrays
        for (h0, n0, t0, m0) in held:
            a0, b0 = h0 % ring.cap_h, h0 % ring.cap_h + n0
            assert b0 <= ph or ph + nh <= a0 or nh == 0 or n0 == 0    # hit ranges disjoint
            c0, d0 = t0 % ring.cap_t, t0 % ring.cap_t + m0
            assert d0 <= pt or pt + nt <= c0 or nt == 0 or m0 == 0    # track ranges disjoint
        assert vh + nh - (held[0][0] if held else vh) <= ring.cap_h
        ring.vh, ring.vt = vh + nh, vt + nt
        held.append((vh, nh, vt, nt))
        placed += 1
    assert placed > 1000


def _server(nh, nt, max_events, max_hits, max_tracks, group=True):
    s = serve.Server.__new__(serve.Server)
    s.nh, s.nt = np.asarray(nh), np.asarray(nt)
    s.size_class = np.searchsorted(np.asarray(serve.TRACK_EDGES), s.nt, side="left")
    s.max_events, s.max_hits, s.max_tracks = max_events, max_hits, max_tracks
    s.group_by_size = group
    return s


def _pending(s, events):
    p = [deque() for _ in range(len(serve.TRACK_EDGES) + 1)]
    for e in events:
        p[s._class(e)].append(e)
    return p


def test_take_groups_by_size_oldest_first():
    rng = np.random.default_rng(7)
    n = 400
    nt = rng.integers(1, 400, n)
    nh = nt * 120
    s = _server(nh, nt, 64, 10 ** 9, 10 ** 9)
    pending = _pending(s, range(n))
    seen = []
    while any(pending):
        oldest = min(q[0] for q in pending if q)
        ev, taken, nbytes = s._take(pending)
        for c, k in enumerate(taken):
            for _ in range(k):
                pending[c].popleft()
        assert oldest in ev
        assert len(ev) <= 64
        c0 = s.size_class[oldest]
        main = [e for e in ev if s.size_class[e] == c0]
        # the oldest event's class in arrival order
        assert main == sorted(main)
        # other classes only as a top-up of a slot filled below a quarter
        if len(main) < len(ev):
            assert len(main) < 64 // 4
        assert nbytes == int(nh[ev].sum()) * serve.SLOT_BYTES_PER_HIT + int(nt[ev].sum()) * serve.SLOT_BYTES_PER_TRACK
        seen += ev
    assert sorted(seen) == list(range(n))


def test_take_respects_hit_and_track_capacity():
    nt = np.array([10, 20, 30, 5, 5, 5, 40, 2])
    nh = nt * 100
    s = _server(nh, nt, 100, 10 ** 6, 60, group=False)
    ev, _, _ = s._take(_pending(s, range(len(nt))))
    assert ev == [0, 1, 2]          # 10+20+30 tracks = 60 <= 60; the next event would exceed it
    s = _server(nh, nt, 100, 3500, 10 ** 6, group=False)
    ev, _, _ = s._take(_pending(s, range(len(nt))))
    assert ev == [0, 1]             # 1000+2000 hits; the third would exceed 3500
    s = _server(nh, nt, 2, 10 ** 6, 10 ** 6, group=False)
    ev, _, _ = s._take(_pending(s, range(len(nt))))
    assert ev == [0, 1]             # event capacity
