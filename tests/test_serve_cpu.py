"""Host logic of the continuous-batching server, on CPU: the rule that forms
the next batch from the pending events, and the arrival process."""
from types import SimpleNamespace

import numpy as np
import pytest


@pytest.fixture(scope="module")
def serve():
    # the server module loads the library: build it first (host compile only)
    from paper_2402_14670_gb300 import build
    build.build()
    from paper_2402_14670_gb300 import serve as m
    return m


def _fake(nh, nt, max_events, max_hits, max_tracks):
    ro = np.concatenate([[0], np.cumsum(nh)]).astype(np.int64)
    to = np.concatenate([[0], np.cumsum(nt)]).astype(np.int64)
    return SimpleNamespace(ro=ro, to=to, max_events=max_events, max_hits=max_hits, max_tracks=max_tracks)


def _brute(f, head, avail):
    """Longest run head..head+k-1 within every capacity, by trying each k."""
    best = 0
    for k in range(1, min(avail, f.max_events) + 1):
        h = f.ro[head + k] - f.ro[head]
        t = f.to[head + k] - f.to[head]
        if h <= f.max_hits and t <= f.max_tracks:
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
        f = _fake(nh, nt, max_events, max(max_hits, int(nh.max())), max(max_tracks, int(nt.max())))
        for head in (0, 1, 17, 200, 399):
            for avail in sorted({1, min(3, 400 - head), 400 - head}):
                e0, e1, h0, h1, t0, t1, nbytes = serve.Server._take(f, head, avail)
                k = _brute(f, head, avail)
                assert (e0, e1) == (head, head + k)
                assert (h0, h1, t0, t1) == (f.ro[e0], f.ro[e1], f.to[e0], f.to[e1])
                assert nbytes == (h1 - h0) * serve.BYTES_PER_HIT + (t1 - t0) * serve.BYTES_PER_TRACK


def test_take_counts_empty_events_and_refuses_an_event_above_capacity(serve):
    # empty events cost nothing, so they ride along up to the event capacity
    f = _fake([0, 0, 0, 10, 0], [0, 2, 0, 1, 0], 4, 10, 3)
    assert serve.Server._take(f, 0, 5)[:2] == (0, 4)
    f = _fake([5, 11, 1], [1, 1, 1], 10, 10, 10)
    assert serve.Server._take(f, 0, 3)[:2] == (0, 1)
    with pytest.raises(RuntimeError):
        serve.Server._take(f, 1, 2)          # event 1 alone exceeds the hit capacity


def test_poisson_arrivals_rate_and_order(serve):
    t = serve.poisson_arrivals(200_000, 5000.0, seed=3)
    assert np.all(np.diff(t) >= 0) and t[0] >= 0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 5000.0 - 1.0) < 0.01
    # exponential gaps: the coefficient of variation is 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.02
    assert np.array_equal(t, serve.poisson_arrivals(200_000, 5000.0, seed=3))
