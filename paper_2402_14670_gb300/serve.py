"""Continuous-batching server for the forward-tracking path.

Events arrive over time.  The server keeps S slots, each with its own library
context and device buffers of fixed capacity (packed hits, states, outputs,
scratch), allocated once, and runs every batch of a slot through
lf_process_slot: the batch's event count and offsets are written to the
slot's device block by one small copy, and the slot's CUDA graph (captured
once per launch shape) packs, follows and compacts it.  The kernels read the
batch's hits straight from where the events are held, through the batch's
per-event source offsets: no copy of the hits into the slot.

Events are held in device memory:
  - a device-resident pool (events that arrive straight in GPU memory, as
    from a network card writing to it) is read in place;
  - events arriving in page-locked host memory are copied, in arrival order,
    into a device arrival ring (one copy per array per run of arrivals) as
    soon as the ring has room for them: the ring is the admission by free
    device memory, and an event waits on the host while it is full.  Its
    space is reused once every event before it has completed.

Batching by size: a free slot takes the oldest pending events in arrival
order up to its capacity in events, hits and tracks, so a batch's event count
follows its events' sizes.  With group_by_size, pending events are kept per
size class (input tracks per event: 1-32, 33-64, 65-128, 129-256, 257+, the
autotuner's classes) and a free slot takes the class of the oldest pending
event, that class's events in arrival order up to its capacity, and, when
they fill less than a quarter of it, events of the nearest classes.  In both
modes the oldest event is in the next batch, so no event waits behind a
stream of others.  (On the uneven workload the size classes were measured to
serve fewer events per second at a higher p99 than arrival order: the
persistent kernels balance tracks, not events, so a batch of mixed sizes keeps
the GPU fuller than a batch of small events only, and a batch of large events
only leaves the per-event pack with a long tail.)  The launch shape is the
autotuner's choice for the batch's bucket (tuned before serving on the pool's
events); the slot graphs of those shapes are captured before serving.

CUDA streams shared by the slots: arrivals (copies into the ring), offset
blocks (one small copy per batch), compute (two of these, alternating over
the slots) and copies out (per-track results), chained by events: a batch
waits for the copies of its own events only, and the copies of one batch, the
compute of another and the copies out of a third overlap.  A batch
is admitted only while the device bytes of the batches in flight stay within
the memory budget.  Latency is measured per event from its arrival time to
the moment the server sees its batch complete with results in host memory.

Each event's result does not depend on which other events share its batch
(the kernels treat events and tracks independently and deterministically),
which the served-alone-versus-in-mix test checks.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import Dict, List, Optional

import numpy as np
import torch

from . import lf
from .autotune import TRACK_EDGES, Autotuner

NL = 12
# device bytes per hit and per input track of a slot: packed hits 21;
# states 20, outputs 81, persistent-pipeline scratch 161 (event index,
# windows, kept triplet keys and counts)
SLOT_BYTES_PER_HIT = 21
SLOT_BYTES_PER_TRACK = 262
# arrival ring: raw hit 17, input state 20
RING_BYTES_PER_HIT = 17
RING_BYTES_PER_TRACK = 20
HIT_FIELDS = ("x", "z", "dxdy", "w", "plane")
STATE_FIELDS = ("sx", "sy", "stx", "sty", "sqop")


@dataclasses.dataclass
class ServeStats:
    n_events: int
    wall_s: float
    events_per_s: float
    p50_ms: float
    p99_ms: float
    mean_batch_events: float
    n_batches: int
    max_inflight_bytes: int


class _Slot:
    def __init__(self, max_events: int, max_hits: int, max_tracks: int, geometry, params, dev):
        self.tr = lf.Tracker(geometry, params)
        # scratch sized once: growing it mid-stream would free device memory,
        # which synchronises the device
        self.tr.reserve(max_events, max_hits, max_tracks)
        self.buf = lf.SlotBuffers(max_events, max_hits, max_tracks, dev, own_raw=False)
        p = lambda n, dt: torch.empty(n, dtype=dt, pin_memory=True)
        self.h_meta = p(self.buf.meta.numel(), torch.int32)
        self.h_views = self.buf.meta_views(self.h_meta)
        self.h_found = p(max_tracks, torch.uint8)
        self.h_nhits = p(max_tracks, torch.uint8)
        self.h_hits = p((max_tracks, NL), torch.int32)
        self.h_state = p((max_tracks, 6), torch.float32)
        self.h_q = p(max_tracks, torch.float32)
        self.h_perm = p(max_hits, torch.int32)
        self.ev_in = torch.cuda.Event()
        self.ev_comp = torch.cuda.Event()
        self.done = torch.cuda.Event()
        self.busy = False
        self.batch = None      # (events, r_off, t_off, nbytes)

    def close(self):
        self.tr.close()


class _Ring:
    """Device arrival ring for events that arrive in host memory: hit and
    state arrays filled in arrival order.  Positions are virtual (they only
    grow; the array index is the position modulo the capacity); a run of
    events that would cross the end of the arrays starts at the next lap
    instead, and the space between is counted as used until the events
    before it are released."""

    def __init__(self, cap_hits: int, cap_tracks: int, dev):
        self.cap_h, self.cap_t = max(int(cap_hits), 1), max(int(cap_tracks), 1)
        e = lambda n, dt: torch.empty(n, dtype=dt, device=dev)
        for f in HIT_FIELDS:
            setattr(self, f, e(self.cap_h, torch.uint8 if f == "plane" else torch.float32))
        for f in STATE_FIELDS:
            setattr(self, f, e(self.cap_t, torch.float32))
        self.vh = self.vt = 0

    @staticmethod
    def _start(v: int, n: int, cap: int) -> int:
        return v if (v % cap) + n <= cap else (v // cap + 1) * cap

    def place(self, need_h: int, need_t: int, tail) -> Optional[tuple]:
        """Virtual start positions for a run of need_h hits and need_t tracks,
        or None when the ring has no room for it; tail is the (hit, track)
        virtual position of the oldest event still held, None when the ring
        holds none."""
        if tail is None:
            # empty: restart both arrays at a lap boundary
            self.vh = self._start(self.vh, self.cap_h, self.cap_h)
            self.vt = self._start(self.vt, self.cap_t, self.cap_t)
            tail = (self.vh, self.vt)
        sh = self._start(self.vh, need_h, self.cap_h)
        st = self._start(self.vt, need_t, self.cap_t)
        if sh + need_h - tail[0] > self.cap_h or st + need_t - tail[1] > self.cap_t:
            return None
        return sh, st


class Server:
    """S slots over an event pool (an EventBatch: device tensors, or host
    tensors pinned for full copy bandwidth)."""

    def __init__(self, pool, n_slots: int = 4, max_events: int = 4096, budget_bytes: int = 16 << 30,
                 geometry: Optional[dict] = None, params: Optional[dict] = None, tuner: Optional[Autotuner] = None,
                 keep_results: bool = False, device: str = "cuda", group_by_size: bool = False):
        self.pool = pool
        self.dev = torch.device(device)
        self.device_pool = pool.x.is_cuda
        self.group_by_size = group_by_size
        self.ro = pool.raw_offsets.cpu().numpy().astype(np.int64)
        self.to = pool.trk_offsets.cpu().numpy().astype(np.int64)
        self.nh = np.diff(self.ro)
        self.nt = np.diff(self.to)
        self.size_class = np.searchsorted(np.asarray(TRACK_EDGES), self.nt, side="left")
        self.budget = int(budget_bytes)
        free, _ = torch.cuda.mem_get_info(self.dev)
        # slot capacity: max_events of the pool's largest events
        k = min(max_events, pool.n_events)
        max_hits = max(int(np.sort(self.nh)[::-1][:k].sum()) if k else 1, 1)
        max_tracks = max(int(np.sort(self.nt)[::-1][:k].sum()) if k else 1, 1)
        slot_bytes = max_hits * SLOT_BYTES_PER_HIT + max_tracks * SLOT_BYTES_PER_TRACK
        # the arrival ring (host-fed): twice the slots' capacity, within the budget
        ring_h = ring_t = 0
        ring_bytes = 0
        if not self.device_pool:
            ring_h, ring_t = 2 * n_slots * max_hits, 2 * n_slots * max_tracks
            ring_bytes = ring_h * RING_BYTES_PER_HIT + ring_t * RING_BYTES_PER_TRACK
            room = self.budget - slot_bytes
            if ring_bytes > room // 2:
                s = max(room // 2, 1) / ring_bytes
                ring_h, ring_t = max(int(ring_h * s), max_hits), max(int(ring_t * s), max_tracks)
                ring_bytes = ring_h * RING_BYTES_PER_HIT + ring_t * RING_BYTES_PER_TRACK
        n_slots = max(1, min(n_slots, (self.budget - ring_bytes) // max(slot_bytes, 1),
                             int(0.8 * free - ring_bytes) // max(slot_bytes, 1)))
        self.max_events = max_events
        self.max_hits = max_hits
        self.max_tracks = max_tracks
        self.slots = [_Slot(max_events, max_hits, max_tracks, geometry, params, self.dev) for _ in range(n_slots)]
        self.ring = None if self.device_pool else _Ring(ring_h, ring_t, self.dev)
        self.s_in = torch.cuda.Stream(device=self.dev)
        self.s_meta = torch.cuda.Stream(device=self.dev)
        # two compute streams, alternating over the slots: one batch's
        # persistent kernels fill the SMs the other's tail leaves idle (each
        # slot has its own context, so their work is independent)
        self.s_comps = [torch.cuda.Stream(device=self.dev), torch.cuda.Stream(device=self.dev)]
        for i, sl in enumerate(self.slots):
            sl.s_comp = self.s_comps[i % 2]
        self.s_out = torch.cuda.Stream(device=self.dev)
        self.tuner = tuner or Autotuner()
        self.keep_results = keep_results
        self.results: Dict[int, dict] = {}
        self.inflight_bytes = 0
        self.max_inflight = 0

    def close(self):
        for s in self.slots:
            s.close()

    @property
    def source(self):
        """The gather source of the slots: the device pool or the ring."""
        return self.pool if self.device_pool else self.ring

    def tune_buckets(self, sizes=(256, 1024, 2048)) -> dict:
        """Autotune the launch shape for batches of the pool's first n events
        for each n in sizes (their buckets), before serving (the first slot's
        tracker runs the candidates on a device copy of those events), then
        capture every slot's graph for each chosen shape."""
        chosen = {}
        tr = self.slots[0].tr
        for n in sizes:
            n = min(int(n), self.pool.n_events, self.max_events)
            if n <= 0:
                continue
            sub = self.pool.select_events(range(n)).to(self.dev)
            if sub.n_tracks == 0:
                continue
            packed = tr.pack(sub)
            chosen[n] = self.tuner.choose(tr, packed, sub, n)
        torch.cuda.synchronize(self.dev)
        self.capture_graphs([None] + list(chosen.values()))
        return chosen

    def capture_graphs(self, tunings) -> None:
        """Capture each slot's graph for each launch shape now (an empty
        batch), so that no capture falls inside serving."""
        seen = set()
        for tu in tunings:
            key = None if tu is None else tuple(sorted(tu.items()))
            if key in seen:
                continue
            seen.add(key)
            for s in self.slots:
                s.buf.n_dev.zero_()
                s.tr.process_slot(s.buf, self.source, tu, s.s_comp)
        torch.cuda.synchronize(self.dev)

    # -------------------------------------------------------------- batches
    def _take(self, pending: List[deque]) -> tuple:
        """The next batch, not yet removed from pending: the oldest pending
        event's size class in arrival order within the slot's capacity,
        topped up from the nearest classes when it fills less than a quarter
        of the slot.  Returns (events, taken per class, device bytes)."""
        heads = [(q[0], c) for c, q in enumerate(pending) if q]
        first, c0 = min(heads)
        order = [c0] + [c for _, c in sorted((abs(c - c0), c) for c in range(len(pending))
                                             if c != c0 and pending[c])]
        out: List[int] = []
        taken = [0] * len(pending)
        h = t = 0
        for c in order:
            if c != c0 and len(out) >= self.max_events // 4:
                break
            for e in pending[c]:
                if len(out) >= self.max_events or h + self.nh[e] > self.max_hits or t + self.nt[e] > self.max_tracks:
                    break
                out.append(e)
                taken[c] += 1
                h += int(self.nh[e])
                t += int(self.nt[e])
        if not out:
            raise RuntimeError("event %d does not fit a slot" % first)
        return out, taken, h * SLOT_BYTES_PER_HIT + t * SLOT_BYTES_PER_TRACK

    def _launch(self, s: _Slot, events: List[int]):
        ids = np.asarray(events, dtype=np.int64)
        ne = len(ids)
        nh, nt = self.nh[ids], self.nt[ids]
        r_off = np.concatenate([[0], np.cumsum(nh)])
        t_off = np.concatenate([[0], np.cumsum(nt)])
        if self.device_pool:
            hs, ts = self.ro[ids], self.to[ids]
        else:
            hs, ts = self.ring_vh[ids] % self.ring.cap_h, self.ring_vt[ids] % self.ring.cap_t
        hn, hro, hto, hhs, hts = s.h_views
        hn[0] = ne
        hro[:ne + 1] = torch.from_numpy(r_off.astype(np.int32))
        hto[:ne + 1] = torch.from_numpy(t_off.astype(np.int32))
        hhs[:ne] = torch.from_numpy(hs.astype(np.int32))
        hts[:ne] = torch.from_numpy(ts.astype(np.int32))
        with torch.cuda.stream(self.s_meta):
            s.buf.meta.copy_(s.h_meta, non_blocking=True)
            s.ev_in.record(self.s_meta)
        s_comp = s.s_comp
        s_comp.wait_event(s.ev_in)
        if not self.device_pool:
            # the arrival copies of these events (runs complete in order)
            s_comp.wait_event(self.run_events[int(self.ev_run[ids].max())])
        n_t, n_h = int(t_off[-1]), int(r_off[-1])
        tuning = self.tuner.lookup(ne, n_t)
        s.tr.process_slot(s.buf, self.source, tuning, s_comp)
        s.ev_comp.record(s_comp)
        self.s_out.wait_event(s.ev_comp)
        out = s.buf.out
        with torch.cuda.stream(self.s_out):
            # the per-track results come back to the host for every batch
            s.h_found[:n_t].copy_(out["found"][:n_t], non_blocking=True)
            s.h_nhits[:n_t].copy_(out["nhits"][:n_t], non_blocking=True)
            s.h_hits[:n_t].copy_(out["hit_idx"][:n_t], non_blocking=True)
            s.h_state[:n_t].copy_(out["state"][:n_t], non_blocking=True)
            s.h_q[:n_t].copy_(out["quality"][:n_t], non_blocking=True)
            if self.keep_results:
                s.h_perm[:n_h].copy_(s.buf.packed["perm"][:n_h], non_blocking=True)
            s.done.record(self.s_out)
        nbytes = n_h * SLOT_BYTES_PER_HIT + n_t * SLOT_BYTES_PER_TRACK
        s.busy = True
        s.batch = (ids, r_off, t_off, nbytes)
        self.inflight_bytes += nbytes
        self.max_inflight = max(self.max_inflight, self.inflight_bytes)

    def _finish(self, s: _Slot):
        ids, r_off, t_off, nbytes = s.batch
        if self.keep_results:
            nt = int(t_off[-1])
            found = s.h_found[:nt].numpy().astype(bool)
            hits = s.h_hits[:nt].numpy().copy()
            perm = s.h_perm[:int(r_off[-1])].numpy()
            for i, e in enumerate(ids):
                a, b = int(t_off[i]), int(t_off[i + 1])
                f = found[a:b]
                hh = hits[a:b]
                ok = (hh >= 0) & f[:, None]          # hit indices are written only for found tracks
                raw = np.where(ok, perm[np.where(ok, hh, 0)] - int(r_off[i]), -1)
                self.results[int(e)] = dict(found=f.copy(), nhits=s.h_nhits[a:b].numpy().copy(), hits=raw,
                                            state=s.h_state[a:b].numpy().copy(), quality=s.h_q[a:b].numpy().copy())
        s.busy = False
        s.batch = None
        self.inflight_bytes -= nbytes

    def _class(self, e: int) -> int:
        return int(self.size_class[e]) if self.group_by_size else 0

    # ---------------------------------------------------------- arrivals
    def _admit(self, first: int, upto: int) -> int:
        """Copy arrived events first .. upto-1 (as many as the ring holds) into
        the ring; returns the first event not admitted."""
        p = self.pool
        a = first
        while a < upto:
            while self.ring_tail < a and self.ev_done[self.ring_tail]:
                self.ring_tail += 1
            tail = None if self.ring_tail >= a else (int(self.ring_vh[self.ring_tail]),
                                                     int(self.ring_vt[self.ring_tail]))
            # the longest run a .. b-1 that the ring places in one piece (at
            # most a quarter of a slot's events, so that batches can start on
            # the first runs while later ones are still being copied)
            upto_r = min(upto, a + max(self.max_events // 4, 1))
            ch = np.cumsum(self.nh[a:upto_r])
            ct = np.cumsum(self.nt[a:upto_r])
            b = a + int(min(np.searchsorted(ch, self.ring.cap_h, side="right"),
                            np.searchsorted(ct, self.ring.cap_t, side="right")))
            pos = None
            while b > a:
                pos = self.ring.place(int(ch[b - a - 1]), int(ct[b - a - 1]), tail)
                if pos is not None:
                    break
                b = a + (b - a) // 2
            if pos is None:
                break
            vh, vt = pos
            h0, h1, t0, t1 = int(self.ro[a]), int(self.ro[b]), int(self.to[a]), int(self.to[b])
            ph, pt = vh % self.ring.cap_h, vt % self.ring.cap_t
            with torch.cuda.stream(self.s_in):
                if h1 > h0:
                    for f in HIT_FIELDS:
                        getattr(self.ring, f)[ph:ph + h1 - h0].copy_(getattr(p, f)[h0:h1], non_blocking=True)
                if t1 > t0:
                    for f in STATE_FIELDS:
                        getattr(self.ring, f)[pt:pt + t1 - t0].copy_(getattr(p, f)[t0:t1], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.s_in)
            self.run_events.append(ev)
            self.ev_run[a:b] = len(self.run_events) - 1
            self.ring_vh[a:b] = vh + (self.ro[a:b] - h0)
            self.ring_vt[a:b] = vt + (self.to[a:b] - t0)
            self.ring.vh, self.ring.vt = vh + h1 - h0, vt + t1 - t0
            for e in range(a, b):
                self.pending[self._class(e)].append(e)
            a = b
        return a

    # ------------------------------------------------------------------ run
    def run(self, arrivals: np.ndarray, first_event: int = 0) -> ServeStats:
        """Serve events first_event .. first_event+len(arrivals)-1 arriving at
        the given times (seconds from start, non-decreasing)."""
        n = len(arrivals)
        e_end = first_event + n
        done_at = np.zeros(n)
        self.pending = [deque() for _ in range(len(TRACK_EDGES) + 1)]
        self.ev_done = np.zeros(self.pool.n_events + 1, dtype=bool)
        if not self.device_pool:
            self.ring_vh = np.zeros(self.pool.n_events, dtype=np.int64)
            self.ring_vt = np.zeros(self.pool.n_events, dtype=np.int64)
            self.ring_tail = first_event
            self.run_events = []
            self.ev_run = np.zeros(self.pool.n_events, dtype=np.int64)
        nxt = first_event          # events [first_event, nxt) have arrived
        admitted = first_event     # events [first_event, admitted) are held in device memory
        completed = 0
        batches: List[int] = []
        t_start = time.perf_counter()
        while completed < n:
            now = time.perf_counter() - t_start
            nxt = first_event + int(np.searchsorted(arrivals, now, side="right"))
            progressed = False
            for s in self.slots:
                if s.busy and s.done.query():
                    t_done = time.perf_counter() - t_start
                    ids = s.batch[0]
                    self._finish(s)
                    done_at[ids - first_event] = t_done
                    self.ev_done[ids] = True
                    completed += len(ids)
                    progressed = True
            if admitted < nxt:
                if self.device_pool:
                    for e in range(admitted, nxt):
                        self.pending[self._class(e)].append(e)
                    a = nxt
                else:
                    a = self._admit(admitted, nxt)
                progressed = progressed or a > admitted
                admitted = a
            for s in self.slots:
                if not any(self.pending):
                    break
                if s.busy:
                    continue
                ev, taken, need = self._take(self.pending)
                if self.inflight_bytes + need > self.budget and self.inflight_bytes > 0:
                    break      # not admitted yet: wait for memory
                for c, k in enumerate(taken):
                    for _ in range(k):
                        self.pending[c].popleft()
                self._launch(s, ev)
                batches.append(len(ev))
                progressed = True
            if not progressed:
                if nxt < e_end and admitted >= nxt and not any(s.busy for s in self.slots):
                    delay = arrivals[nxt - first_event] - (time.perf_counter() - t_start)
                    if delay > 0:
                        time.sleep(min(delay, 0.001))
                else:
                    time.sleep(2e-5)
        wall = float(done_at.max() - arrivals[0]) if n else 0.0
        lat = (done_at - arrivals) * 1e3
        return ServeStats(n, wall, n / wall if wall > 0 else 0.0, float(np.percentile(lat, 50)) if n else 0.0,
                          float(np.percentile(lat, 99)) if n else 0.0,
                          float(np.mean(batches)) if batches else 0.0, len(batches), self.max_inflight)


def poisson_arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate (events/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n)) - 0.0
