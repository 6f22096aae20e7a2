"""Continuous-batching server for the forward-tracking path.

Events arrive over time into a host-resident pool (pinned memory).  The
server keeps S slots, each with its own library context and device buffers
allocated once (hit, state and output buffers stay resident; geometry and
parameters live in the contexts), and three CUDA streams shared by the slots:
copies in, compute (two of these, alternating over the slots), copies out.
Whenever a slot is free it takes every event that has arrived and is not yet
scheduled (up to the slot's event and hit capacity); its copies in are queued
on the first stream, its pack and find (persistent form, launch shape from the
autotuner for the batch's size bucket, tuned on the pool's events before
serving) on its compute stream after them, and the copies of its per-track
results on the third stream after the compute, chained by events.  So the
copies in of one batch, the compute of another and the copies out of a third
overlap on the device.

The pool may also be device-resident (events that arrive straight in GPU
memory, as from a network card writing to it): batches are then views of the
pool, no copies in are made, and only the per-track results leave the device.  A batch is
admitted only while the device bytes of the batches in flight stay within the
memory budget.  Latency is measured per event from its arrival time to the
moment the server sees its batch complete with results in host memory.

Each event's result does not depend on which other events share its batch
(the kernels treat events and tracks independently and deterministically),
which the served-alone-versus-in-mix test checks.
"""
from __future__ import annotations

import dataclasses
import time
from types import SimpleNamespace
from typing import Dict, List, Optional

import numpy as np
import torch

from . import lf
from .autotune import Autotuner

NL = 12
# device bytes per hit (raw 17 + packed 21) and per input track (states 20,
# outputs 81, persistent-pipeline scratch 161: event index, windows, kept
# triplet keys and counts)
BYTES_PER_HIT = 38
BYTES_PER_TRACK = 262


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
        self.tr.reserve(max_events, max_tracks)
        e = lambda n, dt: torch.empty(n, dtype=dt, device=dev)
        self.raw = dict(x=e(max_hits, torch.float32), z=e(max_hits, torch.float32), dxdy=e(max_hits, torch.float32),
                        w=e(max_hits, torch.float32), plane=e(max_hits, torch.uint8),
                        raw_offsets=e(max_events + 1, torch.int32))
        self.st = dict(trk_offsets=e(max_events + 1, torch.int32), sx=e(max_tracks, torch.float32),
                       sy=e(max_tracks, torch.float32), stx=e(max_tracks, torch.float32),
                       sty=e(max_tracks, torch.float32), sqop=e(max_tracks, torch.float32))
        self.packed = dict(hit_offsets=e(24 * max_events + 1, torch.int32), x=e(max_hits, torch.float32),
                           z=e(max_hits, torch.float32), dxdy=e(max_hits, torch.float32),
                           w=e(max_hits, torch.float32), layer=e(max_hits, torch.uint8),
                           perm=e(max_hits, torch.int32))
        self.out = lf.Tracker.alloc_output(max_tracks, max_events, dev)
        p = lambda n, dt: torch.empty(n, dtype=dt, pin_memory=True)
        self.h_ro = p(max_events + 1, torch.int32)
        self.h_to = p(max_events + 1, torch.int32)
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
        self.batch = None      # (e0, e1, h0, h1, t0, t1, nbytes)

    def close(self):
        self.tr.close()


class Server:
    """S slots over a host event pool (an EventBatch of host tensors, pinned
    for full copy bandwidth)."""

    def __init__(self, pool, n_slots: int = 4, max_events: int = 4096, budget_bytes: int = 16 << 30,
                 geometry: Optional[dict] = None, params: Optional[dict] = None, tuner: Optional[Autotuner] = None,
                 keep_results: bool = False, device: str = "cuda"):
        self.pool = pool
        self.dev = torch.device(device)
        self.device_pool = pool.x.is_cuda
        self.ro = pool.raw_offsets.cpu().numpy().astype(np.int64)
        self.to = pool.trk_offsets.cpu().numpy().astype(np.int64)
        self.budget = int(budget_bytes)
        free, _ = torch.cuda.mem_get_info(self.dev)
        nh = np.diff(self.ro)
        nt = np.diff(self.to)
        # slot capacity: max_events of the pool's largest events
        k = min(max_events, pool.n_events)
        max_hits = int(np.sort(nh)[::-1][:k].sum()) if k else 1
        max_tracks = int(np.sort(nt)[::-1][:k].sum()) if k else 1
        slot_bytes = max_hits * BYTES_PER_HIT + max_tracks * BYTES_PER_TRACK
        n_slots = max(1, min(n_slots, self.budget // max(slot_bytes, 1), int(0.8 * free) // max(slot_bytes, 1)))
        self.max_events = max_events
        self.max_hits = max(max_hits, 1)
        self.max_tracks = max(max_tracks, 1)
        self.slots = [_Slot(max_events, self.max_hits, self.max_tracks, geometry, params, self.dev)
                      for _ in range(n_slots)]
        self.s_in = torch.cuda.Stream(device=self.dev)
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

    def tune_buckets(self, sizes=(256, 1024, 2048)) -> dict:
        """Autotune the launch shape for batches of the pool's first n events
        for each n in sizes (their buckets), before serving: the first slot's
        tracker runs the candidates on a device copy of those events."""
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
        return chosen

    # -------------------------------------------------------------- batches
    def _take(self, head: int, avail: int) -> tuple:
        """The next batch: the longest run of the pending events head ..
        head+avail-1 (arrival order is pool order) within the slot's event,
        hit and track capacity."""
        k = min(avail, self.max_events)
        ch = self.ro[head + 1:head + k + 1] - self.ro[head]
        ct = self.to[head + 1:head + k + 1] - self.to[head]
        k = min(k, int(np.searchsorted(ch, self.max_hits, side="right")),
                int(np.searchsorted(ct, self.max_tracks, side="right")))
        if k == 0:
            raise RuntimeError("event %d does not fit a slot" % head)
        e0, e1 = head, head + k
        h0, h1, t0, t1 = int(self.ro[e0]), int(self.ro[e1]), int(self.to[e0]), int(self.to[e1])
        nbytes = (h1 - h0) * BYTES_PER_HIT + (t1 - t0) * BYTES_PER_TRACK
        return e0, e1, h0, h1, t0, t1, nbytes

    def _launch(self, s: _Slot, batch):
        e0, e1, h0, h1, t0, t1, nbytes = batch
        ne, nh, nt = e1 - e0, h1 - h0, t1 - t0
        p = self.pool
        if self.device_pool:
            # the events are in device memory already: the batch is a view of
            # the pool, with its offsets rebased on the device
            with torch.cuda.stream(self.s_in):
                torch.sub(p.raw_offsets[e0:e1 + 1], p.raw_offsets[e0:e0 + 1], out=s.raw["raw_offsets"][:ne + 1])
                torch.sub(p.trk_offsets[e0:e1 + 1], p.trk_offsets[e0:e0 + 1], out=s.st["trk_offsets"][:ne + 1])
                s.ev_in.record(self.s_in)
            src_h = {f: getattr(p, f)[h0:h1] for f in ("x", "z", "dxdy", "w", "plane")}
            src_t = {f: getattr(p, f)[t0:t1] for f in ("sx", "sy", "stx", "sty", "sqop")}
        else:
            s.h_ro[:ne + 1].copy_(torch.from_numpy((self.ro[e0:e1 + 1] - h0).astype(np.int32)))
            s.h_to[:ne + 1].copy_(torch.from_numpy((self.to[e0:e1 + 1] - t0).astype(np.int32)))
            # a slot is launched only when its previous batch has completed, so
            # its buffers are free
            with torch.cuda.stream(self.s_in):
                for f in ("x", "z", "dxdy", "w", "plane"):
                    s.raw[f][:nh].copy_(getattr(p, f)[h0:h1], non_blocking=True)
                s.raw["raw_offsets"][:ne + 1].copy_(s.h_ro[:ne + 1], non_blocking=True)
                s.st["trk_offsets"][:ne + 1].copy_(s.h_to[:ne + 1], non_blocking=True)
                for f in ("sx", "sy", "stx", "sty", "sqop"):
                    s.st[f][:nt].copy_(getattr(p, f)[t0:t1], non_blocking=True)
                s.ev_in.record(self.s_in)
            src_h = {f: s.raw[f][:nh] for f in ("x", "z", "dxdy", "w", "plane")}
            src_t = {f: s.st[f][:nt] for f in ("sx", "sy", "stx", "sty", "sqop")}
        s_comp = s.s_comp
        s_comp.wait_event(s.ev_in)
        with torch.cuda.stream(s_comp):
            raw = SimpleNamespace(n_events=ne, raw_offsets=s.raw["raw_offsets"][:ne + 1], **src_h)
            pk = {k: (v[:24 * ne + 1] if k == "hit_offsets" else v[:nh]) for k, v in s.packed.items()}
            s.tr.pack(raw, s_comp, out=pk)
            st = SimpleNamespace(trk_offsets=s.st["trk_offsets"][:ne + 1], **src_t)
            out = {k: v for k, v in s.out.items()}
            for k in ("found", "nhits", "hit_idx", "state", "quality"):
                out[k] = s.out[k][:nt]
            out["out_offsets"] = s.out["out_offsets"][:ne + 1]
            out["out_trk"] = s.out["out_trk"][:max(nt, 1)]
            tuning = self.tuner.lookup(ne, nt)
            s.tr.find(pk, st, ne, "batched", tuning, s_comp, out=out)
            s.ev_comp.record(s_comp)
        self.s_out.wait_event(s.ev_comp)
        with torch.cuda.stream(self.s_out):
            # the per-track results come back to the host for every batch
            s.h_found[:nt].copy_(out["found"], non_blocking=True)
            s.h_nhits[:nt].copy_(out["nhits"], non_blocking=True)
            s.h_hits[:nt].copy_(out["hit_idx"], non_blocking=True)
            s.h_state[:nt].copy_(out["state"], non_blocking=True)
            s.h_q[:nt].copy_(out["quality"], non_blocking=True)
            if self.keep_results:
                s.h_perm[:nh].copy_(pk["perm"], non_blocking=True)
            s.done.record(self.s_out)
        s.busy = True
        s.batch = batch
        self.inflight_bytes += nbytes
        self.max_inflight = max(self.max_inflight, self.inflight_bytes)

    def _finish(self, s: _Slot):
        e0, e1, h0, h1, t0, t1, nbytes = s.batch
        if self.keep_results:
            nt = t1 - t0
            found = s.h_found[:nt].numpy().astype(bool)
            hits = s.h_hits[:nt].numpy().copy()
            perm = s.h_perm[:h1 - h0].numpy()
            for e in range(e0, e1):
                a, b = int(self.to[e] - t0), int(self.to[e + 1] - t0)
                base = int(self.ro[e] - h0)
                f = found[a:b]
                hh = hits[a:b]
                ok = (hh >= 0) & f[:, None]          # hit indices are written only for found tracks
                raw = np.where(ok, perm[np.where(ok, hh, 0)] - base, -1)
                self.results[e] = dict(found=f.copy(), nhits=s.h_nhits[a:b].numpy().copy(), hits=raw,
                                       state=s.h_state[a:b].numpy().copy(), quality=s.h_q[a:b].numpy().copy())
        s.busy = False
        s.batch = None
        self.inflight_bytes -= nbytes

    # ------------------------------------------------------------------ run
    def run(self, arrivals: np.ndarray, first_event: int = 0) -> ServeStats:
        """Serve events first_event .. first_event+len(arrivals)-1 arriving at
        the given times (seconds from start, non-decreasing)."""
        n = len(arrivals)
        done_at = np.zeros(n)
        nxt = 0            # events [0, nxt) have arrived
        head = 0           # events [head, nxt) are pending (arrived, not scheduled)
        completed = 0
        batches: List[int] = []
        t_start = time.perf_counter()
        while completed < n:
            now = time.perf_counter() - t_start
            nxt = int(np.searchsorted(arrivals, now, side="right"))
            progressed = False
            for s in self.slots:
                if s.busy and s.done.query():
                    t_done = time.perf_counter() - t_start
                    e0, e1 = s.batch[0], s.batch[1]
                    self._finish(s)
                    done_at[e0 - first_event:e1 - first_event] = t_done
                    completed += e1 - e0
                    progressed = True
            for s in self.slots:
                if head >= nxt:
                    break
                if s.busy:
                    continue
                b = self._take(first_event + head, nxt - head)
                if self.inflight_bytes + b[6] > self.budget and self.inflight_bytes > 0:
                    break      # not admitted yet: wait for memory
                self._launch(s, b)
                head += b[1] - b[0]
                batches.append(b[1] - b[0])
                progressed = True
            if not progressed:
                if nxt < n and head >= nxt and not any(s.busy for s in self.slots):
                    delay = arrivals[nxt] - (time.perf_counter() - t_start)
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
