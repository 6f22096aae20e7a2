"""Sharding of a batch of events over ranks (one process per GPU).

Events are independent (each event's tracks only search that event's hits), so
a batch shards by events with no exchange on the data path: every rank packs
and follows its own events, and the per-track results are gathered on the
host in the batch's event order.  The partition balances an estimate of the
work per event, input tracks x hits (the triplet and extension stages scale
with the tracks, their window searches with the hits per bucket): events are
taken in decreasing cost and each goes to the rank with the least work so far
(longest-processing-time first), and every rank's events are kept in batch
order.
"""
from __future__ import annotations

import heapq
from typing import Dict, List, Sequence

import numpy as np


def event_costs(raw_offsets: np.ndarray, trk_offsets: np.ndarray) -> np.ndarray:
    """Work estimate per event: max(1, tracks) x max(1, hits)."""
    nh = np.diff(np.asarray(raw_offsets, np.int64))
    nt = np.diff(np.asarray(trk_offsets, np.int64))
    return np.maximum(nt, 1) * np.maximum(nh, 1)


def partition(costs: Sequence[float], world: int) -> List[np.ndarray]:
    """Event indices of each of `world` ranks (sorted), greedy by cost."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, np.float64)
    order = np.argsort(-costs, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    owner = np.empty(costs.size, np.int64)
    for e in order:
        load, r = heapq.heappop(heap)
        owner[e] = r
        heapq.heappush(heap, (load + float(costs[e]), r))
    return [np.nonzero(owner == r)[0] for r in range(world)]


def gather(parts: Dict[int, dict], shards: List[np.ndarray], n_events: int) -> List[dict]:
    """Per-event results of all ranks in batch order.  parts[r] maps each of
    rank r's events (batch index) to its result."""
    out: List[dict] = [None] * n_events  # type: ignore[list-item]
    for r, events in enumerate(shards):
        for e in events:
            out[int(e)] = parts[r][int(e)]
    if any(v is None for v in out):
        raise ValueError("an event has no result")
    return out
