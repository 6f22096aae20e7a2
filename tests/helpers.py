"""Shared test helpers: crafted events and geometry conversion."""
from __future__ import annotations

import dataclasses
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2402_14670_gb300 import synth  # noqa: E402

W_DEFAULT = 1.0 / (0.08 * 0.08)


def geo_dict(geo: synth.Geometry = None) -> dict:
    geo = geo or synth.Geometry()
    d = dataclasses.asdict(geo)
    d["z"] = list(d["z"])
    d["dxdy"] = list(d["dxdy"])
    return d


def make_batch(events, geo: synth.Geometry = None) -> synth.EventBatch:
    """Build a raw EventBatch from explicit content.

    ``events`` is a list of dicts with
      hits:   list of (layer, zone, x) or (layer, zone, x, z, dxdy, w); raw order as given
      states: list of (xs, ys, txs, tys, qop)
    """
    geo = geo or synth.Geometry()
    xs, zs, ds, ws, pl, nh, nt, st = [], [], [], [], [], [], [], []
    for ev in events:
        hits = ev.get("hits", [])
        for h in hits:
            layer, zone, x = int(h[0]), int(h[1]), float(h[2])
            z = float(h[3]) if len(h) > 3 else geo.z[layer]
            d = float(h[4]) if len(h) > 4 else geo.dxdy[layer]
            w = float(h[5]) if len(h) > 5 else W_DEFAULT
            xs.append(x); zs.append(z); ds.append(d); ws.append(w); pl.append(zone * 12 + layer)
        nh.append(len(hits))
        nt.append(len(ev.get("states", [])))
        st.extend(ev.get("states", []))
    off = lambda n: torch.tensor(np.concatenate([[0], np.cumsum(n)]).astype(np.int32))
    f = lambda a: torch.tensor(np.asarray(a, np.float32).reshape(-1))
    s = np.asarray(st, np.float64).reshape(-1, 5)
    return synth.EventBatch(len(events), off(nh), f(xs), f(zs), f(ds), f(ws),
                            torch.tensor(np.asarray(pl, np.uint8).reshape(-1)), off(nt),
                            f(s[:, 0]), f(s[:, 1]), f(s[:, 2]), f(s[:, 3]), f(s[:, 4]))


def track_hits(tx, ty, qop, geo: synth.Geometry = None, layers=range(12), offsets=None):
    """Exact hits of a simulated particle: list of (layer, zone, x_measured)."""
    _, y, xm = synth.trajectory(tx, ty, qop, geo)
    out = []
    for l in layers:
        d = 0.0 if offsets is None else float(offsets.get(l, 0.0))
        out.append((l, 1 if y[l] >= 0 else 0, float(xm[l]) + d))
    return out


def raw_ids_in_windows(res: dict, t: int) -> dict:
    """layer -> sorted raw hit indices inside track t's (capped) window."""
    perm = res["packed"]["perm"]
    out = {}
    for l in range(12):
        b, c = int(res["win_begin"][t, l]), int(res["win_count"][t, l])
        out[l] = sorted(int(perm[i]) for i in range(b, b + c))
    return out
