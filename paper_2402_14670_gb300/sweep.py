"""Throughput against synthetic efficiency for window caps and tolerances.

The paper scans n_hits^window and finds that efficiency plateaus above 64
hits while throughput falls as the windows grow (Sec. "Performance").  This
module repeats that scan on the synthetic workloads: for each setting it runs
pack + persistent find on the GPU (device time from CUDA events) and scores
the result against the generator's truth with the paper's matching rule (a
track is matched to a particle when more than 70 % of its hits belong to it;
Sec. "Benchmarking setup"):

  efficiency   found and matched input tracks / reconstructible input tracks
               (the input track's particle left >= 9 hits with a stereo hit
               in every station and all three hits of a triplet configuration)
  fake rate    found tracks not matched to the input track's particle / found

Usage: python -m paper_2402_14670_gb300.sweep [--config 1] [--events 1000]
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import lf, synth


def _np(a) -> np.ndarray:
    return a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)


def reconstructible(batch, layer_of_hit: np.ndarray) -> np.ndarray:
    """Per input track: its particle is reconstructible (see module doc)."""
    hit_mcp = _np(batch.hit_mcp)
    trk_mcp = _np(batch.trk_mcp)
    n_p = int(max(hit_mcp.max(initial=-1), trk_mcp.max(initial=-1))) + 1
    has = np.zeros((max(n_p, 1), 12), bool)
    m = hit_mcp >= 0
    has[hit_mcp[m], layer_of_hit[m]] = True
    n_hits = has.sum(1)
    uv_ok = np.ones(len(has), bool)
    for s in range(3):
        uv_ok &= has[:, 4 * s + 1] | has[:, 4 * s + 2]
    trip = has[:, [0, 4, 8]].all(1) | has[:, [3, 7, 11]].all(1)
    part_ok = (n_hits >= 9) & uv_ok & trip
    out = np.zeros(len(trk_mcp), bool)
    mt = trk_mcp >= 0
    out[mt] = part_ok[trk_mcp[mt]]
    return out


def score(batch, packed: dict, out: dict) -> dict:
    """Efficiency and fake rate of one result against the batch's truth.
    ``packed["perm"]`` maps packed to raw hit indices; ``out`` holds the
    per-input-track ``found`` flags and ``hit_idx`` rows (packed indices,
    -1 padded), as the library or any other producer writes them."""
    perm = _np(packed["perm"])
    hit_mcp = _np(batch.hit_mcp)
    trk_mcp = _np(batch.trk_mcp)
    layer_raw = (_np(batch.plane) % 12).astype(np.int64)
    found = _np(out["found"]).astype(bool)
    hits = _np(out["hit_idx"]).reshape(len(found), -1)
    ok = (hits >= 0) & found[:, None]
    raw = np.where(ok, perm[np.where(ok, hits, 0)], 0)
    same = ok & (hit_mcp[raw] == trk_mcp[:, None]) & (trk_mcp[:, None] >= 0)
    n = ok.sum(1)
    frac = np.where(n > 0, same.sum(1) / np.maximum(n, 1), 0.0)
    matched = found & (frac > 0.7)
    reco = reconstructible(batch, layer_raw)
    mcp_p = None
    if batch.mcp is not None:
        qop = _np(batch.mcp["qop"])
        mcp_p = 1.0 / np.abs(qop)
    hi_p = np.zeros(len(trk_mcp), bool)
    if mcp_p is not None:
        mt = trk_mcp >= 0
        hi_p[mt] = mcp_p[trk_mcp[mt]] > 5.0
    eff = matched[reco].sum() / max(reco.sum(), 1)
    eff5 = matched[reco & hi_p].sum() / max((reco & hi_p).sum(), 1)
    fake = (found & ~matched).sum() / max(found.sum(), 1)
    return dict(efficiency=float(eff), efficiency_p_gt_5GeV=float(eff5), fake_rate=float(fake),
                found=int(found.sum()), reconstructible=int(reco.sum()))


def run_setting(batch, params: dict, reps: int = 5) -> dict:
    tr = lf.Tracker(None, params)
    packed, out = tr.run(batch)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        tr.pack(batch, out=packed)
        tr.find(packed, batch, batch.n_events, "batched", out=out)
        b.record(s)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ms = float(np.median(times))
    res = score(batch, packed, out)
    res.update(ms=ms, events_per_s=batch.n_events / (ms / 1e3))
    tr.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--events", type=int, default=1000)
    ap.add_argument("--caps", type=str, default="8,16,24,32,48,64")
    ap.add_argument("--xtol-scales", type=str, default="1.0")
    args = ap.parse_args()
    batch = synth.generate(args.config, n_events=args.events, device="cuda", truth=True)
    for scale in [float(v) for v in args.xtol_scales.split(",")]:
        for cap in [int(v) for v in args.caps.split(",")]:
            p = lf.default_params()
            p["n_hits_window"] = cap
            p["xtol_c"] *= scale
            p["xtol_p"] *= scale
            r = run_setting(batch, p)
            r.update(config=args.config, events=args.events, n_hits_window=cap, xtol_scale=scale)
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
