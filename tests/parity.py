"""GPU-vs-oracle comparison helpers (used by the gpu-marked tests and smoke)."""
from __future__ import annotations

import numpy as np
import torch

import oracle

NL = 12


def to_np(t):
    return t.detach().cpu().numpy()


def rel_close(a, b, rtol=1e-4, atol=1e-6):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) <= atol + rtol * np.abs(b)


def compare_pack(pk_gpu: dict, pk_ora: dict) -> None:
    for k in ("hit_offsets", "perm", "layer"):
        g, o = to_np(pk_gpu[k]), pk_ora[k]
        assert np.array_equal(g, o), "pack %s differs at %s" % (k, np.nonzero(g != o)[0][:10])
    for k in ("x", "z", "dxdy", "w"):
        g, o = to_np(pk_gpu[k]), pk_ora[k]
        assert np.array_equal(g.view(np.uint32), o.view(np.uint32)), "pack %s not bit-identical" % k


def compare_stages(dbg: dict, res: dict) -> None:
    wb, wc = to_np(dbg["win_begin"]), to_np(dbg["win_count"])
    assert np.array_equal(wc, res["win_count"]), "window counts differ: tracks %s" % (
        np.nonzero((wc != res["win_count"]).any(1))[0][:10])
    m = wc > 0
    assert np.array_equal(wb[m], res["win_begin"][m]), "window begins differ"
    nt_g = to_np(dbg["n_trip"])
    assert np.array_equal(nt_g, res["n_trip"]), "triplet counts differ: %s" % np.nonzero(nt_g != res["n_trip"])[0][:10]
    trip_g, chi_g = to_np(dbg["trip"]), to_np(dbg["trip_chi2"])
    for t in np.nonzero(nt_g)[0]:
        n = nt_g[t]
        assert np.array_equal(trip_g[t, :n], res["trip"][t, :n]), ("triplets", t, trip_g[t, :n], res["trip"][t, :n])
        assert np.array_equal(chi_g[t, :n].view(np.uint32), res["trip_chi2"][t, :n].view(np.uint32)), ("chi2", t)


def compare_outputs(out: dict, res: dict, strict_bits: bool = True) -> dict:
    found_g = to_np(out["found"]).astype(bool)
    found_o = res["found"].astype(bool)
    n = found_o.size
    mism = np.nonzero(found_g != found_o)[0]
    both = found_g & found_o
    hg = to_np(out["hit_idx"])
    hit_mism = np.nonzero(both & np.any(hg != res["hit_idx"], axis=1))[0]
    n_bad = len(mism) + len(hit_mism)
    assert n_bad == 0, "track mismatches: found %s, hits %s (of %d)" % (mism[:10], hit_mism[:10], n)
    nh = to_np(out["nhits"])
    assert np.array_equal(nh[both], res["nhits"][both])
    st_g, st_o = to_np(out["state"])[both], res["state"][both]
    q_g, q_o = to_np(out["quality"])[both], res["quality"][both]
    assert np.all(rel_close(st_g, st_o, 1e-4, 1e-6)), "states beyond 1e-4 relative"
    assert np.all(rel_close(q_g, q_o, 1e-4, 1e-7)), "quality beyond 1e-4 relative"
    bit_state = np.array_equal(st_g.view(np.uint32), st_o.view(np.uint32))
    bit_q = np.array_equal(q_g.view(np.uint32), q_o.view(np.uint32))
    if strict_bits:
        assert bit_state and bit_q, "states not bit-identical"
    oo = to_np(out["out_offsets"])
    assert np.array_equal(oo, res["out_offsets"]), "compaction offsets differ"
    n_out = int(to_np(out["n_out"])[0])
    assert n_out == len(res["out_trk"])
    assert np.array_equal(to_np(out["out_trk"])[:n_out], res["out_trk"]), "compacted track list differs"
    return dict(n_tracks=int(n), n_found=int(found_o.sum()), bit_state=bit_state, bit_q=bit_q)


def run_both(tracker, batch_gpu, mode="batched", geometry=None, params=None, tuning=None, stages=False):
    """Run the library on a GPU batch and the oracle on the same events."""
    packed, out = tracker.run(batch_gpu, mode=mode, tuning=tuning)
    dbg = tracker.debug_stages(packed, batch_gpu, batch_gpu.n_events) if stages else None
    torch.cuda.synchronize()
    flags = tracker.status()
    assert flags == 0, "device status flags 0x%x" % flags
    res = oracle.run_batch(batch_gpu, geometry=geometry, params=params, dumps=stages)
    compare_pack(packed, res["packed"])
    if stages:
        compare_stages(dbg, res)
    info = compare_outputs(out, res)
    return info, packed, out, res
