"""CUDA library against the oracle, element by element, on the same inputs.

Both forms (plain: one kernel per stage; batched: persistent stage kernels over
device work queues, or on request the tile kernel) must give the oracle's packed hits bit for bit, the same windows and triplet
lists, the same selected hit lists for every input track and the same states
and Q (compared bit for bit, within 1e-4 relative at worst).
"""
import time

import numpy as np
import pytest
import torch

import oracle
from helpers import geo_dict, make_batch
from parity import compare_outputs, compare_pack, run_both, to_np
from paper_2402_14670_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_14670_gb300 import build
    build.build()
    from paper_2402_14670_gb300 import lf
    return lf


def _tracker(lfm, geometry=None, params=None):
    return lfm.Tracker(geometry, params)


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_tiny_event(lfm, mode):
    b = synth.generate(0).to("cuda")
    tr = _tracker(lfm)
    info, *_ = run_both(tr, b, mode=mode, stages=True)
    assert info["n_found"] >= 10


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_minimum_bias_subset(lfm, mode):
    b = synth.generate(1, n_events=300).to("cuda")
    tr = _tracker(lfm)
    info, *_ = run_both(tr, b, mode=mode, stages=(mode == "plain"))
    assert info["n_found"] > 8000


def test_high_occupancy_subset(lfm):
    # ~25k hits per event: most buckets exceed one warp's sort and take the block path
    b = synth.generate(4, n_events=30).to("cuda")
    tr = _tracker(lfm)
    info, *_ = run_both(tr, b, mode="batched", stages=True)
    assert info["n_found"] > 1000


def test_uneven_subset(lfm):
    b = synth.generate(2, n_events=200).to("cuda")
    tr = _tracker(lfm)
    run_both(tr, b, mode="batched")


def test_paper_constants_and_magdown(lfm):
    geo = synth.Geometry(polarity=-1)
    b = synth.generate(1, n_events=100, geometry=geo).to("cuda")
    g = geo_dict(geo)
    p = lfm.default_params(paper_K=True)
    tr = _tracker(lfm, g, p)
    run_both(tr, b, mode="plain", geometry=g, params=p, stages=True)
    run_both(tr, b, mode="batched", geometry=g, params=p)


@pytest.mark.parametrize("polarity", [1, -1])
def test_qop_polynomial(lfm, polarity):
    """q/p from Eq. pt_kick with the polynomial field integral (Sec.
    "Calculation of momentum and track states"), coefficients fitted on toy
    tracks: states bit-identical to the oracle's in both forms."""
    from paper_2402_14670_gb300 import qop_fit
    geo = synth.Geometry(polarity=polarity)
    g = geo_dict(geo)
    p = lfm.qop_poly_params(qop_fit.fit_qop_poly(kappa=1.2))
    b = synth.generate(1, n_events=80, geometry=geo).to("cuda")
    tr = _tracker(lfm, g, p)
    for mode in ("plain", "batched"):
        info, _, out, res = run_both(tr, b, mode=mode, geometry=g, params=p)
        assert info["n_found"] > 2000
    lin = oracle.run_batch(b, geometry=g, dumps=False)
    f = res["found"].astype(bool)
    assert np.any(res["state"][f][:, 5] != lin["state"][f][:, 5])


@pytest.mark.parametrize("cap,nt", [(1, 1), (5, 3), (17, 32), (64, 20), (32, 0)])
def test_parameter_edges(lfm, cap, nt):
    p = lfm.default_params()
    p.update(n_hits_window=cap, n_triplets=nt)
    b = synth.generate(1, n_events=40).to("cuda")
    tr = _tracker(lfm, None, p)
    for mode in ("plain", "batched"):
        run_both(tr, b, mode=mode, params=p, stages=(mode == "plain" and nt > 0))


@pytest.mark.parametrize("tuning", [dict(queue=0, blocks_per_sm=1),
                                    dict(queue=0),
                                    dict(queue=0, extend_form=1),
                                    dict(queue=0, extend_form=2, extend_bps=1, triplet_prefilter=1),
                                    dict(queue=2, warps_per_block=1, grain=1, blocks_per_sm=1),
                                    dict(queue=2, warps_per_block=4, grain=2),
                                    dict(queue=1, warps_per_block=16, grain=2),
                                    dict(queue=1, warps_per_block=8, grain=1, blocks_per_sm=2),
                                    dict(queue=1, warps_per_block=8, grain=2)])
def test_launch_shapes_identical(lfm, tuning):
    b = synth.generate(1, n_events=120).to("cuda")
    tr = _tracker(lfm)
    run_both(tr, b, mode="batched", tuning=tuning)


@pytest.mark.parametrize("cap,nt", [(32, 1), (5, 3), (32, 12), (64, 20), (17, 32), (32, 0)])
def test_extension_block_form_parameters(lfm, cap, nt):
    """The block form of the extension (a tile of min(256 / n_triplets, 32)
    tracks, one candidate per thread) at tile sizes 32, 32, 21, 12, 8 and 32
    tracks, against the oracle."""
    p = lfm.default_params()
    p.update(n_hits_window=cap, n_triplets=nt)
    b = synth.generate(1, n_events=40).to("cuda")
    tr = _tracker(lfm, None, p)
    run_both(tr, b, mode="batched", params=p, tuning=dict(queue=0, extend_form=1))


def _jitter_z(b, frac_events=0.5, seed=5):
    """Move the z of one hit in every few hundred (of half the events) by up to
    +-0.5 mm: buckets whose hits no longer share one z."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    ro = b.raw_offsets.cpu()
    z = b.z.cpu().clone()
    for e in range(b.n_events):
        if torch.rand(1, generator=g).item() >= frac_events:
            continue
        h0, h1 = int(ro[e]), int(ro[e + 1])
        n = h1 - h0
        pick = torch.randint(h0, h1, (max(1, n // 300),), generator=g)
        z[pick] += (torch.rand(len(pick), generator=g) - 0.5).to(torch.float32)
    b.z = z.to(b.z.device)
    return b


@pytest.mark.parametrize("mode,tuning", [("plain", None), ("batched", None), ("batched", dict(queue=1, grain=2)),
                                         ("batched", dict(queue=2, grain=1)),
                                         ("batched", dict(queue=0, extend_form=1))])
def test_hits_with_their_own_z(lfm, mode, tuning):
    """Hits of a layer at different z (one in a few hundred moved by up to
    0.5 mm): every kernel takes each hit's own z, as the oracle does, instead
    of a per-bucket constant."""
    b = _jitter_z(synth.generate(1, n_events=120)).to("cuda")
    tr = _tracker(lfm)
    info, *_ = run_both(tr, b, mode=mode, tuning=tuning)
    assert info["n_found"] > 3000


def test_repeated_launch_shape_direct_capture_replay(lfm):
    """The persistent form launches a new launch shape directly, captures it
    into a CUDA graph when it comes back and replays the graph after that:
    the three calls give identical outputs, also after the inputs change in
    place (a graph reads the buffers, not copies of them)."""
    b = synth.generate(1, n_events=150).to("cuda")
    tr = _tracker(lfm)
    packed = tr.pack(b)
    out = tr.alloc_output(b.n_tracks, b.n_events, "cuda")
    res = []
    for _ in range(3):
        out["found"].fill_(7)
        tr.find(packed, b, b.n_events, "batched", out=out)
        torch.cuda.synchronize()
        res.append({k: to_np(v).copy() for k, v in out.items()})
    for r in res[1:]:
        f = res[0]["found"].astype(bool)
        assert np.array_equal(r["found"], res[0]["found"])
        assert np.array_equal(r["hit_idx"][f], res[0]["hit_idx"][f])
        assert np.array_equal(r["state"][f].view(np.uint32), res[0]["state"][f].view(np.uint32))
        assert np.array_equal(r["out_trk"][:int(r["n_out"][0])], res[0]["out_trk"][:int(res[0]["n_out"][0])])
    # new input values in the same buffers: the replayed graph follows them
    b.sqop.mul_(-1.0)                                  # flip every charge: different windows and tracks
    tr.find(packed, b, b.n_events, "batched", out=out)
    torch.cuda.synchronize()
    ref = oracle.run_batch(b, dumps=False)
    compare_outputs(out, ref)
    # one output buffer replaced, the others kept: a new launch shape, so the
    # results land in the new buffers (a replay would fill the old ones)
    out2 = dict(out)
    out2["hit_idx"] = torch.full_like(out["hit_idx"], -7)
    out2["state"] = torch.full_like(out["state"], 7.0)
    for _ in range(2):
        tr.find(packed, b, b.n_events, "batched", out=out2)
        torch.cuda.synchronize()
        compare_outputs(out2, ref)


def test_ragged_and_empty_events(lfm):
    geo = synth.Geometry()
    tx, ty, q = 0.1, 0.05, 1 / 8.0
    _, y, xm = synth.trajectory(tx, ty, q)
    full = [(l, 1, float(xm[l])) for l in range(12)]
    st = synth.state_of(tx, ty, q)
    events = [
        dict(hits=[], states=[]),                        # nothing
        dict(hits=full, states=[]),                      # hits, no tracks
        dict(hits=[], states=[st, st]),                  # tracks, no hits
        dict(hits=full + [(0, 1, float(xm[0]))] * 3, states=[st]),   # duplicate x values
        dict(hits=full, states=[st] * 40),               # many identical tracks
        dict(hits=[], states=[]),
    ]
    b = make_batch(events, geo).to("cuda")
    tr = _tracker(lfm)
    for mode in ("plain", "batched"):
        info, *_ = run_both(tr, b, mode=mode, stages=(mode == "plain"))
        assert info["n_found"] == 41


def test_empty_batch(lfm):
    b = make_batch([], synth.Geometry()).to("cuda")
    tr = _tracker(lfm)
    for mode in ("plain", "batched"):
        packed, out = tr.run(b, mode=mode)
        torch.cuda.synchronize()
        assert int(to_np(out["n_out"])[0]) == 0
        assert to_np(packed["hit_offsets"]).tolist() == [0]


def test_bucket_over_capacity_is_reported(lfm):
    # one bucket above the largest sortable size: the pack skips it and flags it
    n = 16385   # LF_MAX_BUCKET + 1
    hits = [(0, 1, float(i % 5000)) for i in range(n)]
    b = make_batch([dict(hits=hits, states=[])], synth.Geometry()).to("cuda")
    tr = _tracker(lfm)
    tr.pack(b)
    with pytest.raises(lfm.LFError) as ei:
        tr.status()
    assert ei.value.status == lfm.LF_ERR_CAPACITY
    assert tr.status() == 0  # cleared


def _raw_event(rng, n, x, plane):
    z = rng.uniform(7800.0, 9400.0, n).astype(np.float32)
    d = rng.uniform(-0.1, 0.1, n).astype(np.float32)
    w = rng.uniform(100.0, 200.0, n).astype(np.float32)
    return np.asarray(x, np.float32), z, d, w, np.asarray(plane, np.uint8)


def _batch_of(parts, n_states=0):
    cat = lambda i: torch.from_numpy(np.concatenate([p[i] for p in parts]))
    nh = [len(p[0]) for p in parts]
    ro = torch.tensor(np.concatenate([[0], np.cumsum(nh)]).astype(np.int32))
    to = torch.zeros(len(parts) + 1, dtype=torch.int32)
    e = torch.zeros(0, dtype=torch.float32)
    return synth.EventBatch(len(parts), ro, cat(0), cat(1), cat(2), cat(3), cat(4), to, e, e, e, e, e)


def test_pack_paths_exact(lfm):
    """Both pack paths against the oracle, bit for bit: events sorted in one
    piece in shared memory (up to 34432 hits), larger events sorted in chunks
    of consecutive bins, and an event above 65535 hits (32-bit bins and
    indices); ties in x (ordered by raw index), -0.0 and +0.0, a skewed x
    distribution and random plane codes."""
    rng = np.random.default_rng(11)
    parts = []
    for n in (1, 3000, 34432, 34433, 50000, 70000):
        x = rng.uniform(-3000.0, 3000.0, n)
        if n >= 3000:
            x[: n // 3] = np.round(x[: n // 3] * 2.0) / 2.0     # many exact ties
            x[n // 3: n // 3 + 50] = 0.0
            x[n // 3 + 50: n // 3 + 100] = -0.0
        parts.append(_raw_event(rng, n, x, rng.integers(0, 24, n)))
    # skewed: 3000 hits inside one millimetre and one far outlier, one bucket
    x = np.concatenate([rng.uniform(10.0, 11.0, 3000), [2900.0]])
    parts.append(_raw_event(rng, 3001, x, np.full(3001, 5)))
    b = _batch_of(parts).to("cuda")
    tr = _tracker(lfm)
    packed = tr.pack(b)
    torch.cuda.synchronize()
    assert tr.status() == 0
    ref = oracle.pack(*(t.cpu().numpy() for t in (b.raw_offsets, b.x, b.z, b.dxdy, b.w, b.plane)))
    compare_pack(packed, ref)
    # the coarse index the pack writes for the window searches: every 32nd x
    xs = packed["x"].cpu().numpy()
    assert np.array_equal(packed["x_coarse"].cpu().numpy()[:(len(xs) + 31) // 32].view(np.uint32),
                          xs[::32].view(np.uint32))


def test_pack_single_x_bucket_bounded_time(lfm):
    """Adversarial x: a bucket of 16 384 hits (the largest sortable) at one
    single x, beside the same in a chunked event and a bucket with a few
    hundred hits per bin.  A bin above a few dozen hits is ordered by the
    whole block (bitonic network, O(n log^2 n)), not by one thread's insertion
    sort (O(n^2)): the pack stays bit-exact and finishes in well under a
    second."""
    rng = np.random.default_rng(13)
    n1 = 16384
    parts = [_raw_event(rng, n1, np.full(n1, 123.25), np.full(n1, 9)),
             _raw_event(rng, n1 + 30000, np.concatenate([np.full(n1, -7.5), rng.uniform(-3000, 3000, 30000)]),
                        np.concatenate([np.full(n1, 14), (14 + rng.integers(1, 24, 30000)) % 24])),
             _raw_event(rng, 12000, np.repeat(rng.uniform(-3000, 3000, 40), 300), np.full(12000, 3))]
    b = _batch_of(parts).to("cuda")
    tr = _tracker(lfm)
    tr.pack(b)                      # warm-up (module load, first launch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    packed = tr.pack(b)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert tr.status() == 0
    ref = oracle.pack(*(t.cpu().numpy() for t in (b.raw_offsets, b.x, b.z, b.dxdy, b.w, b.plane)))
    compare_pack(packed, ref)
    assert dt < 0.5, "pack of the adversarial batch took %.3f s" % dt


def test_pack_flagged_bucket_beside_sorted_ones(lfm):
    """A bucket above LF_MAX_BUCKET in an event whose other buckets are
    sorted: those match the oracle, the flagged bucket's perm is -1."""
    rng = np.random.default_rng(12)
    n_big, n_rest = 16385, 9000
    plane = np.concatenate([np.full(n_big, 7), rng.integers(8, 24, n_rest)])
    x = rng.uniform(-3000.0, 3000.0, n_big + n_rest)
    order = rng.permutation(n_big + n_rest)
    parts = [_raw_event(rng, 500, rng.uniform(-100, 100, 500), rng.integers(0, 24, 500)),
             _raw_event(rng, n_big + n_rest, x[order], plane[order])]
    b = _batch_of(parts).to("cuda")
    tr = _tracker(lfm)
    packed = tr.pack(b)
    torch.cuda.synchronize()
    with pytest.raises(lfm.LFError) as ei:
        tr.status()
    assert ei.value.status == lfm.LF_ERR_CAPACITY
    ref = oracle.pack(*(t.cpu().numpy() for t in (b.raw_offsets, b.x, b.z, b.dxdy, b.w, b.plane)))
    ho = to_np(packed["hit_offsets"])
    assert np.array_equal(ho, ref["hit_offsets"])
    lo, hi = int(ho[24 + 7]), int(ho[24 + 8])          # event 1, bucket 7
    perm = to_np(packed["perm"])
    assert np.all(perm[lo:hi] == -1)
    keep = np.ones(perm.size, bool)
    keep[lo:hi] = False
    assert np.array_equal(perm[keep], ref["perm"][keep])
    for k in ("x", "z", "dxdy", "w"):
        assert np.array_equal(to_np(packed[k])[keep].view(np.uint32), ref[k][keep].view(np.uint32))
    assert np.array_equal(to_np(packed["layer"]), ref["layer"])


def test_bad_parameters_rejected(lfm):
    p = lfm.default_params()
    p["n_hits_window"] = 65
    with pytest.raises(lfm.LFError):
        lfm.Tracker(None, p)
    p = lfm.default_params()
    p["min_hits"] = 8
    with pytest.raises(lfm.LFError):
        lfm.Tracker(None, p)


@pytest.mark.parametrize("config,n_sample,min_cmp", [(2, 48, 1000), (4, 12, 2000)])
def test_full_size_sampled(lfm, config, n_sample, min_cmp):
    """The uneven (100 000 events) and high-occupancy (20 000 events)
    workloads at full size in the launch configuration the benchmark times;
    the oracle recomputes a sample of events one by one (plus the events with
    the most tracks and hits, and the last)."""
    b = synth.generate(config, device="cuda", truth=False)
    tr = _tracker(lfm)
    packed, out = tr.run(b, mode="batched")
    torch.cuda.synchronize()
    assert tr.status() == 0
    ro = to_np(b.raw_offsets).astype(np.int64)
    to = to_np(b.trk_offsets).astype(np.int64)
    ntrk = np.diff(to)
    rng = np.random.default_rng(5)
    sample = sorted(set(rng.choice(b.n_events, n_sample, replace=False).tolist()) |
                    {int(np.argmax(ntrk)), int(np.argmax(np.diff(ro))), b.n_events - 1})
    sub = b.select_events(sample).to("cpu")
    res = oracle.run_batch(sub, dumps=False)
    perm_g = to_np(packed["perm"])
    found_g = to_np(out["found"]).astype(bool)
    hit_g = to_np(out["hit_idx"])
    st_g = to_np(out["state"])
    q_g = to_np(out["quality"])
    ro_s = to_np(sub.raw_offsets).astype(np.int64)
    to_s = to_np(sub.trk_offsets).astype(np.int64)
    perm_o = res["packed"]["perm"]
    n_cmp = 0
    for k, e in enumerate(sample):
        for j in range(to_s[k + 1] - to_s[k]):
            ts, tg = to_s[k] + j, to[e] + j
            assert bool(res["found"][ts]) == found_g[tg], ("found", e, j)
            if not found_g[tg]:
                continue
            raw_o = [ro[e] + (perm_o[h] - ro_s[k]) if h >= 0 else -1 for h in res["hit_idx"][ts]]
            raw_g = [perm_g[h] if h >= 0 else -1 for h in hit_g[tg]]
            assert raw_o == raw_g, ("hits", e, j)
            assert np.array_equal(st_g[tg].view(np.uint32), res["state"][ts].view(np.uint32)), ("state", e, j)
            assert q_g[tg] == res["quality"][ts]
            n_cmp += 1
    assert n_cmp > min_cmp
    # compaction over the whole batch
    f = found_g.astype(np.int64)
    cnt = np.add.reduceat(f, to[:-1]) if f.size else f
    cnt = np.where(ntrk > 0, cnt, 0)
    assert np.array_equal(to_np(out["out_offsets"]), np.concatenate([[0], np.cumsum(cnt)]))
    n_out = int(to_np(out["n_out"])[0])
    assert np.array_equal(to_np(out["out_trk"])[:n_out], np.nonzero(found_g)[0])


@pytest.mark.parametrize("chunk_hits", [0, 150_000])
def test_end_to_end_host_pipeline(lfm, chunk_hits):
    """lf_process_host (host buffers, chunked and double-buffered) gives the
    device path's results, with hit indices mapped back to raw indices."""
    b = synth.generate(1, n_events=120)           # host tensors
    bp = b.pin_memory()
    tr = _tracker(lfm)
    ho = tr.process_host(bp, chunk_hits=chunk_hits)
    packed, out = tr.run(b.to("cuda"), mode="batched")
    torch.cuda.synchronize()
    found = to_np(out["found"]).astype(bool)
    assert np.array_equal(ho["found"].numpy().astype(bool), found)
    perm = to_np(packed["perm"])
    hd = to_np(out["hit_idx"])[found]
    raw = np.where(hd >= 0, perm[np.maximum(hd, 0)], -1)
    assert np.array_equal(ho["hit_idx"].numpy()[found], raw)
    assert np.array_equal(ho["state"].numpy()[found].view(np.uint32), to_np(out["state"])[found].view(np.uint32))
    res = oracle.run_batch(b, dumps=False)
    assert np.array_equal(res["found"].astype(bool), found)


def test_end_to_end_refuses_bad_offsets(lfm):
    """lf_process_host checks the host offsets before any copy: decreasing
    offsets are refused with LF_ERR_ARG and the context stays usable."""
    b = synth.generate(1, n_events=8)             # host tensors
    tr = _tracker(lfm)
    ro = b.raw_offsets.clone()
    assert int(ro[2]) < int(ro[3])
    b.raw_offsets[2] = ro[3]
    b.raw_offsets[3] = ro[2]                      # same ends, decreasing at event 2
    with pytest.raises(lfm.LFError) as ei:
        tr.process_host(b)
    assert ei.value.status == lfm.LF_ERR_ARG
    b.raw_offsets.copy_(ro)
    ho = tr.process_host(b)
    assert int(ho["found"].sum()) > 0


def test_host_arena_is_page_locked(lfm):
    """lf_host_alloc gives exact-size page-locked memory that torch sees as
    pinned, so copies from it are asynchronous."""
    ar = lfm.HostArena(5 * (1 << 20) + 17)
    try:
        a = ar.take(1 << 20, torch.float32)
        b = ar.take(5, torch.uint8)
        assert a.is_pinned() and b.is_pinned()
        assert a.data_ptr() % 256 == 0 and b.data_ptr() % 256 == 0
        a.copy_(torch.arange(a.numel(), dtype=torch.float32))
        d = a.to("cuda", non_blocking=True)
        torch.cuda.synchronize()
        assert torch.equal(d.cpu(), a)
        with pytest.raises(ValueError):
            ar.take(1 << 20, torch.float32)
    finally:
        ar.close()


@pytest.mark.parametrize("mode,tuning", [("plain", None), ("batched", None), ("batched", dict(queue=1, grain=2))])
def test_coarse_index_from_the_pack_or_the_find(lfm, mode, tuning):
    """The window searches give the same results whether the coarse index
    comes from the pack (lf_packed.x_coarse) or is computed by the find
    (a batch without it), and both agree with the oracle."""
    b = synth.generate(2, n_events=300, seed=17).to("cuda")
    tr = _tracker(lfm)
    packed = tr.pack(b)
    with_idx = tr.find(packed, b, b.n_events, mode, tuning)
    bare = {k: v for k, v in packed.items() if k != "x_coarse"}
    without = tr.find(bare, b, b.n_events, mode, tuning)
    torch.cuda.synchronize()
    assert tr.status() == 0
    for k in ("found", "out_offsets", "n_out"):
        assert torch.equal(with_idx[k], without[k]), k
    f = with_idx["found"].bool()          # per-track outputs are written for found tracks only
    for k in ("nhits", "hit_idx"):
        assert torch.equal(with_idx[k][f], without[k][f]), k
    for k in ("state", "quality"):
        assert torch.equal(with_idx[k][f].view(torch.int32), without[k][f].view(torch.int32)), k
    run_both(tr, b, mode=mode, tuning=tuning)


def test_validate_batch(lfm):
    """lf_validate_batch (debug mode, outside the hot path) passes a packed
    batch and names the first broken convention: a decreasing or
    out-of-range hit offset, track offsets that do not end at n_tracks, x out
    of order inside a bucket (also NaN), a coarse index that differs from x."""
    import copy
    b = synth.generate(1, n_events=50).to("cuda")
    tr = _tracker(lfm)
    packed = tr.pack(b)
    torch.cuda.synchronize()
    tr.validate(packed, b, b.n_events)

    def fails(pk, st, pattern):
        with pytest.raises(lfm.LFError, match=pattern) as ei:
            tr.validate(pk, st, b.n_events)
        assert ei.value.status == lfm.LF_ERR_ARG

    ho = packed["hit_offsets"]
    bad = dict(packed, hit_offsets=ho.clone())
    bad["hit_offsets"][30] = ho[31] + 1
    fails(bad, b, r"hit_offsets\[30\]")
    bad = dict(packed, hit_offsets=ho.clone())
    bad["hit_offsets"][-1] = b.n_hits + 5
    fails(bad, b, r"hit_offsets\[%d\]" % (24 * b.n_events))
    st = copy.copy(b)
    st.trk_offsets = b.trk_offsets.clone()
    st.trk_offsets[-1] -= 1
    fails(packed, st, r"trk_offsets\[%d\]" % b.n_events)
    # two hits of one bucket swapped (the first bucket with two distinct x)
    hoh = to_np(ho)
    xs = to_np(packed["x"])
    q = next(q for q in range(24 * b.n_events) if hoh[q + 1] - hoh[q] >= 2 and xs[hoh[q]] < xs[hoh[q] + 1])
    s0 = int(hoh[q])
    x2 = packed["x"].clone()
    x2[s0], x2[s0 + 1] = packed["x"][s0 + 1], packed["x"][s0]
    fails(dict(packed, x=x2, x_coarse=None), b, r"packed hits %d and %d" % (s0, s0 + 1))
    x3 = packed["x"].clone()
    x3[s0 + 1] = float("nan")
    fails(dict(packed, x=x3, x_coarse=None), b, r"packed hits %d and %d" % (s0, s0 + 1))
    xc = packed["x_coarse"].clone()
    xc[3] += 1.0
    fails(dict(packed, x_coarse=xc), b, r"x_coarse\[3\]")
    tr.validate(packed, b, b.n_events)      # the packed batch itself still passes
