"""Slot form (lf_process_slot): one captured graph per slot serves batches of
every size, reading the batch's event count from device memory; its results
are bit-identical to lf_pack_hits + lf_find_tracks_batched on the same
batch, with the slot's own hit buffers and when it gathers the batch's
events (any subset, in any order) from a device-resident pool."""
import numpy as np
import pytest
import torch

from paper_2402_14670_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_14670_gb300 import build
    build.build()
    from paper_2402_14670_gb300 import lf
    return lf


@pytest.fixture(scope="module")
def pool():
    return synth.generate(2, n_events=400, seed=11)


def _reference(lf, tr, pool_cpu, idx, tuning):
    b = pool_cpu.select_events(idx).to("cuda")
    packed, out = tr.run(b, mode="batched", tuning=tuning)
    torch.cuda.synchronize()
    return b, packed, out


def _fill_offsets(slot, pool_cpu, idx):
    ro = pool_cpu.raw_offsets.numpy().astype(np.int64)
    to = pool_cpu.trk_offsets.numpy().astype(np.int64)
    nh = ro[np.asarray(idx) + 1] - ro[idx]
    nt = to[np.asarray(idx) + 1] - to[idx]
    r_off = np.concatenate([[0], np.cumsum(nh)]).astype(np.int32)
    t_off = np.concatenate([[0], np.cumsum(nt)]).astype(np.int32)
    n = len(idx)
    slot.raw_offsets[:n + 1].copy_(torch.from_numpy(r_off))
    slot.trk_offsets[:n + 1].copy_(torch.from_numpy(t_off))
    slot.hit_src[:n].copy_(torch.from_numpy(ro[idx].astype(np.int32)))
    slot.trk_src[:n].copy_(torch.from_numpy(to[idx].astype(np.int32)))
    slot.n_dev.fill_(n)
    return int(r_off[-1]), int(t_off[-1])


def _compare(slot, n, nh, nt, packed, out):
    o = slot.out
    f = o["found"][:nt].cpu().numpy()
    assert np.array_equal(f, out["found"].cpu().numpy())
    fb = f.astype(bool)
    assert np.array_equal(o["nhits"][:nt].cpu().numpy()[fb], out["nhits"].cpu().numpy()[fb])
    assert np.array_equal(o["hit_idx"][:nt].cpu().numpy()[fb], out["hit_idx"].cpu().numpy()[fb])
    assert np.array_equal(o["state"][:nt].cpu().numpy()[fb].view(np.uint32),
                          out["state"].cpu().numpy()[fb].view(np.uint32))
    assert np.array_equal(o["quality"][:nt].cpu().numpy()[fb].view(np.uint32),
                          out["quality"].cpu().numpy()[fb].view(np.uint32))
    assert np.array_equal(o["out_offsets"][:n + 1].cpu().numpy(), out["out_offsets"].cpu().numpy())
    m = int(out["n_out"].item())
    assert int(o["n_out"].item()) == m
    assert np.array_equal(o["out_trk"][:m].cpu().numpy(), out["out_trk"][:m].cpu().numpy())
    assert np.array_equal(slot.packed["perm"][:nh].cpu().numpy(), packed["perm"].cpu().numpy())
    assert np.array_equal(slot.packed["hit_offsets"][:24 * n + 1].cpu().numpy(), packed["hit_offsets"].cpu().numpy())
    assert np.array_equal(slot.packed["x"][:nh].cpu().numpy().view(np.uint32),
                          packed["x"].cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("tuning", [None, {"queue": 1, "warps_per_block": 8, "grain": 2}],
                         ids=["stages", "tile"])
def test_slot_gather_one_graph_many_sizes(mods, pool, tuning):
    lf = mods
    rng = np.random.default_rng(5)
    dpool = pool.to("cuda")
    tr = lf.Tracker()
    ref_tr = lf.Tracker()
    cap_ev = 160
    cap_h = int(np.sort(np.diff(pool.raw_offsets.numpy()))[::-1][:cap_ev].sum())
    cap_t = int(np.sort(np.diff(pool.trk_offsets.numpy()))[::-1][:cap_ev].sum())
    slot = lf.SlotBuffers(cap_ev, cap_h, cap_t, "cuda", own_raw=False)
    g0 = tr.graph_count()
    sizes = [1, 37, 160, 0, 96, 5]
    for k, n in enumerate(sizes):
        if k % 2:
            idx = np.sort(rng.choice(pool.n_events, n, replace=False))       # any subset
        else:
            s0 = int(rng.integers(0, pool.n_events - n + 1))
            idx = np.arange(s0, s0 + n)[::-1].copy()                          # a reversed run
        nh, nt = _fill_offsets(slot, pool, idx)
        tr.process_slot(slot, dpool, tuning)
        torch.cuda.synchronize()
        assert tr.status() == 0
        if n == 0:
            assert int(slot.out["n_out"].item()) == 0
            continue
        _, packed, out = _reference(lf, ref_tr, pool, idx, tuning)
        _compare(slot, n, nh, nt, packed, out)
    # one graph for every batch of this slot
    assert tr.graph_count() - g0 == 1
    tr.close()
    ref_tr.close()


def test_slot_own_buffers(mods, pool):
    lf = mods
    tr = lf.Tracker()
    ref_tr = lf.Tracker()
    cap_ev = 64
    cap_h = int(np.sort(np.diff(pool.raw_offsets.numpy()))[::-1][:cap_ev].sum())
    cap_t = int(np.sort(np.diff(pool.trk_offsets.numpy()))[::-1][:cap_ev].sum())
    slot = lf.SlotBuffers(cap_ev, cap_h, cap_t, "cuda", own_raw=True)
    ro = pool.raw_offsets.numpy()
    to = pool.trk_offsets.numpy()
    g0 = tr.graph_count()
    for e0, n in ((0, 64), (100, 3), (200, 50)):
        idx = np.arange(e0, e0 + n)
        h0, h1, t0, t1 = int(ro[e0]), int(ro[e0 + n]), int(to[e0]), int(to[e0 + n])
        for f in ("x", "z", "dxdy", "w", "plane"):
            slot.raw[f][:h1 - h0].copy_(getattr(pool, f)[h0:h1])
        for f in ("sx", "sy", "stx", "sty", "sqop"):
            slot.states[f][:t1 - t0].copy_(getattr(pool, f)[t0:t1])
        slot.raw_offsets[:n + 1].copy_(torch.from_numpy((ro[e0:e0 + n + 1] - h0).astype(np.int32)))
        slot.trk_offsets[:n + 1].copy_(torch.from_numpy((to[e0:e0 + n + 1] - t0).astype(np.int32)))
        slot.n_dev.fill_(n)
        tr.process_slot(slot)
        torch.cuda.synchronize()
        _, packed, out = _reference(lf, ref_tr, pool, idx, None)
        _compare(slot, n, h1 - h0, t1 - t0, packed, out)
    assert tr.graph_count() - g0 == 1
    tr.close()
    ref_tr.close()


def test_slot_count_clamped_to_capacity(mods, pool):
    """A device event count above the slot's capacity is clamped to it."""
    lf = mods
    tr = lf.Tracker()
    ref_tr = lf.Tracker()
    cap_ev = 24
    idx = np.arange(cap_ev)
    nh_all = int(pool.raw_offsets[cap_ev]) + 1
    nt_all = int(pool.trk_offsets[cap_ev]) + 1
    slot = lf.SlotBuffers(cap_ev, nh_all, nt_all, "cuda", own_raw=False)
    nh, nt = _fill_offsets(slot, pool, idx)
    slot.n_dev.fill_(cap_ev + 1000)
    tr.process_slot(slot, pool.to("cuda"))
    torch.cuda.synchronize()
    _, packed, out = _reference(lf, ref_tr, pool, idx, None)
    _compare(slot, cap_ev, nh, nt, packed, out)
    tr.close()
    ref_tr.close()


def test_slot_rejects_batch_arrays_other_than_the_packed_ones(mods, pool):
    lf = mods
    tr = lf.Tracker()
    slot = lf.SlotBuffers(8, 200000, 2000, "cuda", own_raw=True)
    raw, pk, b, o = slot.structs()
    other = torch.empty(200000, dtype=torch.float32, device="cuda")
    b.x = other.data_ptr()
    with pytest.raises(lf.LFError) as ei:
        lf.lf_process_slot(tr.ctx, raw, pk, b, None, slot.n_dev.data_ptr(), o, None, None)
    assert ei.value.status == lf.LF_ERR_ARG
    raw, pk, b, o = slot.structs()
    b.n_hits = slot.max_hits - 1          # capacities of raw and batch differ
    with pytest.raises(lf.LFError) as ei:
        lf.lf_process_slot(tr.ctx, raw, pk, b, None, slot.n_dev.data_ptr(), o, None, None)
    assert ei.value.status == lf.LF_ERR_ARG
    tr.close()


def test_graph_cache_keeps_the_most_recent_shapes(mods, pool):
    """More launch shapes than the cache holds (64): the least recently used
    graphs are dropped and recaptured when they come back; every replay gives
    the direct launch's results."""
    lf = mods
    b = pool.select_events(range(40)).to("cuda")
    tr = lf.Tracker()
    packed = tr.pack(b)
    ref = tr.find(packed, b, b.n_events, "batched")
    torch.cuda.synchronize()
    outs = [lf.Tracker.alloc_output(b.n_tracks, b.n_events, "cuda") for _ in range(70)]
    g0 = tr.graph_count()
    for rep in range(3):
        for o in outs:                      # each output set is a launch shape of its own
            for k in ("found", "nhits"):
                o[k].fill_(7)
            tr.find(packed, b, b.n_events, "batched", out=o)
        torch.cuda.synchronize()
        m = int(ref["n_out"].item())
        for o in outs:
            assert torch.equal(o["found"], ref["found"]) and int(o["n_out"].item()) == m
            assert torch.equal(o["out_trk"][:m], ref["out_trk"][:m])
    # first pass: launched directly (first sight); second: 70 captures, the
    # oldest 6 dropped; third: the 6 oldest (and those they push out) again
    n = tr.graph_count() - g0
    assert n >= 70 and n <= 140
    tr.close()
