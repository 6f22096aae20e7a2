"""Continuous-batching server: each event's result is the same served alone
(one event per batch) as served in a mix (many events per batch, several
batches in flight on several streams, batched by size or in arrival order,
fed from host memory through the arrival ring or read in place from device
memory), and equals the whole-batch path."""
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
    from paper_2402_14670_gb300 import lf, serve
    return lf, serve


def _same(a, b):
    assert np.array_equal(a["found"], b["found"])
    f = a["found"]
    assert np.array_equal(a["hits"][f], b["hits"][f])
    assert np.array_equal(a["nhits"][f], b["nhits"][f])
    assert np.array_equal(a["state"][f].view(np.uint32), b["state"][f].view(np.uint32))
    assert np.array_equal(a["quality"][f].view(np.uint32), b["quality"][f].view(np.uint32))


@pytest.mark.parametrize("where,group", [("host", True), ("device", True), ("device", False)],
                         ids=["host-fed-by-size", "device-by-size", "device-arrival-order"])
def test_served_alone_equals_in_mix(mods, where, group):
    lf, serve = mods
    n = 96
    pool = synth.generate(1, n_events=n).pin_memory()
    src = pool if where == "host" else pool.to("cuda")
    srv = serve.Server(src, n_slots=4, max_events=32, keep_results=True, budget_bytes=4 << 30, group_by_size=group)
    g0 = sum(sl.tr.graph_count() for sl in srv.slots)
    st_alone = srv.run(np.arange(n) * 0.004)          # spaced out: one event per batch
    alone = dict(srv.results)
    srv.results = {}
    st_mix = srv.run(np.zeros(n))                      # all at once: full batches, slots overlapping
    mix = dict(srv.results)
    # one graph per slot (default launch shape) for every batch
    assert sum(sl.tr.graph_count() for sl in srv.slots) - g0 <= len(srv.slots)
    srv.close()
    assert st_alone.mean_batch_events < 1.5
    assert st_mix.mean_batch_events > 4
    assert len(alone) == len(mix) == n
    for e in range(n):
        _same(alone[e], mix[e])
    # and the same as the whole batch through the device path
    b = pool.to("cuda")
    tr = lf.Tracker()
    packed, out = tr.run(b, mode="batched")
    torch.cuda.synchronize()
    perm = packed["perm"].cpu().numpy()
    ro = pool.raw_offsets.numpy()
    to = pool.trk_offsets.numpy()
    found = out["found"].cpu().numpy().astype(bool)
    hits = out["hit_idx"].cpu().numpy()
    n_found = 0
    for e in range(n):
        a, c = to[e], to[e + 1]
        f = found[a:c]
        ok = (hits[a:c] >= 0) & f[:, None]
        raw = np.where(ok, perm[np.where(ok, hits[a:c], 0)] - ro[e], -1)
        assert np.array_equal(f, mix[e]["found"])
        assert np.array_equal(raw[f], mix[e]["hits"][f])
        n_found += int(f.sum())
    assert n_found > 1000


def test_admission_budget_limits_inflight(mods):
    lf, serve = mods
    pool = synth.generate(1, n_events=64).pin_memory()
    budget = 64 << 20   # smaller than two full batches
    srv = serve.Server(pool, n_slots=4, max_events=16, keep_results=False, budget_bytes=budget)
    st = srv.run(np.zeros(64))
    srv.close()
    assert st.n_events == 64
    assert st.max_inflight_bytes <= max(budget, 0) or st.n_batches >= 4


def test_device_resident_pool_matches_host_pool(mods):
    """Events already in device memory (read in place by the slots) give the
    same per-event results as events copied in from host memory through the
    arrival ring."""
    lf, serve = mods
    pool = synth.generate(1, n_events=80)
    res = []
    for p in (pool.pin_memory(), pool.to("cuda")):
        srv = serve.Server(p, n_slots=3, max_events=24, keep_results=True, budget_bytes=4 << 30)
        st = srv.run(np.zeros(80))
        assert st.n_events == 80 and st.mean_batch_events > 4
        res.append(dict(srv.results))
        srv.close()
    assert len(res[0]) == len(res[1]) == 80
    for e in range(80):
        _same(res[0][e], res[1][e])


def test_arrival_ring_wraps(mods):
    """A small budget gives a ring of a few slots' worth of events: all
    arrivals at once make it wrap several times, and every event's result is
    still the one read in place from device memory."""
    lf, serve = mods
    pool = synth.generate(1, n_events=96, seed=21)
    res = []
    for p in (pool.pin_memory(), pool.to("cuda")):
        srv = serve.Server(p, n_slots=4, max_events=8, keep_results=True, budget_bytes=8 << 20)
        if srv.ring is not None:
            assert srv.ring.cap_h * 3 < int(pool.raw_offsets[-1])      # the pool passes through it 3+ times
        st = srv.run(np.zeros(96))
        assert st.n_events == 96
        if srv.ring is not None:
            assert srv.ring.vh > 3 * srv.ring.cap_h
        res.append(dict(srv.results))
        srv.close()
    for e in range(96):
        _same(res[0][e], res[1][e])
