"""lf_find_tracks_static: the entry point for callers that cannot allocate.

Some callers may not call cudaMalloc (their device memory is owned by their
own pool, or allocation is forbidden on their latency-critical path), so they
cannot create a context.  lf_find_tracks_static runs the persistent form with
its scratch in a static device array instead.  This test calls it through the
C ABI and checks it against lf_find_tracks_batched on two calls in a row (two
different batches, so the second call starts from the array the first one
left behind), and checks the size limit.  It sits in its own file, collected
last, and passes alone in a fresh process or after the other tests.
"""
import numpy as np
import pytest
import torch

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


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("cap,nt", [(32, 12), (16, 12), (64, 12), (32, 20)])
def test_static_entry_point_matches_batched(lfm, cap, nt):
    """Window caps 16/32/64 select different kernel instantiations; more than
    16 kept triplets put one track instead of two on a warp."""
    p = lfm.default_params()
    p.update(n_hits_window=cap, n_triplets=nt)
    tr = lfm.Tracker(None, p)
    stream = torch.cuda.current_stream()
    for config, n_ev in ((1, 300), (2, 150)):   # two calls in a row, different batches
        b = synth.generate(config, n_events=n_ev).to("cuda")
        packed = tr.pack(b)
        ref = tr.find(packed, b, b.n_events, "batched")
        out = tr.alloc_output(b.n_tracks, b.n_events, "cuda")
        out["found"].fill_(7)
        out["n_out"].fill_(-1)
        bs = tr.batch_struct(packed, b, b.n_events)
        os_ = tr.output_struct(out)
        lfm.lf_find_tracks_static(tr.geometry, tr.params, bs, os_, lfm._P(stream.cuda_stream))
        torch.cuda.synchronize()
        found = _np(ref["found"]).astype(bool)
        assert np.array_equal(_np(out["found"]).astype(bool), found)
        assert found.sum() > 1000
        assert np.array_equal(_np(out["nhits"])[found], _np(ref["nhits"])[found])
        assert np.array_equal(_np(out["hit_idx"])[found], _np(ref["hit_idx"])[found])
        s, r = _np(out["state"])[found].astype(np.float64), _np(ref["state"])[found].astype(np.float64)
        assert np.all(np.abs(s - r) <= 1e-6 + 1e-4 * np.abs(r))
        q, rq = _np(out["quality"])[found].astype(np.float64), _np(ref["quality"])[found].astype(np.float64)
        assert np.all(np.abs(q - rq) <= 1e-7 + 1e-4 * np.abs(rq))
        assert np.array_equal(_np(out["out_offsets"]), _np(ref["out_offsets"]))
        n_out = int(_np(out["n_out"])[0])
        assert n_out == int(_np(ref["n_out"])[0])
        assert np.array_equal(_np(out["out_trk"])[:n_out], _np(ref["out_trk"])[:n_out])
    tr.close()


def test_static_entry_point_events_without_tracks(lfm):
    """Events without input tracks: no track kernel runs, the compaction
    still writes every event's offset and n_out = 0 over the shared array
    the previous call left behind."""
    tr = lfm.Tracker()
    stream = torch.cuda.current_stream()
    b = synth.generate(1, n_events=50).to("cuda")
    packed = tr.pack(b)
    out = tr.alloc_output(b.n_tracks, b.n_events, "cuda")
    lfm.lf_find_tracks_static(tr.geometry, tr.params, tr.batch_struct(packed, b, b.n_events),
                              tr.output_struct(out), lfm._P(stream.cuda_stream))
    torch.cuda.synchronize()
    assert int(_np(out["n_out"])[0]) > 0
    # the same hits with every event's track range empty
    b.trk_offsets = torch.zeros_like(b.trk_offsets)
    for k in ("sx", "sy", "stx", "sty", "sqop"):
        setattr(b, k, getattr(b, k)[:0])
    out0 = tr.alloc_output(0, b.n_events, "cuda")
    out0["out_offsets"].fill_(-5)
    out0["n_out"].fill_(-1)
    lfm.lf_find_tracks_static(tr.geometry, tr.params, tr.batch_struct(packed, b, b.n_events),
                              tr.output_struct(out0), lfm._P(stream.cuda_stream))
    torch.cuda.synchronize()
    assert int(_np(out0["n_out"])[0]) == 0
    assert np.array_equal(_np(out0["out_offsets"]), np.zeros(b.n_events + 1, np.int32))
    tr.close()


def test_static_entry_point_rejects_oversize(lfm):
    tr = lfm.Tracker()
    b = synth.generate(0).to("cuda")
    packed = tr.pack(b)
    out = tr.alloc_output(b.n_tracks, b.n_events, "cuda")
    bs = tr.batch_struct(packed, b, b.n_events)
    bs.n_events = 262144 + 1            # above LF_STATIC_MAX_EVENTS: refused before any launch
    with pytest.raises(lfm.LFError) as ei:
        lfm.lf_find_tracks_static(tr.geometry, tr.params, bs, tr.output_struct(out),
                                  lfm._P(torch.cuda.current_stream().cuda_stream))
    assert ei.value.status == lfm.LF_ERR_CAPACITY
    tr.close()
