"""The no-UT variant (Sec. "No-UT tuning") on the GPU against the oracle.

Both forms that follow it (plain stages, and the persistent staged pipeline)
must give the oracle's two window sets per track, its pooled triplet list
(side bit included), hit lists, states and Q bit for bit.
"""
import numpy as np
import pytest
import torch

from helpers import geo_dict, make_batch, track_hits
from parity import run_both
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


def _p(lfm, **kw):
    p = lfm.no_ut_params()
    p.update(kw)
    return p


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_no_ut_tiny_event(lfm, mode):
    p = _p(lfm)
    b = synth.generate(0).to("cuda")
    info, *_ = run_both(lfm.Tracker(None, p), b, mode=mode, params=p, stages=True)
    assert info["n_found"] >= 5


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_no_ut_minimum_bias_subset(lfm, mode):
    p = _p(lfm)
    b = synth.generate(1, n_events=150).to("cuda")
    info, *_ = run_both(lfm.Tracker(None, p), b, mode=mode, params=p, stages=(mode == "plain"))
    assert info["n_found"] > 2500


def test_no_ut_high_occupancy_subset(lfm):
    # ~1000 hits per bucket: the 64-hit cap binds on most one-sided windows
    p = _p(lfm)
    b = synth.generate(4, n_events=12).to("cuda")
    info, *_ = run_both(lfm.Tracker(None, p), b, mode="batched", params=p, stages=True)
    assert info["n_found"] > 300


def test_no_ut_uneven_subset(lfm):
    p = _p(lfm)
    b = synth.generate(2, n_events=120).to("cuda")
    run_both(lfm.Tracker(None, p), b, mode="batched", params=p)


def test_no_ut_magdown(lfm):
    geo = synth.Geometry(polarity=-1)
    g = geo_dict(geo)
    p = _p(lfm)
    b = synth.generate(1, n_events=60, geometry=geo).to("cuda")
    tr = lfm.Tracker(g, p)
    run_both(tr, b, mode="plain", geometry=g, params=p, stages=True)
    run_both(tr, b, mode="batched", geometry=g, params=p)


@pytest.mark.parametrize("cap,nt", [(1, 1), (17, 5), (33, 32), (64, 0)])
def test_no_ut_parameter_edges(lfm, cap, nt):
    p = _p(lfm, n_hits_window=cap, n_triplets=nt)
    b = synth.generate(1, n_events=30).to("cuda")
    tr = lfm.Tracker(None, p)
    for mode in ("plain", "batched"):
        run_both(tr, b, mode=mode, params=p, stages=(mode == "plain" and nt > 0))


def test_no_ut_overlap_twins_and_ragged(lfm):
    """Hits in the 5 mm overlap seed the same triplets on both sides (equal
    chi2, side 0 first); events without hits or tracks sit in between."""
    p = _p(lfm)
    straight = [(l, 1, 100.0) for l in (0, 3, 4, 7, 8, 11)]
    tx, ty, q = 0.04, 0.07, 1.0 / 5000.0
    events = [dict(hits=straight, states=[(100.0, 270.0, 0.0, 0.07, 0.0)]),
              dict(hits=[], states=[]),
              dict(hits=[], states=[synth.state_of(tx, ty, q)]),
              dict(hits=track_hits(tx, ty, q), states=[synth.state_of(tx, ty, q), synth.state_of(-tx, ty, q)]),
              dict(hits=straight, states=[])]
    b = make_batch(events).to("cuda")
    tr = lfm.Tracker(None, p)
    for mode in ("plain", "batched"):
        info, _, _, res = run_both(tr, b, mode=mode, params=p, stages=True)
        assert list(res["trip"][0, :4, 0]) == [0, 1, 2, 3]
        assert res["found"][2]   # the 5 TeV particle (tracks: 0 | - | 1 | 2, 3 | -)


def test_no_ut_tile_forms_refused(lfm):
    p = _p(lfm)
    tr = lfm.Tracker(None, p)
    b = synth.generate(1, n_events=4).to("cuda")
    packed = tr.pack(b)
    for q in (1, 2):
        with pytest.raises(lfm.LFError):
            tr.find(packed, b, b.n_events, "batched", dict(queue=q))
    out = tr.alloc_output(b.n_tracks, b.n_events, packed["x"].device)
    with pytest.raises(lfm.LFError) as ei:
        lfm.lf_find_tracks_static(tr.geometry, tr.params, tr.batch_struct(packed, b, b.n_events),
                                  tr.output_struct(out), lfm._P(torch.cuda.current_stream().cuda_stream))
    assert ei.value.status == lfm.LF_ERR_ARG
    tr.close()
