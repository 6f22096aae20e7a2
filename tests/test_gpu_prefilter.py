"""The half-precision pre-filter of the triplet pairs (lf_tuning.triplet_prefilter,
Sec. "Performance": the triplet seeding's chi2 in half2 arithmetic, every
kept pair re-checked in binary32).

With the pre-filter the persistent triplet kernel must keep exactly the
oracle's triplet lists (decoded from the stage pipeline's own scratch, not
from a re-run of the plain form), and the outputs must stay bit-identical:
on the three workloads' slices, at other window caps (an odd cap, whose last
hit has no partner in its binary16 pair), a wider triplet cut, the paper's K
constants, and hits that do not share one z per layer (where the pre-filter
does not apply).  It is refused where it does not run.
"""
import numpy as np
import pytest
import torch

import oracle
from parity import compare_outputs, compare_pack, to_np
from paper_2402_14670_gb300 import synth

pytestmark = pytest.mark.gpu

HP = dict(queue=0, triplet_prefilter=1)


@pytest.fixture(scope="module")
def lfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_14670_gb300 import build
    build.build()
    from paper_2402_14670_gb300 import lf
    return lf


def _compare_triplets(trip: dict, res: dict) -> int:
    nt_g = to_np(trip["n_trip"])
    assert np.array_equal(nt_g, res["n_trip"]), "triplet counts differ: %s" % np.nonzero(nt_g != res["n_trip"])[0][:10]
    tg, cg = to_np(trip["trip"]), to_np(trip["trip_chi2"])
    for t in np.nonzero(nt_g)[0]:
        n = nt_g[t]
        assert np.array_equal(tg[t, :n], res["trip"][t, :n]), ("triplets", t, tg[t, :n], res["trip"][t, :n])
        assert np.array_equal(cg[t, :n].view(np.uint32), res["trip_chi2"][t, :n].view(np.uint32)), ("chi2", t)
    return int(nt_g.sum())


def _run(lfm, b, params=None):
    tr = lfm.Tracker(None, params)
    packed, out = tr.run(b, mode="batched", tuning=HP)
    trip = tr.last_triplets(packed, b, b.n_events)
    torch.cuda.synchronize()
    assert tr.status() == 0
    res = oracle.run_batch(b, params=params, dumps=True)
    compare_pack(packed, res["packed"])
    n_trip = _compare_triplets(trip, res)
    info = compare_outputs(out, res)
    tr.close()
    return n_trip, info


@pytest.mark.parametrize("config,n_events", [(0, None), (1, 300), (2, 120), (4, 20)])
def test_prefilter_exact(lfm, config, n_events):
    b = synth.generate(config, n_events=n_events).to("cuda")
    n_trip, info = _run(lfm, b)
    assert n_trip >= info["n_found"] > 0
    assert info["n_found"] >= (10 if config == 0 else 500)


@pytest.mark.parametrize("cap,nt,T", [(16, 12, 8.0), (25, 12, 8.0), (64, 20, 8.0), (32, 12, 60.0), (32, 12, 3000.0)])
def test_prefilter_parameters(lfm, cap, nt, T):
    """T = 3000: sqrt(T) + margin above 2048 - PF_SPAN, where the pre-filter
    switches itself off."""
    p = lfm.default_params()
    p.update(n_hits_window=cap, n_triplets=nt, T_triplet=T)
    b = synth.generate(1, n_events=60).to("cuda")
    _run(lfm, b, p)


def test_prefilter_paper_constants(lfm):
    p = oracle.default_params(paper_K=True)
    b = synth.generate(1, n_events=60).to("cuda")
    _run(lfm, b, p)


def test_prefilter_hits_with_their_own_z(lfm):
    from test_gpu_parity import _jitter_z
    b = _jitter_z(synth.generate(1, n_events=80)).to("cuda")
    _run(lfm, b)


def test_prefilter_refused_where_it_does_not_run(lfm):
    b = synth.generate(0).to("cuda")
    tr = lfm.Tracker()
    packed = tr.pack(b)
    with pytest.raises(lfm.LFError) as ei:
        tr.find(packed, b, b.n_events, "batched", dict(queue=1, grain=2, triplet_prefilter=1))
    assert ei.value.status == lfm.LF_ERR_ARG
    with pytest.raises(lfm.LFError) as ei:
        tr.find(packed, b, b.n_events, "batched", dict(queue=0, triplet_prefilter=2))
    assert ei.value.status == lfm.LF_ERR_ARG
    tr.close()
    tn = lfm.Tracker(None, oracle.no_ut_params())
    packed = tn.pack(b)
    with pytest.raises(lfm.LFError) as ei:
        tn.find(packed, b, b.n_events, "batched", HP)
    assert ei.value.status == lfm.LF_ERR_ARG
    # the block form of the extension likewise
    with pytest.raises(lfm.LFError) as ei:
        tn.find(packed, b, b.n_events, "batched", dict(queue=0, extend_form=1))
    assert ei.value.status == lfm.LF_ERR_ARG
    tn.close()
