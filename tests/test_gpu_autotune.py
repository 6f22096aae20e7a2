"""The launch-shape autotuner on the GPU: it times every candidate on a
batch, keeps the fastest per batch bucket, and the chosen shape gives the
oracle's results (every candidate computes the same thing)."""
import numpy as np
import pytest
import torch

import oracle
from parity import compare_outputs
from paper_2402_14670_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_14670_gb300 import build
    build.build()
    from paper_2402_14670_gb300 import autotune, lf
    return lf, autotune


def test_tune_picks_a_candidate_and_keeps_results(mods, tmp_path):
    lf, autotune = mods
    b = synth.generate(2, n_events=300).to("cuda")
    tr = lf.Tracker()
    packed = tr.pack(b)
    tuner = autotune.Autotuner(cache_path=str(tmp_path / "tune.json"), reps=2)
    choice = tuner.tune(tr, packed, b, b.n_events)
    assert choice in autotune.CANDIDATES
    key = tuner._key(autotune.bucket_of(b.n_events, b.n_tracks))
    assert len(tuner.timings[key]) == len(autotune.CANDIDATES)
    assert all(v > 0 for v in tuner.timings[key].values())
    # the table persists and is looked up by bucket
    again = autotune.Autotuner(cache_path=str(tmp_path / "tune.json"))
    assert again.lookup(b.n_events, b.n_tracks) == choice
    assert tuner.choose(tr, packed, b, b.n_events) == choice
    out = tr.find(packed, b, b.n_events, "batched", choice)
    torch.cuda.synchronize()
    assert tr.status() == 0
    compare_outputs(out, oracle.run_batch(b, dumps=False))
    tr.close()
