"""The truth scoring of the window-cap sweep (host logic, no GPU).

Scored outputs: the oracle's own result, an output built from the truth (every
input track given exactly its particle's hits: efficiency 1, no fakes), and
that output with one track's hits swapped for another particle's (one fake).
"""
import numpy as np
import pytest

import oracle
from paper_2402_14670_gb300 import synth, sweep


@pytest.fixture(scope="module")
def minbias():
    batch = synth.generate(1, n_events=4, device="cpu", truth=True)
    res = oracle.run_batch(batch, dumps=False)
    return batch, res


def _truth_output(batch, perm):
    hit_mcp = batch.hit_mcp.numpy()
    trk_mcp = batch.trk_mcp.numpy()
    layer = batch.plane.numpy() % 12
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size, dtype=perm.dtype)
    hit_idx = np.full((trk_mcp.size, 12), -1, np.int32)
    for t, m in enumerate(trk_mcp):
        if m < 0:
            continue
        for r in np.nonzero(hit_mcp == m)[0]:
            hit_idx[t, layer[r]] = inv[r]
    return dict(found=trk_mcp >= 0, hit_idx=hit_idx)


def test_oracle_result_scores_in_range(minbias):
    batch, res = minbias
    s = sweep.score(batch, res["packed"], res)
    assert s["reconstructible"] > 0
    assert 0.5 < s["efficiency"] <= 1.0
    assert 0.0 <= s["fake_rate"] < 0.5
    assert s["found"] == int(res["found"].sum())


def test_truth_output_is_perfect(minbias):
    batch, res = minbias
    perm = res["packed"]["perm"]
    out = _truth_output(batch, perm)
    s = sweep.score(batch, res["packed"], out)
    assert s["efficiency"] == 1.0
    assert s["fake_rate"] == 0.0


def test_swapped_hits_make_one_fake(minbias):
    batch, res = minbias
    perm = res["packed"]["perm"]
    out = _truth_output(batch, perm)
    trk_mcp = batch.trk_mcp.numpy()
    reco = sweep.reconstructible(batch, batch.plane.numpy() % 12)
    a, b = np.nonzero(reco)[0][:2]
    assert trk_mcp[a] != trk_mcp[b]
    out["hit_idx"][a] = out["hit_idx"][b]
    s = sweep.score(batch, res["packed"], out)
    n_found = int(out["found"].sum())
    assert s["fake_rate"] == pytest.approx(1.0 / n_found)
    assert s["efficiency"] == pytest.approx(1.0 - 1.0 / int(reco.sum()))


def test_reconstructible_needs_a_triplet_configuration():
    """A particle with 11 hits but no hit on layer 4 or layer 7 has neither
    seeding configuration (0,4,8) nor (3,7,11)."""
    batch = synth.generate(1, n_events=1, device="cpu", truth=True)
    layer = (batch.plane.numpy() % 12).copy()
    hit_mcp = batch.hit_mcp.numpy()
    reco = sweep.reconstructible(batch, layer)
    t = int(np.nonzero(reco)[0][0])
    m = batch.trk_mcp.numpy()[t]
    for lost in (4, 7):
        layer[(hit_mcp == m) & (layer == lost)] = 5  # moved onto a stereo layer
    assert not sweep.reconstructible(batch, layer)[t]
