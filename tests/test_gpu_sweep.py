"""The window-cap and tolerance sweep (Sec. "Performance": the n_hits^window
scan) on the GPU: every setting's result equals the oracle's with the same
parameters, and its truth score is a proper efficiency and fake rate."""
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
    from paper_2402_14670_gb300 import lf, sweep
    return lf, sweep


@pytest.mark.parametrize("cap,scale", [(8, 1.0), (16, 1.0), (32, 1.0), (64, 1.0), (32, 0.5), (32, 1.5)])
def test_sweep_setting_matches_oracle(mods, cap, scale):
    lf, sweep = mods
    batch = synth.generate(1, n_events=60, device="cuda", truth=True)
    p = lf.default_params()
    p.update(n_hits_window=cap, xtol_c=p["xtol_c"] * scale, xtol_p=p["xtol_p"] * scale)
    tr = lf.Tracker(None, p)
    packed, out = tr.run(batch)
    torch.cuda.synchronize()
    assert tr.status() == 0
    res = oracle.run_batch(batch, params=p, dumps=False)
    compare_outputs(out, res)
    s = sweep.score(batch, packed, out)
    assert s["reconstructible"] > 1000
    assert 0.0 < s["efficiency"] <= 1.0 and 0.0 <= s["fake_rate"] < 1.0
    r = sweep.run_setting(batch, p, reps=2)
    assert r["efficiency"] == s["efficiency"] and r["ms"] > 0.0
    tr.close()


def test_sweep_efficiency_grows_with_the_cap(mods):
    """A window that keeps more hits cannot lose the true hit more often:
    on the same events the efficiency at cap 64 is at least that at cap 8."""
    lf, sweep = mods
    batch = synth.generate(1, n_events=100, device="cuda", truth=True)
    eff = {}
    for cap in (8, 64):
        p = lf.default_params()
        p["n_hits_window"] = cap
        eff[cap] = sweep.run_setting(batch, p, reps=1)["efficiency"]
    assert eff[64] >= eff[8]
