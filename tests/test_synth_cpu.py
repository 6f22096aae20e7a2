"""Self-checks of the seeded event generator (CPU).

The generator is the detector simulation that feeds both the oracle and the
library (it holds none of the method's arithmetic).  Checked here: noise-free
particle hits lie on the trajectory model (a straight line to the magnet,
the pT kick, then x(z) = x_ref + t_x dz + c dz^2 (1 + dRatio dz) about z_ref
and y linear), a hit's zone is the sign of its y, a stereo layer records
x - y dxdy, noise hits come in the configured numbers and are unmatched, and
a configuration with its seed reproduces its batch exactly.
"""
import numpy as np
import torch

from paper_2402_14670_gb300 import synth


def _noise_free(n_tracks=30, seed=77):
    cfg = synth.EventConfig("self-check", 1, seed, ("fixed", n_tracks), match_frac=1.0, extra=("none",),
                            noise=("per_layer", 0), sigma=0.0, efficiency=1.0, qop_smear=0.0)
    return synth.generate(cfg)


def test_hits_on_the_trajectory_model():
    geo = synth.Geometry()
    b = _noise_free()
    mcp = {k: v.numpy() for k, v in b.mcp.items()}
    hm = b.hit_mcp.numpy()
    plane = b.plane.numpy().astype(np.int64)
    layer, zone = plane % 12, plane // 12
    x64 = b.hit_x64.numpy()
    z = np.asarray(geo.z, np.float64)
    dxdy = np.asarray(geo.dxdy, np.float64)
    n = 0
    for m in np.unique(hm[hm >= 0]):
        tx, ty, qop = mcp["tx"][m], mcp["ty"][m], mcp["qop"][m]
        # the model, from its definition: straight from the origin to the
        # magnet plane, kicked, then the x(z) polynomial about z_ref
        txf = tx + geo.polarity * geo.kappa * qop
        c = geo.polarity * geo.gamma * qop
        dz = z - geo.z_ref
        x_ref = tx * geo.z_magnet + txf * (geo.z_ref - geo.z_magnet)
        x = x_ref + txf * dz + c * dz * dz * (1.0 + geo.dratio * dz)
        y = ty * z
        for h in np.nonzero(hm == m)[0]:
            l = layer[h]
            assert zone[h] == (1 if y[l] >= 0 else 0)
            assert abs(x64[h] - (x[l] - y[l] * dxdy[l])) < 1e-9 * max(1.0, abs(x[l]))
            assert b.x[h].item() == np.float32(x64[h])      # sigma = 0: the binary32 copy of the truth
            n += 1
    assert n > 200


def test_noise_counts_and_truth_labels():
    cfg = synth.CONFIGS[0]
    b = synth.generate(0)
    hm = b.hit_mcp.numpy()
    layer = b.plane.numpy().astype(np.int64) % 12
    per = cfg.noise[1]
    for l in range(12):
        assert np.sum((hm < 0) & (layer == l)) == per
    assert np.all(np.abs(b.x.numpy()[hm < 0]) <= cfg.x_acc)
    # every input state of a particle names it; the others name none
    tm = b.trk_mcp.numpy()
    assert np.all((tm >= -1) & (tm < len(b.mcp["qop"])))


def test_seeded_batches_reproduce():
    a = synth.generate(1, n_events=40)
    b = synth.generate(1, n_events=40)
    for f in ("raw_offsets", "x", "z", "dxdy", "w", "plane", "trk_offsets", "sx", "sy", "stx", "sty", "sqop"):
        assert torch.equal(getattr(a, f), getattr(b, f)), f
    c = synth.generate(synth.EventConfig(**{**synth.CONFIGS[1].__dict__, "seed": 99}), n_events=40)
    assert not torch.equal(a.x[:100], c.x[:100])
