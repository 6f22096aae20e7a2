"""The oracle's boundary cases on the GPU, element by element.

The CPU pins fix the oracle at the method's boundaries: cuts that are strict
at exactly the threshold (chi2, Q, |t_y fit - t_y in|), the bending filter at
an unchanged slope, the zone of a track with t_y = 0, the magnet tolerance and
T_uv with negative slopes, a window model with a far reference plane, a
particle with a missing x layer.  Here the same crafted events go through both
launch forms of the library and must give the oracle's packed hits, windows,
triplets and outputs bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import pins
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


def _up(v):
    return float(np.nextafter(np.float32(v), np.float32(np.inf), dtype=np.float32))


def _cases():
    """(name, batch, params, geometry) of the boundary events."""
    orc = oracle.default()
    out = []
    # triplet chi2 exactly at T_triplet, and one step above
    st = pins._vertical_track()
    b = make_batch([dict(hits=[(0, 1, 100.0), (8, 1, 100.0), (4, 1, 101.25)], states=[st])])
    chi2 = float(np.float32(orc.run_batch(b)["trip_chi2"][0, 0]))
    out += [("chi2 == T_triplet", b, pins._params(T_triplet=chi2), None),
            ("chi2 < T_triplet", b, pins._params(T_triplet=_up(chi2)), None)]
    # Q exactly at T_Q
    hits, st, _, _ = pins.known_residual_event((1, 6))
    b = make_batch([dict(hits=hits, states=[st])])
    q = float(np.float32(orc.run_batch(b)["quality"][0]))
    out += [("Q == T_Q", b, pins._params(T_Q=q), None), ("Q < T_Q", b, pins._params(T_Q=_up(q)), None)]
    # |t_y fit - t_y in| exactly at T_ty
    tx, ty, p = 0.1, 0.1, 10.0
    xs, ys, txs, tys, qop = synth.state_of(tx, ty, 1.0 / p)
    b = make_batch([dict(hits=track_hits(tx, ty, 1.0 / p), states=[(xs, ys, txs, tys + 0.012, qop)])])
    r0 = orc.run_batch(b, params=pins._params(T_uv_min=1e4))
    d = float(np.abs(np.float32(r0["state"][0, 3]) - np.float32(tys + 0.012)))
    out += [("dty == T_ty", b, pins._params(T_ty=d, T_uv_min=1e4), None),
            ("dty < T_ty", b, pins._params(T_ty=_up(d), T_uv_min=1e4), None)]
    # a doublet with exactly the input slope, both charges, below p_bend
    g = synth.Geometry()
    z0, z1, z2 = (float(np.float32(g.z[l])) for l in (0, 4, 8))
    x0, txd = 10.0, 0.0625
    x2 = x0 + txd * (z2 - z0)
    x1 = x0 + txd * (z1 - z0) + 0.5
    x_mag = x0 + txd * (g.z_magnet - z0)
    for qop in (1.0 / 3.0, -1.0 / 3.0):
        st = (x_mag - txd * (g.z_magnet - g.z_state), 270.0, txd, 0.1, qop)
        b = make_batch([dict(hits=[(0, 1, x0), (8, 1, x2), (4, 1, x1)], states=[st])])
        out.append(("unchanged slope, q/p %+.3f" % qop, b, pins._params(xtol_c=5000.0, uv_tol=5000.0), None))
    # t_y = 0: hits in either zone
    hits = track_hits(0.05, 0.0, 0.1)
    st = synth.state_of(0.05, 0.0, 0.1)
    for zone in (1, 0):
        b = make_batch([dict(hits=[(l, zone, x) for (l, _, x) in hits], states=[st])])
        out.append(("t_y = 0, zone %d" % zone, b, None, None))
    # negative slopes: T_uv above its floor, a stereo hit just inside / outside
    for tx_, ty_ in ((-0.09, 0.06), (0.09, -0.06), (-0.09, -0.06)):
        t_uv = max(2.0, 50.0 * (abs(tx_) + abs(ty_)))
        for f in (1.0 - 1e-3, 1.0 + 1e-3):
            hits, st = pins._extension_track(tx_, ty_, offsets={5: f * np.sqrt(t_uv)})
            out.append(("T_uv, slopes %+.2f %+.2f, x %.3f" % (tx_, ty_, f), make_batch([dict(hits=hits, states=[st])]),
                        None, None))
    # extension cuts exactly at T_x and T_uv (a straight track at x = 100 mm, y = 0)
    qop = 0.05
    st = (100.0 + 1.2 * qop * 2500.0, 0.0, -1.2 * qop, 0.0, qop)
    for probe, layer, key, value in ((101.5, 3, "T_x", 2.25), (102.0, 5, "T_uv_min", 4.0)):
        b = make_batch([dict(hits=[(l, 1, probe if l == layer else 100.0) for l in range(11)], states=[st])])
        for thr in (value, _up(value)):
            par = pins._params(T_uv_scale=0.0, T_ty=1.0, T_Q=1e3)
            par.update({key: thr} if key == "T_uv_min" else dict(T_x=thr, T_uv_min=4.0))
            out.append(("%s at %.7g" % (key, thr), b, par, None))
    # the bending filter at p = p_bend exactly and one step above
    hits = track_hits(0.05, 0.1, 0.25)
    st = synth.state_of(0.05, 0.1, -0.2)
    b = make_batch([dict(hits=hits, states=[st])])
    for pb in (5.0, _up(5.0)):
        out.append(("p == p_bend %.7g" % pb, b, pins._params(p_bend=pb, xtol_c=5000.0, uv_tol=5000.0), None))
    # a missing x layer
    hits, st = pins._extension_track(-0.12, -0.06, 4.0, drop=(3,))
    out.append(("missing x layer", make_batch([dict(hits=hits, states=[st])]), None, None))
    # far reference plane (large curvature term), both polarities, noise-free events
    for pol in (1, -1):
        geo = synth.Geometry(polarity=pol, z_ref=6000.0)
        cfg = synth.EventConfig("far z_ref", 1, 31 + pol, ("fixed", 30), match_frac=1.0, extra=("none",),
                                noise=("per_layer", 20), sigma=0.05, efficiency=1.0, qop_smear=0.0)
        out.append(("z_ref 6000, polarity %+d" % pol, synth.generate(cfg, geometry=geo), None, geo_dict(geo)))
    return out


CASES = _cases()


@pytest.mark.parametrize("mode", ["plain", "batched"])
@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_boundary_case(lfm, case, mode):
    name, b, params, geo = CASES[case]
    tr = lfm.Tracker(geo, params)
    run_both(tr, b.to("cuda"), mode=mode, geometry=geo, params=params, stages=(mode == "plain"))
    tr.close()
