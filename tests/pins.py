"""Pins of the oracle to facts outside itself.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle disagrees with what the paper or the mathematics fixes.  The same
functions run against the committed oracle (they must pass) and against
copies with a planted mistake (at least one must fail).

What pins what:
  pack            numpy lexsort over (plane, x, raw index)           [library routine]
  closed form     noise-free particles from the exact trajectory model are
                  recovered with exactly their hits; the binary64 refit returns
                  the generating parameters to 1e-5                   [closed form]
  window edges    half widths x_tol = 150 + 2000/p, the 100 mm asymmetry side
                  and the 800 mm stereo tolerance (Sec. Defining the search
                  windows), hand-worked in tests/golden/window_examples.txt
  window cap      32 hits kept symmetrically around the centre, clamped at the
                  window ends
  closest tie     equal distances pick the lower packed index
  triplet chi2/K  chi2 of a hit placed at a known offset from the straight line;
                  K multiplies the intercept (Sec. Triplet Seeding)
  top-n           kept triplets are the smallest chi2 (prefix property)
  brute force     every (h0, h1, h2) of tiny events enumerated in numpy binary32
                  gives the oracle's triplet lists, order and chi2 bits
  bending filter  below 5 GeV the doublet must bend with the charge
  magnet tol      doublets inside/outside the 8..40 mm tolerance
  known-residual Q  Q of the paper's formula on residuals fixed by construction,
                  for n_hits = 9..12 (Table C_nhits, nDoF_x, nDoF_y)
  T_Q, T_ty       acceptance thresholds
  invariants      unique hits, >= 9 hits, >= 1 stereo hit per station, Q < T_Q,
                  hits inside windows, true hits inside pre-cap windows
  binary32 fit    the binary32 fit agrees with the binary64 refit
  strict cuts     the oracle's own chi2, Q and |dty| as thresholds are refused,
                  one binary32 step above accepted (reading R12); hits exactly
                  at sqrt(T_x) and sqrt(T_uv) from an exact straight model
                  likewise; the bending filter strictly below p_bend
  bending at 0    a doublet with exactly the input slope fails below p_bend
  zone at ty = 0  the upper zone
  window centre   x-layer centres equal the generator's true x with a far
                  reference plane (the curvature and dRatio terms of the model)
  missing x layer the x refit over five x hits stays exact
  selection       the lowest accepted Q wins, whatever the triplet rank
  compact         exclusive scan of per-event counts
  no-UT (Sec. No-UT tuning, Eq. tol_noUT, Eq. noUT_size_window, Table poly_tol):
    window edges  hand-worked x_tol of the polynomial at the assumed momentum,
                  the two one-sided windows with their 5 mm overlap and the
                  1200 mm u/v tolerance (tests/golden/no_ut_window_examples.txt)
    closed form   noise-free particles well above the assumed momentum are
                  recovered with exactly their hits from the window side of
                  their charge; q/p from the kick to 1e-5 in binary64
    overlap       a straight track seeds identical triplets on both sides,
                  ranked side 0 first
    magnet tol    the fixed 10 mm doublet tolerance at the magnet
    q/p unused    the input q/p does not change any result
"""
from __future__ import annotations

import os

import numpy as np
import torch

import oracle
from helpers import geo_dict, make_batch, raw_ids_in_windows, track_hits
from paper_2402_14670_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _params(**kw):
    p = oracle.default_params()
    p.update(kw)
    return p


def _rel_close(a, b, rtol, atol):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.all(np.abs(a - b) <= atol + rtol * np.abs(b))


# --------------------------------------------------------------------- pack

def pin_pack_lexsort(orc):
    b = synth.generate(1, n_events=4)
    x = b.x.numpy().copy()
    plane = b.plane.numpy()
    ro = b.raw_offsets.numpy()
    # plant exact duplicates and a negative zero inside buckets
    for e in range(4):
        s = ro[e]
        x[s + 1] = x[s]
        plane[s + 1] = plane[s]
        x[s + 3] = -0.0
        x[s + 4] = 0.0
        plane[s + 4] = plane[s + 3]
    pk = orc.pack(ro, x, b.z.numpy(), b.dxdy.numpy(), b.w.numpy(), plane)
    for e in range(4):
        idx = np.arange(ro[e], ro[e + 1])
        order = np.lexsort((idx, x[idx].astype(np.float64), plane[idx]))
        assert np.array_equal(pk["perm"][ro[e]:ro[e + 1]], idx[order]), "pack order"
        cnt = np.bincount(plane[idx], minlength=24)
        exp_off = ro[e] + np.concatenate([[0], np.cumsum(cnt)[:-1]])
        assert np.array_equal(pk["hit_offsets"][24 * e:24 * e + 24], exp_off), "bucket offsets"
    assert pk["hit_offsets"][-1] == ro[-1]
    assert np.array_equal(pk["x"], x[pk["perm"]])
    assert not np.any(np.signbit(pk["x"][pk["x"] == 0.0])), "negative zero kept"
    assert np.array_equal(pk["layer"], plane[pk["perm"]] % 12)


# --------------------------------------------------------------- closed form

def closed_form_batch(polarity=1, n_tracks=60, seed=11):
    geo = synth.Geometry(polarity=polarity)
    cfg = synth.EventConfig("closed form", 1, seed, ("fixed", n_tracks), match_frac=1.0,
                            extra=("none",), noise=("per_layer", 0), sigma=0.0, efficiency=1.0,
                            qop_smear=0.0)
    return geo, synth.generate(cfg, geometry=geo)


def pin_closed_form(orc, polarity=1):
    geo, b = closed_form_batch(polarity)
    res = orc.run_batch(b, geometry=geo_dict(geo), use_x64=True)
    perm = res["packed"]["perm"]
    hit_mcp = b.hit_mcp.numpy()[perm]
    layer = res["packed"]["layer"]
    trk_mcp = b.trk_mcp.numpy()
    mc = {k: v.numpy() for k, v in b.mcp.items()}
    n_checked = 0
    for t in range(b.n_tracks):
        m = trk_mcp[t]
        own = np.nonzero(hit_mcp == m)[0]
        lay = set(layer[own].tolist())
        uv_st = [any(l in lay for l in (4 * s + 1, 4 * s + 2)) for s in range(3)]
        trip_ok = {0, 4, 8} <= lay or {3, 7, 11} <= lay
        reco = len(own) >= 9 and all(uv_st) and trip_ok
        if not reco:
            continue
        n_checked += 1
        assert res["found"][t], "reconstructible track %d not found" % t
        got = res["hit_idx"][t]
        got = np.sort(got[got >= 0])
        assert np.array_equal(got, np.sort(own)), "track %d hit set" % t
        truth = synth.truth_params(mc["tx"][m], mc["ty"][m], mc["qop"][m], geo)
        st64 = res["state64"][t]
        # binary64 refit on binary64 hits: all five parameters and q/p to 1e-5
        for k, (rt, at) in enumerate([(1e-5, 1e-6), (1e-5, 1e-6), (1e-5, 1e-9), (1e-5, 1e-9),
                                      (1e-5, 1e-15), (1e-5, 1e-9)]):
            assert _rel_close(st64[k], truth[k], rt, at), ("state64", t, k, st64[k], truth[k])
        st = res["state"][t]
        # binary32 path: 1e-5 relative with absolute floors; c to a few ulp of x
        for k, (rt, at) in enumerate([(1e-5, 1e-3), (1e-5, 2e-2), (1e-5, 1e-6), (1e-5, 2e-5),
                                      (0.0, 5e-9), (1e-5, 1e-6)]):
            assert _rel_close(st[k], truth[k], rt, at), ("state", t, k, st[k], truth[k])
    assert n_checked >= 20
    # no noise: every found track is made of a single particle's hits (an input
    # state whose own particle left the acceptance may pick up a neighbour)
    for t in np.nonzero(res["found"])[0]:
        h = res["hit_idx"][t]
        assert len(set(hit_mcp[h[h >= 0]].tolist())) == 1


def pin_closed_form_md(orc):
    pin_closed_form(orc, polarity=-1)


def _qop_poly_params(polarity=1):
    from paper_2402_14670_gb300 import qop_fit
    c = qop_fit.fit_qop_poly(kappa=1.2)
    p = oracle.default_params()
    p.update(qop_poly=1, qop_c=c.tolist())
    return p


def pin_qop_polynomial(orc, polarity=1):
    """Sec. "Calculation of momentum and track states": with q/p from Eq.
    pt_kick and the field integral fitted on toy tracks (fourth order in
    dSlope, 2-D polynomials in the VELO slopes), noise-free particles of the
    exact trajectory model are found with exactly their hits and their q/p
    is the generating one to the fit's accuracy (0.3 % over 3-50 GeV on the
    fit grid; 0.5 % allowed); the binary64 refit agrees the same way."""
    geo, b = closed_form_batch(polarity)
    p = _qop_poly_params(polarity)
    res = orc.run_batch(b, geometry=geo_dict(geo), params=p, use_x64=True)
    lin = orc.run_batch(b, geometry=geo_dict(geo), use_x64=True)
    trk_mcp = b.trk_mcp.numpy()
    qop_true = b.mcp["qop"].numpy()
    f = res["found"].astype(bool)
    assert np.array_equal(f, lin["found"].astype(bool))
    assert np.array_equal(res["hit_idx"][f], lin["hit_idx"][f])
    assert np.array_equal(res["state"][f][:, :5], lin["state"][f][:, :5])   # only q/p changes
    # tracks made of their own particle's hits (an input state whose particle
    # left the acceptance may pick up a neighbour's)
    hit_mcp = b.hit_mcp.numpy()[res["packed"]["perm"]]
    own = np.array([f[t] and np.all(hit_mcp[res["hit_idx"][t][res["hit_idx"][t] >= 0]] == trk_mcp[t])
                    for t in range(b.n_tracks)])
    q = res["state"][own][:, 5].astype(np.float64)
    qt = qop_true[trk_mcp[own]]
    assert own.sum() >= 20
    assert np.all(np.abs(q / qt - 1.0) < 5e-3), np.max(np.abs(q / qt - 1.0))
    q64 = res["state64"][own][:, 5]
    assert np.all(np.abs(q64 / qt - 1.0) < 5e-3)
    # the polynomial form differs from the linear one (it is evaluated)
    assert np.any(res["state"][f][:, 5] != lin["state"][f][:, 5])


def pin_qop_polynomial_md(orc):
    pin_qop_polynomial(orc, polarity=-1)


# ------------------------------------------------------------------- windows

def _golden_windows():
    rows = []
    with open(os.path.join(GOLDEN, "window_examples.txt")) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            p, q, pol, xt, le, ri = ln.split()
            rows.append((float(p), int(q), int(pol), float(xt), float(le), float(ri)))
    return rows


def pin_window_edges(orc):
    tx, ty = 0.05, 0.1
    for (p, q, pol, x_tol, left, right) in _golden_windows():
        geo = synth.Geometry(polarity=pol)
        qop = q / p
        _, y, xm = synth.trajectory(tx, ty, qop, geo)
        hits, expect = [], {}
        for l in range(12):
            if l % 4 in (0, 3):
                lo, hi = xm[l] - (x_tol + left), xm[l] + (x_tol + right)
            else:
                lo, hi = xm[l] - 800.0, xm[l] + 800.0
            probes = [(lo - 0.5, False), (lo + 0.5, True), (hi - 0.5, True), (hi + 0.5, False)]
            expect[l] = []
            for xv, inside in probes:
                if inside:
                    expect[l].append(len(hits))
                hits.append((l, 1, float(xv)))
        b = make_batch([dict(hits=hits, states=[synth.state_of(tx, ty, qop, geo)])], geo)
        res = orc.run_batch(b, geometry=geo_dict(geo))
        got = raw_ids_in_windows(res, 0)
        for l in range(12):
            assert got[l] == sorted(expect[l]), ("window", p, q, pol, l, got[l], expect[l])


def pin_window_edges_inclusive(orc):
    """Reading R10 of Sec. "Defining the search windows": a window holds the
    hits with xmin <= x <= xmax, so a hit lying exactly on either edge is
    inside and the next binary32 value beyond the edge is outside.  The edges
    are the ones the oracle reports for the track (their values are pinned by
    pin_window_edges); the hits are placed on them bit for bit."""
    for (tx, ty, qop) in ((0.05, 0.1, 0.1), (-0.12, -0.07, -1.0 / 4.0)):
        st = synth.state_of(tx, ty, qop)
        zone = 1 if ty >= 0 else 0
        probe = orc.run_batch(make_batch([dict(hits=[(0, zone, 0.0)], states=[st])]))
        xmin = probe["win_xmin"][0].astype(np.float32)
        xmax = probe["win_xmax"][0].astype(np.float32)
        hits, expect = [], {}
        for l in range(12):
            lo, hi = np.float32(xmin[l]), np.float32(xmax[l])
            below = np.nextafter(lo, np.float32(-np.inf), dtype=np.float32)
            above = np.nextafter(hi, np.float32(np.inf), dtype=np.float32)
            expect[l] = [len(hits) + 1, len(hits) + 2]
            for xv in (below, lo, hi, above):
                hits.append((l, zone, float(xv)))
        res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]))
        got = raw_ids_in_windows(res, 0)
        assert np.array_equal(res["win_xmin"][0], probe["win_xmin"][0])
        for l in range(12):
            assert got[l] == expect[l], ("inclusive window edges", tx, ty, qop, l, got[l], expect[l])


def _extension_track(tx=0.05, ty=0.1, p=10.0, drop=(11,), offsets=None):
    """Noise-free hits of one particle without the layers in `drop` (layer 11
    dropped: configuration (3, 7, 11) cannot seed, so the only candidate is the
    triplet (0, 4, 8), extended into layers 3 and 7 and the six stereo layers)."""
    layers = [l for l in range(12) if l not in drop]
    hits = track_hits(tx, ty, 1.0 / p, layers=layers, offsets=offsets)
    return hits, synth.state_of(tx, ty, 1.0 / p)


def pin_extension_T_x(orc):
    """Sec. "Extending triplets to other layers": a hit in a missing x layer is
    added when (x_hit - x_expected)^2 < T_x, x_expected from the three-point
    solution through the triplet.  The particle's hits lie on the exact
    trajectory model, so x_expected is the true x up to binary32 rounding
    (~1e-4 mm); the layer-3 hit is moved by sqrt(T_x)*(1 -+ 1e-3) and must be
    kept just inside and dropped just outside (T_x = 2 mm^2)."""
    T_x = oracle.default_params()["T_x"]
    for sign in (1.0, -1.0):
        for f, kept in ((1.0 - 1e-3, True), (1.0 + 1e-3, False)):
            d = sign * f * np.sqrt(T_x)
            hits, st = _extension_track(offsets={3: d})
            res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]))
            assert res["found"][0], ("T_x", d)
            assert res["n_trip"][0] == 1 and res["trip"][0, 0, 0] == 0
            assert (res["hit_idx"][0, 3] >= 0) == kept, ("T_x acceptance", d, res["hit_idx"][0, 3])
            assert res["nhits"][0] == (11 if kept else 10)
            assert res["hit_idx"][0, 7] >= 0 and res["hit_idx"][0, 11] < 0


def pin_extension_T_uv(orc):
    """Sec. "Extending triplets to other layers" and Table tolerances: a stereo
    hit is added when its squared distance (measured coordinate) to the x model
    corrected by y_in * dxdy is below T_uv = max(T_uv_min, 50 (|t_x| + |t_y|)).
    The layer-5 hit of a noise-free particle is moved by sqrt(T_uv)(1 -+ 1e-3):
    kept just inside, dropped just outside; once with slopes that put T_uv on
    its floor (2 mm^2) and once above it."""
    p = oracle.default_params()
    for tx, ty in ((0.008, 0.006), (0.09, 0.06), (-0.09, 0.06), (0.09, -0.06), (-0.09, -0.06)):
        st = synth.state_of(tx, ty, 0.1)
        t_uv = np.float32(p["T_uv_scale"]) * (np.float32(abs(np.float32(st[2]))) +
                                              np.float32(abs(np.float32(st[3]))))
        t_uv = max(np.float32(p["T_uv_min"]), np.float32(t_uv))
        if abs(tx) < 0.05:
            assert t_uv == np.float32(p["T_uv_min"])
        else:
            assert t_uv > 2.5 * p["T_uv_min"]
        for sign in (1.0, -1.0):
            for f, kept in ((1.0 - 1e-3, True), (1.0 + 1e-3, False)):
                d = sign * f * float(np.sqrt(np.float64(t_uv)))
                hits, st = _extension_track(tx, ty, offsets={5: d})
                res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]))
                assert res["found"][0], ("T_uv", tx, d)
                assert (res["hit_idx"][0, 5] >= 0) == kept, ("T_uv acceptance", tx, d)
                assert res["nhits"][0] == (11 if kept else 10)
                assert res["hit_idx"][0, 6] >= 0


def pin_window_cap(orc):
    tx, ty, qop = 0.05, 0.1, 1.0 / 20.0
    _, y, xm = synth.trajectory(tx, ty, qop)
    c0 = float(xm[0])
    cases = [
        ([c0 + (k - 24.5) * 2.0 for k in range(50)], list(range(9, 41))),   # symmetric
        ([c0 + 1.0 + 2.0 * k for k in range(50)], list(range(0, 32))),     # all above the centre
        ([c0 - 1.0 - 2.0 * k for k in range(50)], list(range(18, 50))),    # all below (ids in x order)
        ([c0 + (k - 9.5) * 2.0 for k in range(50)], list(range(0, 32))),    # centre near the low edge
    ]
    for xs, exp_rank in cases:
        order = np.argsort(np.asarray(xs), kind="stable")
        hits = [(0, 1, x) for x in xs]
        b = make_batch([dict(hits=hits, states=[synth.state_of(tx, ty, qop)])])
        res = orc.run_batch(b)
        got = raw_ids_in_windows(res, 0)[0]
        exp = sorted(int(order[r]) for r in exp_rank)
        assert got == exp, ("cap", got, exp)


# ----------------------------------------------------------------- triplets

def _vertical_track():
    """p = 20 GeV, q = +1, MagUp, slope after the kick 0: x = 100 mm in the T stations."""
    qop = 0.05
    txs = -1.2 * qop
    return (100.0 - txs * 2500.0, 270.0, txs, 0.1, qop)


def pin_closest_tie(orc):
    st = _vertical_track()
    hits = [(0, 1, 100.0), (8, 1, 100.0), (4, 1, 100.5), (4, 1, 99.5)]
    res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]))
    perm = res["packed"]["perm"]
    assert res["n_trip"][0] >= 1
    cfg, h0, h1, h2 = res["trip"][0, 0]
    assert cfg == 0 and perm[h1] == 3, ("closest tie", perm[h1])
    assert abs(res["trip_chi2"][0, 0] - 0.25) < 1e-6


def pin_triplet_chi2_K(orc):
    st = _vertical_track()
    for d, kept in ((1.5, True), (2.9, False)):
        hits = [(0, 1, 100.0), (8, 1, 100.0), (4, 1, 100.0 + d)]
        res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]))
        assert (res["n_trip"][0] == 1) == kept, ("T_triplet", d)
        if kept:
            assert abs(res["trip_chi2"][0, 0] - d * d) < 1e-4
    # sloped doublet: K multiplies the intercept at z = 0 of the h0-h2 line
    qop = 0.05
    txs = 0.1 - 1.2 * qop
    st = (100.0 - txs * 2500.0, 270.0, txs, 0.1, qop)
    g = synth.Geometry()
    x0 = 100.0 + 0.1 * (g.z[0] - 5200.0)
    x2 = 100.0 + 0.1 * (g.z[8] - 5200.0)
    tx_d = (x2 - x0) / (g.z[8] - g.z[0])
    K = oracle.default_params(paper_K=True)["K_first"]
    x1_paper = g.z[4] * tx_d + (x0 - tx_d * g.z[0]) * K
    x1_line = x0 + tx_d * (g.z[4] - g.z[0])
    hits = [(0, 1, x0), (8, 1, x2), (4, 1, x1_paper)]
    b = make_batch([dict(hits=hits, states=[st])])
    rp = orc.run_batch(b, params=oracle.default_params(paper_K=True))
    r1 = orc.run_batch(b)
    assert rp["n_trip"][0] == 1 and rp["trip_chi2"][0, 0] < 1e-5, rp["trip_chi2"][0, 0]
    assert r1["n_trip"][0] == 1
    assert abs(r1["trip_chi2"][0, 0] - (x1_paper - x1_line) ** 2) < 2e-4 * max(1.0, (x1_paper - x1_line) ** 2)


def _key(row, chi2):
    cfg, h0, h1, h2 = row
    return (float(chi2), int(cfg), int(h0), int(h2))


def pin_top_n(orc):
    b = synth.generate(1, n_events=6)
    r12 = orc.run_batch(b, params=_params(n_triplets=12))
    r32 = orc.run_batch(b, params=_params(n_triplets=32))
    n_full = 0
    for t in range(b.n_tracks):
        n12, n32 = r12["n_trip"][t], r32["n_trip"][t]
        assert n12 == min(12, n32)
        k32 = [_key(r32["trip"][t, r], r32["trip_chi2"][t, r]) for r in range(n32)]
        k12 = [_key(r12["trip"][t, r], r12["trip_chi2"][t, r]) for r in range(n12)]
        assert k32 == sorted(k32), "triplets not ascending"
        assert k12 == k32[:n12], "kept triplets are not the smallest"
        n_full += n32 > 12
    assert n_full > 10


def pin_bending_filter(orc):
    tx, ty, p = 0.05, 0.1, 4.0
    hits = track_hits(tx, ty, 1.0 / p)
    wide = dict(xtol_c=5000.0, uv_tol=5000.0)   # windows that hold the hits whatever the charge
    p5 = float(1.0 / abs(np.float32(-0.2)))             # 5.0: 1/|q/p| of q/p = -0.2 in binary32
    assert np.float32(1.0) / np.abs(np.float32(-0.2)) == np.float32(5.0) == np.float32(p5)
    above = float(np.nextafter(np.float32(5.0), np.float32(np.inf), dtype=np.float32))
    # the filter applies strictly below p_bend: at p = p_bend exactly the
    # wrongly bending doublet is kept, one binary32 step above it refused
    for qop_in, p_bend, found in ((1.0 / p, 5.0, True), (-1.0 / p, 5.0, False), (-1.0 / p, 0.0, True),
                                  (-0.2, 5.0, True), (-0.2, above, False)):
        st = synth.state_of(tx, ty, qop_in)
        res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]), params=_params(p_bend=p_bend, **wide))
        assert bool(res["found"][0]) == found, ("bending filter", qop_in, p_bend)


def pin_magnet_tolerance(orc):
    # p = 20 GeV, slope 0.3 after the kick, x = 100 mm at the magnet centre;
    # then the mirror image (negative slope and charge: the tolerance grows
    # with |t_x^doublet|)
    p, T0 = 20.0, 0.3
    g = synth.Geometry()
    dz = g.z[8] - g.z[0]
    r = (g.z[0] - g.z_magnet) / dz          # x offset at the magnet per unit x2 offset
    # decoy h2 shifted by s: |dx_mag| = r*s against tol = 8 + 96/p + 10*(T0 + s/dz)
    s_star = (8.0 + 96.0 / p + 10.0 * T0) / (r - 10.0 / dz)
    for sg in (1.0, -1.0):
        qop = sg / p
        txs = sg * T0 - 1.2 * qop
        st = (sg * 100.0 - txs * 2500.0, 270.0, txs, 0.1, qop)
        line = lambda z: sg * (100.0 + T0 * (z - g.z_magnet))
        for s, inside in ((s_star - 0.05, True), (s_star + 0.05, False)):
            x1 = line(g.z[4]) + sg * s * (g.z[4] - g.z[0]) / dz
            hits = [(0, 1, line(g.z[0])), (8, 1, line(g.z[8])), (4, 1, line(g.z[4])),
                    (8, 1, line(g.z[8]) + sg * s), (4, 1, x1)]
            res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]))
            perm = res["packed"]["perm"]
            h2s = {int(perm[res["trip"][0, k, 3]]) for k in range(res["n_trip"][0])}
            assert 1 in h2s, "true doublet lost"
            assert (3 in h2s) == inside, ("magnet tolerance", sg, s, h2s)


# ------------------------------------------------------------------- quality

def _orth(v, cols):
    q, _ = np.linalg.qr(cols)
    return v - q @ (q.T @ v)


def known_residual_event(drop_uv=(), ax=0.35, ay=4.0, tx=0.1, ty=0.08, p=10.0, dty_in=0.0):
    """A track whose x hits are displaced orthogonally to the x model and whose
    stereo hits are displaced orthogonally (in y) to the y line, so the fits
    return the true parameters and every residual is known."""
    geo = synth.Geometry()
    qop = 1.0 / p
    _, y, xm = synth.trajectory(tx, ty, qop, geo)
    z = np.asarray(geo.z, np.float64)
    u = (z - geo.z_ref) * 1e-3
    f2 = u * u * (1.0 + geo.dratio * 1000.0 * u)
    xl = [l for l in range(12) if l % 4 in (0, 3)]
    uvl = [l for l in range(12) if l % 4 in (1, 2) and l not in drop_uv]
    rng = np.random.default_rng(7)
    dx = _orth(rng.standard_normal(len(xl)), np.stack([np.ones(len(xl)), u[xl], f2[xl]], 1))
    dx *= ax / np.linalg.norm(dx)
    dy = _orth(rng.standard_normal(len(uvl)), np.stack([np.ones(len(uvl)), u[uvl]], 1))
    dy *= ay / np.linalg.norm(dy)
    off = {l: dx[i] for i, l in enumerate(xl)}
    dxdy = np.asarray(geo.dxdy, np.float64)
    for i, l in enumerate(uvl):
        off[l] = -dy[i] * dxdy[l]
    hits = track_hits(tx, ty, qop, geo, layers=xl + uvl, offsets=off)
    T_uv = max(2.0, 50.0 * (abs(tx) + abs(ty)))
    n, n_uv = len(xl) + len(uvl), len(uvl)
    Qx = np.sum(dx ** 2) / 2.0 + np.sum((dy * dxdy[uvl]) ** 2) / T_uv
    Qy = np.sum(dy ** 2) / 800.0
    C = {9: 5.0, 10: 1.0, 11: 0.8, 12: 0.5}[n]
    Q = (Qx / (n - 3) + Qy / (n_uv - 2)) * C
    xs, ys, txs, tys, qo = synth.state_of(tx, ty, qop, geo)
    # an input t_y slightly off the truth moves the stereo search centre but
    # not the fits, so Q is unchanged
    return hits, (xs, ys, txs, tys + dty_in, qo), Q, n


def pin_known_residual_Q(orc):
    for drop, dty in (((), 0.0), ((1,), 0.0), ((1, 6), 0.0), ((1, 6, 9), 0.0), ((), 0.003)):
        hits, st, Q, n = known_residual_event(drop, dty_in=dty)
        res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]))
        assert res["found"][0] and res["nhits"][0] == n, ("known residual", drop, res["nhits"][0])
        assert abs(res["quality"][0] - Q) <= 5e-3 * Q, ("Q", drop, res["quality"][0], Q)


def pin_T_Q(orc):
    # nine hits (one stereo hit per station): Q = (Q_x/6 + Q_y/1) * 5; scale
    # the y residuals so that Q lands just below and just above T_Q = 0.5
    drop = (1, 6, 9)
    _, _, q0, _ = known_residual_event(drop, ax=0.2, ay=0.0)
    _, _, q1, _ = known_residual_event(drop, ax=0.2, ay=1.0)
    for target, acc in ((0.47, True), (0.53, False)):
        ay = np.sqrt((target - q0) / (q1 - q0))
        hits, st, Q, n = known_residual_event(drop, ax=0.2, ay=ay)
        assert abs(Q - target) < 1e-9
        res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]))
        assert bool(res["found"][0]) == acc, ("T_Q", Q)
        status = res["cand_status"][0, :res["n_trip"][0]]
        assert acc or np.any(status == 5), status


def pin_ty_cut(orc):
    tx, ty, p = 0.1, 0.1, 10.0
    hits = track_hits(tx, ty, 1.0 / p)
    for d, found in ((0.015, True), (-0.015, True), (0.025, False), (-0.025, False)):
        xs, ys, txs, tys, qop = synth.state_of(tx, ty, 1.0 / p)
        res = orc.run_batch(make_batch([dict(hits=hits, states=[(xs, ys, txs, tys + d, qop)])]),
                            params=_params(T_uv_min=1e4))
        assert bool(res["found"][0]) == found, ("T_ty", d)


# ------------------------------------------------------------ cut boundaries

def pin_cuts_strict(orc):
    """Reading R12: the method's cuts are strict (the paper prints "<").  The
    oracle's own chi2 of a triplet, Q of a candidate and |t_y fit - t_y in|
    of a track are set as the thresholds T_triplet, T_Q and T_ty: at exactly
    that value the triplet or track is refused, one binary32 step above it
    accepted."""
    up = lambda v: float(np.nextafter(np.float32(v), np.float32(np.inf), dtype=np.float32))
    st = _vertical_track()
    b = make_batch([dict(hits=[(0, 1, 100.0), (8, 1, 100.0), (4, 1, 101.25)], states=[st])])
    r0 = orc.run_batch(b)
    assert r0["n_trip"][0] == 1
    chi2 = float(np.float32(r0["trip_chi2"][0, 0]))
    assert chi2 > 1.0
    assert orc.run_batch(b, params=_params(T_triplet=chi2))["n_trip"][0] == 0, "chi2 == T_triplet kept"
    assert orc.run_batch(b, params=_params(T_triplet=up(chi2)))["n_trip"][0] == 1
    # Q against T_Q (ten hits with known residuals, Q about 0.1)
    hits, st, _, _ = known_residual_event((1, 6))
    b = make_batch([dict(hits=hits, states=[st])])
    r0 = orc.run_batch(b)
    assert r0["found"][0]
    q = float(np.float32(r0["quality"][0]))
    assert 0.0 < q < 0.5
    assert not orc.run_batch(b, params=_params(T_Q=q))["found"][0], "Q == T_Q accepted"
    assert orc.run_batch(b, params=_params(T_Q=up(q)))["found"][0]
    # |t_y fit - t_y in| against T_ty (input t_y 0.012 off the particle's)
    tx, ty, p = 0.1, 0.1, 10.0
    hits = track_hits(tx, ty, 1.0 / p)
    xs, ys, txs, tys, qop = synth.state_of(tx, ty, 1.0 / p)
    b = make_batch([dict(hits=hits, states=[(xs, ys, txs, tys + 0.012, qop)])])
    par = dict(T_uv_min=1e4)
    r0 = orc.run_batch(b, params=_params(**par))
    assert r0["found"][0]
    d = float(np.abs(np.float32(r0["state"][0, 3]) - np.float32(tys + 0.012)))
    assert 0.005 < d < 0.02
    assert not orc.run_batch(b, params=_params(T_ty=d, **par))["found"][0], "|dty| == T_ty accepted"
    assert orc.run_batch(b, params=_params(T_ty=up(d), **par))["found"][0]


def pin_extension_cuts_strict(orc):
    """Reading R12 for the extension cuts of Sec. "Extending triplets to
    other layers": a hit whose squared distance to the expectation equals T_x
    (missing x layer) or T_uv (stereo layer) is refused, one binary32 step of
    the threshold above it is accepted.  The particle is straight at
    x = 100 mm with y = 0 in the T stations (no layer 11, so only (0, 4, 8)
    seeds), so the three-point solution and the refit are x = 100 exactly and
    the probe hits at 101.5 and 102 mm sit at exactly 1.5 and 2 mm."""
    up = lambda v: float(np.nextafter(np.float32(v), np.float32(np.inf), dtype=np.float32))
    qop = 0.05
    txs = -1.2 * qop
    st = (100.0 - txs * 2500.0, 0.0, txs, 0.0, qop)
    loose = dict(T_ty=1.0, T_Q=1e3)
    for probe, layer, key, value in ((101.5, 3, "T_x", 2.25), (102.0, 5, "T_uv_min", 4.0)):
        hits = [(l, 1, probe if l == layer else 100.0) for l in range(11)]
        b = make_batch([dict(hits=hits, states=[st])])
        for thr, kept in ((value, False), (up(value), True)):
            par = _params(T_uv_scale=0.0, **loose)
            if key == "T_x":
                par.update(T_x=thr, T_uv_min=4.0)
            else:
                par.update(T_uv_min=thr)
            res = orc.run_batch(b, params=par)
            assert res["found"][0], (key, thr)
            assert (res["hit_idx"][0, layer] >= 0) == kept, ("extension cut at equality", key, thr)


def pin_bending_filter_zero(orc):
    """Reading R6 of Sec. "Triplet Seeding": below p_bend the doublet slope
    must move away from the input slope in the charge's bending direction; a
    doublet with exactly the input slope fails, for either charge.  Here
    (x2 - x0) / (z2 - z0) = 0.0625 exactly in binary32 and the input t_x is
    0.0625; the same doublet seeds once the filter is off (p_bend = 0)."""
    g = synth.Geometry()
    z0, z1, z2 = (float(np.float32(g.z[l])) for l in (0, 4, 8))
    txd = 0.0625
    x0 = 10.0
    x2 = x0 + txd * (z2 - z0)                         # 95.4375, exact
    assert np.float32(np.float32(x2 - x0) / np.float32(z2 - z0)) == np.float32(txd)
    x1 = x0 + txd * (z1 - z0) + 0.5                   # chi2 = 0.25
    x_mag = x0 + txd * (g.z_magnet - z0)              # the doublet's line at the magnet
    wide = dict(xtol_c=5000.0, uv_tol=5000.0)
    for qop in (1.0 / 3.0, -1.0 / 3.0):
        st = (x_mag - txd * (g.z_magnet - g.z_state), 270.0, txd, 0.1, qop)
        b = make_batch([dict(hits=[(0, 1, x0), (8, 1, x2), (4, 1, x1)], states=[st])])
        assert orc.run_batch(b, params=_params(**wide))["n_trip"][0] == 0, ("no bend accepted", qop)
        assert orc.run_batch(b, params=_params(p_bend=0.0, **wide))["n_trip"][0] == 1


def pin_zone_at_zero_ty(orc):
    """Reading R20 of Sec. "Defining the search windows": an input track with
    t_y = 0 exactly searches the upper zone (y >= 0)."""
    tx, p = 0.05, 10.0
    hits = track_hits(tx, 0.0, 1.0 / p)
    st = synth.state_of(tx, 0.0, 1.0 / p)
    assert st[3] == 0.0
    for zone, found in ((1, True), (0, False)):
        hz = [(l, zone, x) for (l, _, x) in hits]
        res = orc.run_batch(make_batch([dict(hits=hz, states=[st])]))
        assert bool(res["found"][0]) == found, ("zone at t_y = 0", zone)


def pin_window_centre_model(orc):
    """Sec. "Defining the search windows" with Eq. pt_kick and Eq.
    dratio_model_x_expected: an x layer's window centre is the track's x
    there, extrapolated to the magnet, kicked, and carried on the x(z) model
    (c dz^2 (1 + dRatio dz) around z_ref); for particles of the generator
    with exact q/p it is their true x.  With z_ref = 6000 mm the curvature
    term is 10 to 60 um at these momenta, far above the binary32 rounding of
    the centre (< 2 um at |x| < 4000 mm), so a dropped or wrong curvature or
    dRatio term is seen."""
    for pol in (1, -1):
        geo = synth.Geometry(polarity=pol, z_ref=6000.0)
        for tx, ty, qop in ((0.05, 0.1, 1.0 / 2.0), (-0.1, -0.05, -1.0 / 3.0), (0.2, 0.02, -1.0 / 1.5)):
            _, _, xm = synth.trajectory(tx, ty, qop, geo)
            st = synth.state_of(tx, ty, qop, geo)
            zone = 1 if ty >= 0 else 0
            res = orc.run_batch(make_batch([dict(hits=[(0, zone, 0.0)], states=[st])], geo),
                                geometry=geo_dict(geo))
            z = np.asarray(geo.z, np.float64)
            dz = z - geo.z_ref
            curv = np.abs(pol * geo.gamma * qop * dz * dz * (1.0 + geo.dratio * dz))
            for l in (0, 3, 4, 7, 8, 11):
                err = abs(float(res["win_centre"][0, l]) - float(np.ravel(xm)[l]))
                assert err < 2e-3, ("window centre", pol, tx, qop, l, err)
            assert curv[11] > 5e-3 and curv[11] * geo.dratio * dz[11] / (1.0 + geo.dratio * dz[11]) > 4e-3


def pin_closed_form_missing_x_layer(orc):
    """Closed form with a missing x layer: without its layer-3 hit a particle
    seeds only from (0, 4, 8), finds nothing in layer 3, and the x refit over
    the five x hits it has still returns the generating parameters (binary64
    refit to 1e-5; binary32 as in pin_closed_form)."""
    for tx, ty, p in ((0.05, 0.1, 10.0), (-0.12, -0.06, 4.0)):
        hits, st = _extension_track(tx, ty, p, drop=(3,))
        b = make_batch([dict(hits=hits, states=[st])])
        b.hit_x64 = None
        res = orc.run_batch(b)
        assert res["found"][0] and res["nhits"][0] == 11 and res["hit_idx"][0, 3] < 0, ("missing x layer", tx)
        truth = synth.truth_params(tx, ty, 1.0 / p)
        for k, (rt, at) in enumerate([(1e-5, 1e-3), (1e-5, 2e-2), (1e-5, 1e-6), (1e-5, 2e-5),
                                      (0.0, 5e-9), (1e-5, 1e-6)]):
            assert _rel_close(res["state"][0, k], truth[k], rt, at), ("state", tx, k, res["state"][0, k], truth[k])


def pin_selection_lowest_Q(orc):
    """Sec. "Quality Filter": the track keeps, of its accepted candidates, the
    one with the lowest Q (reading R18), whatever its triplet's rank.  On a
    minimum-bias sample the output Q of every found track is the smallest Q
    among its candidates that passed, and some tracks' lowest Q is not their
    first candidate (so the rule is exercised)."""
    b = synth.generate(1, n_events=25)
    res = orc.run_batch(b)
    n_not_first = 0
    for t in np.nonzero(res["found"])[0]:
        n = res["n_trip"][t]
        ok = res["cand_status"][t, :n] == 0
        q = res["cand_q"][t, :n]
        assert ok.any()
        qmin = np.min(q[ok])
        assert np.float32(res["quality"][t]) == np.float32(qmin), ("selected Q", t)
        first_ok = int(np.argmax(ok))
        n_not_first += bool(q[first_ok] > qmin)
    for t in np.nonzero(~res["found"].astype(bool))[0]:
        assert not np.any(res["cand_status"][t, :res["n_trip"][t]] == 0)
    assert n_not_first > 10


# --------------------------------------------------------------- brute force

def pin_triplets_brute_force(orc):
    """Brute force on tiny events (Sec. "Triplet Seeding"): for every input
    track, every (h0, h1, h2) of its windows in both configurations is
    enumerated in binary32 (numpy), each (h0, h2) takes the h1 of smallest
    |x1 - x1_expected| (ties to the lower index) if the doublet passes the
    bending and magnet filters, and the triplets with chi2 < T_triplet sorted
    by (chi2, configuration, h0, h2) and cut to n_triplets must be the
    oracle's list, order and chi2 bits included.  Windows are the oracle's
    (pinned separately); the paper's K constants make K != 1."""
    f = np.float32
    cfg_l = ((0, 4, 8), (3, 7, 11))
    for paper_K, nt in ((False, 12), (True, 5)):
        par = _params(n_hits_window=8, n_triplets=nt, **({} if not paper_K else
                      dict(K_first=oracle.default_params(paper_K=True)["K_first"],
                           K_last=oracle.default_params(paper_K=True)["K_last"])))
        cfg = synth.EventConfig("tiny", 6, 41, ("fixed", 12), match_frac=0.8, extra=("none",),
                                noise=("per_layer", 30), p_min=2.0)
        b = synth.generate(cfg)
        res = orc.run_batch(b, params=par)
        pk = res["packed"]
        x, z = pk["x"].astype(np.float32), pk["z"].astype(np.float32)
        g = synth.Geometry()
        st = np.stack([b.sx.numpy(), b.sy.numpy(), b.stx.numpy(), b.sty.numpy(), b.sqop.numpy()], 1).astype(np.float32)
        n_checked = 0
        for t in range(b.n_tracks):
            xs, ys, txs, tys, qop = (f(v) for v in st[t])
            x_mag_in = xs + txs * (f(g.z_magnet) - f(g.z_state))
            pmom = f(1.0) / abs(qop)
            pol = f(g.polarity)
            bend = pol if qop > f(0.0) else -pol
            tol_base = f(par["magtol_min"]) + f(par["magtol_c"]) / pmom
            found = []
            for c, (L0, L1, L2) in enumerate(cfg_l):
                K = f(par["K_first"] if c == 0 else par["K_last"])
                z1 = f(g.z[L1])
                w = lambda l: range(int(res["win_begin"][t, l]), int(res["win_begin"][t, l] + res["win_count"][t, l]))
                for h0 in w(L0):
                    for h2 in w(L2):
                        tx_d = (x[h2] - x[h0]) / (z[h2] - z[h0])
                        if pmom < f(par["p_bend"]):
                            d = tx_d - txs
                            if not ((d > f(0.0)) if bend > f(0.0) else (d < f(0.0))):
                                continue
                        x_mag_d = x[h0] + tx_d * (f(g.z_magnet) - z[h0])
                        tol = tol_base + f(par["magtol_tx"]) * abs(tx_d)
                        tol = min(max(tol, f(par["magtol_min"])), f(par["magtol_max"]))
                        if not (abs(x_mag_d - x_mag_in) < tol):
                            continue
                        x1e = z1 * tx_d + (x[h0] - tx_d * z[h0]) * K
                        h1s = list(w(L1))
                        if not h1s:
                            continue
                        dist = [abs(x[h] - x1e) for h in h1s]
                        h1 = h1s[int(np.argmin(dist))]          # first of the smallest
                        dx = x[h1] - x1e
                        chi2 = dx * dx
                        if chi2 < f(par["T_triplet"]):
                            found.append((chi2, c, h0, h2, h1))
            found.sort(key=lambda v: (v[0], v[1], v[2], v[3]))
            found = found[:nt]
            n = int(res["n_trip"][t])
            assert n == len(found), ("brute force count", t, n, len(found))
            for r, (chi2, c, h0, h2, h1) in enumerate(found):
                assert tuple(res["trip"][t, r]) == (c, h0, h1, h2), ("brute force triplet", t, r)
                assert np.float32(res["trip_chi2"][t, r]).view(np.uint32) == np.float32(chi2).view(np.uint32)
            n_checked += n
        assert n_checked > 50, n_checked


# ---------------------------------------------------------------- invariants

def pin_invariants(orc):
    b = synth.generate(1, n_events=25)
    res = orc.run_batch(b)
    layer = res["packed"]["layer"]
    ho = res["packed"]["hit_offsets"]
    to = b.trk_offsets.numpy()
    ev_of = np.repeat(np.arange(b.n_events), np.diff(to))
    nf = 0
    for t in np.nonzero(res["found"])[0]:
        nf += 1
        h = res["hit_idx"][t]
        used = h[h >= 0]
        assert len(set(used.tolist())) == len(used)
        assert res["nhits"][t] == len(used) >= 9
        zone = 1 if b.sty[t] >= 0 else 0
        for l in range(12):
            if h[l] < 0:
                continue
            assert layer[h[l]] == l
            bk = 24 * ev_of[t] + 12 * zone + l
            assert ho[bk] <= h[l] < ho[bk + 1], "hit outside the track's zone bucket"
            wb, wc = res["win_begin"][t, l], res["win_count"][t, l]
            assert wb <= h[l] < wb + wc, "hit outside its window"
        for s in range(3):
            assert h[4 * s + 1] >= 0 or h[4 * s + 2] >= 0, "no stereo hit in a station"
        assert all(h[l] >= 0 for l in (0, 4, 8)) or all(h[l] >= 0 for l in (3, 7, 11))
        assert res["quality"][t] < 0.5
        assert np.all(np.isfinite(res["state"][t]))
        assert np.all(res["win_count"][t] <= 32)
    assert nf > 500


def pin_true_hits_in_window(orc):
    b = synth.generate(1, n_events=10, qop_smear=0.0)
    res = orc.run_batch(b)
    perm = res["packed"]["perm"]
    hit_mcp = b.hit_mcp.numpy()[perm]
    layer = res["packed"]["layer"]
    x = res["packed"]["x"]
    trk_mcp = b.trk_mcp.numpy()
    n = 0
    for t in range(b.n_tracks):
        m = trk_mcp[t]
        if m < 0:
            continue
        for h in np.nonzero(hit_mcp == m)[0]:
            l = layer[h]
            assert res["win_xmin"][t, l] <= x[h] <= res["win_xmax"][t, l], ("true hit outside", t, l)
            n += 1
    assert n > 1000


def pin_fit32_vs_fit64(orc):
    b = synth.generate(1, n_events=10)
    res = orc.run_batch(b)
    f = res["found"].astype(bool)
    st, s64 = res["state"][f].astype(np.float64), res["state64"][f]
    tol = [(1e-6, 2e-3), (1e-5, 0.2), (1e-5, 2e-6), (1e-4, 5e-5), (0.0, 2e-8), (1e-5, 2e-6)]
    for k, (rt, at) in enumerate(tol):
        assert _rel_close(st[:, k], s64[:, k], rt, at), ("fit32 vs fit64", k, np.max(np.abs(st[:, k] - s64[:, k])))


def pin_compact(orc):
    b = synth.generate(1, n_events=8)
    res = orc.run_batch(b)
    to = b.trk_offsets.numpy()
    found = res["found"].astype(np.int64)
    cnt = np.array([found[to[e]:to[e + 1]].sum() for e in range(b.n_events)])
    assert np.array_equal(res["out_offsets"], np.concatenate([[0], np.cumsum(cnt)]))
    assert np.array_equal(res["out_trk"], np.nonzero(found)[0])


# ------------------------------------------------------------------- no-UT

def _no_ut(**kw):
    p = oracle.no_ut_params()
    p.update(kw)
    return p


def _golden_no_ut_windows(name="no_ut_window_examples.txt"):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                rows.append(tuple(float(v) for v in ln.split()))
    return rows


def _side_ids(res, t, side):
    """layer -> sorted raw ids inside window set `side` of track t."""
    perm = res["packed"]["perm"]
    out = {}
    for l in range(12):
        b = int(res["win_begin"][t, side * 12 + l])
        c = int(res["win_count"][t, side * 12 + l])
        out[l] = sorted(int(perm[i]) for i in range(b, b + c))
    return out


def pin_no_ut_window_edges(orc, golden="no_ut_window_examples.txt", **params):
    g = synth.Geometry()
    xs, ys = 37.0, -21.0
    for (tx, ty, _p, x_tol) in _golden_no_ut_windows(golden):
        zone = 1 if ty >= 0 else 0
        hits, inside = [], {0: {}, 1: {}}
        for l in range(12):
            x_line = xs + tx * (g.z[l] - g.z_state)
            if l % 4 in (0, 3):
                c, tol = x_line, x_tol
            else:
                y = ys + ty * (g.z[l] - g.z_state)
                c, tol = x_line - y * g.dxdy[l], 1200.0
            lo0, hi0 = c - tol, c + 5.0      # side 0
            lo1, hi1 = c - 5.0, c + tol      # side 1
            e = 0.1  # far above the rounding of x_tol (ulp ~ 1e-4 mm), below each term checked
            probes = [lo0 - e, lo0 + e, hi0 - e, hi0 + e, lo1 - e, lo1 + e, hi1 - e, hi1 + e]
            inside[0][l], inside[1][l] = [], []
            for xv in probes:
                for sd, (lo, hi) in enumerate(((lo0, hi0), (lo1, hi1))):
                    if lo <= xv <= hi:
                        inside[sd][l].append(len(hits))
                hits.append((l, zone, float(xv)))
        # the input q/p is not used by the variant: give it a nonsense value
        st = (xs, ys, tx, ty, 0.7)
        b = make_batch([dict(hits=hits, states=[st])], g)
        res = orc.run_batch(b, params=_no_ut(**params))
        for sd in (0, 1):
            got = _side_ids(res, 0, sd)
            for l in range(12):
                assert got[l] == sorted(inside[sd][l]), ("no-UT window", tx, ty, sd, l, got[l], inside[sd][l])


def pin_no_ut_pt_min(orc):
    """Eq. tol_noUT at an assumed momentum set by the pT threshold: with
    pT_min = 1.5 GeV the hand-worked windows of
    tests/golden/no_ut_window_examples_ptmin.txt (the default pT_min of 1 GeV
    cannot tell pT_min / sin(theta) from sin(theta) * pT_min)."""
    pin_no_ut_window_edges(orc, golden="no_ut_window_examples_ptmin.txt", pt_min=1.5)


def pin_no_ut_closed_form(orc, polarity=1):
    geo, b = closed_form_batch(polarity, seed=23)
    res = orc.run_batch(b, geometry=geo_dict(geo), params=_no_ut(), use_x64=True)
    perm = res["packed"]["perm"]
    hit_mcp = b.hit_mcp.numpy()[perm]
    layer = res["packed"]["layer"]
    trk_mcp = b.trk_mcp.numpy()
    mc = {k: v.numpy() for k, v in b.mcp.items()}
    n_checked = 0
    for t in range(b.n_tracks):
        m = trk_mcp[t]
        own = np.nonzero(hit_mcp == m)[0]
        lay = set(layer[own].tolist())
        reco = (len(own) >= 9 and all(any(l in lay for l in (4 * s + 1, 4 * s + 2)) for s in range(3))
                and ({0, 4, 8} <= lay or {3, 7, 11} <= lay))
        # the windows hold the particle when its momentum is well above the
        # assumed one (the tighter of 5 GeV and pT = 1 GeV at its polar angle)
        tx, ty = mc["tx"][m], mc["ty"][m]
        sin_t = np.sqrt(tx * tx + ty * ty) / np.sqrt(1.0 + tx * tx + ty * ty)
        if not reco or abs(1.0 / mc["qop"][m]) < 1.25 * max(5.0, 1.0 / sin_t):
            continue
        n_checked += 1
        assert res["found"][t], "no-UT: reconstructible track %d not found" % t
        got = res["hit_idx"][t]
        assert np.array_equal(np.sort(got[got >= 0]), np.sort(own)), "no-UT hit set %d" % t
        # the winning candidate was seeded on the side its charge bends to
        acc = [r for r in range(res["n_trip"][t]) if res["cand_status"][t, r] == 0]
        best = min(acc, key=lambda r: (res["cand_q"][t, r], r))
        side = int(res["trip"][t, best, 0]) // 2
        assert side == (1 if polarity * mc["qop"][m] > 0 else 0), ("no-UT side", t, side)
        truth = synth.truth_params(mc["tx"][m], mc["ty"][m], mc["qop"][m], geo)
        assert _rel_close(res["state64"][t][5], truth[5], 1e-5, 1e-9), ("no-UT q/p", t)
        assert _rel_close(res["state"][t][5], truth[5], 1e-5, 1e-6), ("no-UT q/p f32", t)
    assert n_checked >= 15, n_checked


def pin_no_ut_closed_form_md(orc):
    pin_no_ut_closed_form(orc, polarity=-1)


def pin_no_ut_overlap(orc):
    """Hits inside the 5 mm overlap serve both charge assumptions.  A track
    with x = 100 mm in every x layer and a straight input line through it
    gives chi2 = 0 exactly in both configurations and on both sides, so the
    ranking (chi2, side, configuration) alone orders the four triplets.  A
    p = 5 TeV particle (bend under a millimetre) is found."""
    hits = [(l, 1, 100.0) for l in (0, 3, 4, 7, 8, 11)]
    st = (100.0, 270.0, 0.0, 0.07, 0.0)
    res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]), params=_no_ut())
    n = res["n_trip"][0]
    assert n == 4, n
    assert list(res["trip"][0, :n, 0]) == [0, 1, 2, 3], res["trip"][0, :n, 0]   # cfg + 2*side
    assert np.all(res["trip_chi2"][0, :n] == 0.0)
    assert np.array_equal(res["trip"][0, 0, 1:], res["trip"][0, 2, 1:])
    r1 = orc.run_batch(make_batch([dict(hits=hits, states=[st])]), params=_no_ut(n_triplets=1))
    assert r1["n_trip"][0] == 1 and r1["trip"][0, 0, 0] == 0
    tx, ty, qop = 0.04, 0.07, 1.0 / 5000.0
    b = make_batch([dict(hits=track_hits(tx, ty, qop), states=[synth.state_of(tx, ty, qop)])])
    res = orc.run_batch(b, params=_no_ut())
    assert res["found"][0] and res["nhits"][0] == 12
    assert set((res["trip"][0, :res["n_trip"][0], 0] // 2).tolist()) == {0, 1}


def pin_no_ut_magnet_tolerance(orc):
    # straight input line with x = 100 mm at the magnet centre, T-station slope
    # 0.1 (a 200 mm bend at T3, inside the side-1 windows)
    T0 = 0.1
    g = synth.Geometry()
    txs = 0.05
    st = (100.0 + txs * (g.z_state - g.z_magnet), 270.0, txs, 0.1, 0.0)
    line = lambda z: 100.0 + T0 * (z - g.z_magnet)
    dz = g.z[8] - g.z[0]
    r = (g.z[0] - g.z_magnet) / dz          # x offset at the magnet per unit x2 offset
    s_star = 10.0 / r                       # a fixed 10 mm, whatever p and slope
    for s, inside in ((s_star - 0.05, True), (s_star + 0.05, False)):
        x1 = line(g.z[4]) + s * (g.z[4] - g.z[0]) / dz
        hits = [(0, 1, line(g.z[0])), (8, 1, line(g.z[8])), (4, 1, line(g.z[4])),
                (8, 1, line(g.z[8]) + s), (4, 1, x1)]
        res = orc.run_batch(make_batch([dict(hits=hits, states=[st])]), params=_no_ut())
        perm = res["packed"]["perm"]
        h2s = {int(perm[res["trip"][0, k, 3]]) for k in range(res["n_trip"][0])}
        assert 1 in h2s, "no-UT: true doublet lost"
        assert (3 in h2s) == inside, ("no-UT magnet tolerance", s, h2s)


def pin_no_ut_qop_unused(orc):
    b = synth.generate(1, n_events=3)
    r0 = orc.run_batch(b, params=_no_ut())
    gen = np.random.default_rng(5)
    b.sqop = b.sqop.clone()
    b.sqop[:] = torch.as_tensor(gen.uniform(-1.0, 1.0, b.n_tracks).astype(np.float32))
    r1 = orc.run_batch(b, params=_no_ut())
    for k in ("found", "hit_idx", "state", "quality", "win_begin", "win_count", "n_trip", "trip"):
        assert np.array_equal(r0[k], r1[k]), k
    assert r0["found"].sum() > 10


ALL_PINS = [pin_pack_lexsort, pin_closed_form, pin_closed_form_md, pin_qop_polynomial, pin_qop_polynomial_md,
            pin_window_edges,
            pin_window_edges_inclusive, pin_extension_T_x, pin_extension_T_uv, pin_window_cap,
            pin_closest_tie, pin_triplet_chi2_K, pin_top_n, pin_bending_filter,
            pin_magnet_tolerance, pin_known_residual_Q, pin_T_Q, pin_ty_cut, pin_invariants,
            pin_true_hits_in_window, pin_fit32_vs_fit64, pin_compact,
            pin_no_ut_window_edges, pin_no_ut_closed_form, pin_no_ut_closed_form_md, pin_no_ut_overlap,
            pin_no_ut_magnet_tolerance, pin_no_ut_qop_unused,
            pin_cuts_strict, pin_bending_filter_zero, pin_zone_at_zero_ty, pin_window_centre_model,
            pin_closed_form_missing_x_layer, pin_selection_lowest_Q, pin_no_ut_pt_min,
            pin_extension_cuts_strict, pin_triplets_brute_force]
