"""The margin of the half-precision triplet pre-filter, checked on the CPU.

The pre-filter (lf_tuning.triplet_prefilter) keeps a pair of hits (h0, h2)
when some hit of its h1 window lies within sqrt(T_triplet) + PF_MARGIN of
x1_expected, with the distances taken in binary16 relative to the window's
first hit and x1_expected formed with the slope as a product by 1/(z2 - z0).
It is exact (no pair the binary32 path accepts is dropped) if PF_MARGIN
bounds the difference between that binary16 distance and the binary32
distance |x1 - x1_expected| of Sec. "Triplet Seeding", for windows spanning
at most PF_SPAN mm.  Here both are evaluated with numpy's binary32 and
binary16 arithmetic (correctly rounded, as on the GPU) on random and
adversarial hits, and the largest difference must stay below the margin
while the binary16 roundings really do reach about 1 mm (so a margin much
below 1 mm would drop pairs).
"""
import numpy as np

PF_SPAN = 2000.0
PF_MARGIN = 1.1          # csrc/lf_internal.h
Z = (7826.0, 8508.0, 9193.0, 8036.0, 8718.0, 9403.0)   # z of layers 0, 4, 8 and 3, 7, 11


def _lf_header_constants():
    import os
    import re
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2402_14670_gb300", "csrc",
                            "lf_internal.h")).read()
    span = float(re.search(r"PF_SPAN = ([0-9.]+)f", src).group(1))
    margin = float(re.search(r"PF_MARGIN = ([0-9.]+)f", src).group(1))
    return span, margin


def _distances(rng, n, cfg, K):
    f32, f16 = np.float32, np.float16
    z0, z1, z2 = (f32(v) for v in (Z[0:3] if cfg == 0 else Z[3:6]))
    dz = f32(z2 - z0)
    rdz = f32(f32(1.0) / dz)
    K = f32(K)
    # window of the h1 layer: first hit xr, span up to PF_SPAN
    xr = rng.uniform(-3000.0, 3000.0 - PF_SPAN, n).astype(f32)
    x0 = rng.uniform(-3000.0, 3000.0, n).astype(f32)
    # x2 such that x1_expected lands inside the window (slopes up to ~1)
    lo = np.maximum(-3000.0, x0 + (xr - x0) * float(dz) / float(z1 - z0) - 50.0)
    x2 = (lo + rng.uniform(0.0, 1.0, n) * (PF_SPAN * float(dz) / float(z1 - z0) + 100.0)).astype(f32)
    # exact binary32 path: tx = (x2 - x0) / (z2 - z0); x1e = z1 tx + (x0 - tx z0) K
    tx = f32(f32(x2 - x0) / dz)
    x1e = f32(f32(z1 * tx) + f32(f32(x0 - f32(tx * z0)) * K))
    # pre-filter: slope as a product, same expression
    t = f32(f32(x2 - x0) * rdz)
    e = f32(f32(z1 * t) + f32(f32(x0 - f32(t * z0)) * K))
    # a hit near the cut from the exact x1_expected, inside the window
    d = rng.uniform(-3.2, 3.2, n).astype(f32)
    x1 = f32(x1e + d)
    inside = (x1 >= xr) & (f32(x1 - xr) <= f32(PF_SPAN))
    a = f32(x1 - xr).astype(f16)
    b = f32(e - xr).astype(f16)
    dh = np.abs((a - b).astype(f16)).astype(np.float64)
    dx = f32(x1 - x1e)
    return dh[inside], np.abs(dx.astype(np.float64))[inside], f32(dx * dx)[inside], (e - x1e)[inside]


def test_margin_bounds_the_binary16_distance():
    span, margin = _lf_header_constants()
    assert (span, margin) == (PF_SPAN, PF_MARGIN)
    rng = np.random.default_rng(2402)
    worst, slope_err = 0.0, 0.0
    for cfg in (0, 1):
        for K in (1.0, 1.00177513, 1.00142634):
            for _ in range(4):
                dh, dx, chi2, de = _distances(rng, 250_000, cfg, K)
                worst = max(worst, float(np.max(np.abs(dh - dx))))
                slope_err = max(slope_err, float(np.max(np.abs(de))))
                # every hit the exact cut accepts passes the pre-filter
                for T in (8.0, 6.0, 2.0, 0.5):
                    bound = np.nextafter(np.float32(np.sqrt(T) + PF_MARGIN), np.float32(np.inf))
                    acc = chi2 < np.float32(T)
                    assert acc.any()
                    assert np.all(dh[acc] < bound), (cfg, K, T)
    # the two roundings to binary16 (ulp 1 mm near 2000) reach about 1 mm ...
    assert worst > 0.9
    # ... and the margin covers them with the slope product's error
    assert worst + slope_err < PF_MARGIN - 0.05
    assert slope_err < 0.05


def test_a_smaller_margin_would_drop_accepted_pairs():
    """A planted margin of 0.5 mm: with T_triplet = 6 (sqrt 2.45 mm) some hit
    the exact cut accepts is 3 mm away in binary16 (near 2000 mm the binary16
    distances are whole millimetres), so it would fail the pre-filter: the
    test above is sensitive to the margin."""
    rng = np.random.default_rng(7)
    dropped = 0
    for cfg in (0, 1):
        dh, dx, chi2, _ = _distances(rng, 250_000, cfg, 1.0)
        acc = chi2 < np.float32(6.0)
        dropped += int(np.sum(dh[acc] >= np.float32(np.sqrt(6.0) + 0.5)))
    assert dropped > 0
