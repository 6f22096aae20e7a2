"""Field-integral parameterisation for the momentum estimate.

Sec. "Calculation of momentum and track states": q/p follows from Eq.
pt_kick, (t_x,f / sqrt(1 + t_x,f^2 + t_y,f^2) - t_x,i / sqrt(1 + t_x,i^2 +
t_y,i^2)) / (polarity F), with the field integral F a fourth-order polynomial
in dSlope = t_x,f - t_x,i whose coefficients are two-dimensional polynomials
in the VELO slopes, c_i = sum c_i^km t_x^k t_y^m with k + m <= 6, m even (F is
even in t_y) and k of the parity of i (mirroring x flips t_x and dSlope).  The
coefficients are fitted on toy tracks that fill the slope acceptance with a
flat q/p spectrum, as the paper does; here the toy tracks follow the
synthetic detector's kick (t_x,f = t_x,i + polarity kappa q/p), so the fit is
a least-squares problem on a grid, solved in binary64 and stored in binary32.

This is calibration on the host (numpy), run once per detector; the result
goes into lf_params.qop_c.
"""
from __future__ import annotations

import numpy as np

# (k, m) of t_x^k t_y^m in each c_i, in coefficient order (even i: 10 terms,
# odd i: 6 terms; the parameter block holds 10 per i)
KM_EVEN = ((0, 0), (0, 2), (0, 4), (0, 6), (2, 0), (2, 2), (2, 4), (4, 0), (4, 2), (6, 0))
KM_ODD = ((1, 0), (1, 2), (1, 4), (3, 0), (3, 2), (5, 0))


def km_of(i: int):
    return KM_EVEN if i % 2 == 0 else KM_ODD


def _design(tx, ty, ds):
    cols = []
    for i in range(5):
        for (k, m) in km_of(i):
            cols.append(tx ** k * ty ** m * ds ** i)
    return np.stack(cols, axis=-1)


def toy_tracks(kappa: float, tx_max: float = 0.3, ty_max: float = 0.25, p_min: float = 1.5,
               n_tx: int = 25, n_ty: int = 21, n_qop: int = 40):
    """Toy tracks on a grid: slopes over the acceptance, q/p flat in
    [-1/p_min, 1/p_min] (zero excluded); returns (tx, ty, qop, tx_f)."""
    tx, ty = np.linspace(-tx_max, tx_max, n_tx), np.linspace(-ty_max, ty_max, n_ty)
    q = np.linspace(-1.0 / p_min, 1.0 / p_min, n_qop)
    q = q[q != 0.0]
    TX, TY, Q = np.meshgrid(tx, ty, q, indexing="ij")
    TX, TY, Q = TX.ravel(), TY.ravel(), Q.ravel()
    return TX, TY, Q, TX + kappa * Q


def field_integral(tx, ty, qop, tx_f):
    """F that makes Eq. pt_kick return the toy track's q/p (MagUp)."""
    sf = tx_f / np.sqrt(1.0 + tx_f * tx_f + ty * ty)
    si = tx / np.sqrt(1.0 + tx * tx + ty * ty)
    return (sf - si) / qop


def fit_qop_poly(kappa: float = 1.2, **grid) -> np.ndarray:
    """Coefficients qop_c[5][10] (binary32; unused slots of odd i are 0)."""
    tx, ty, q, tx_f = toy_tracks(kappa, **grid)
    A = _design(tx, ty, tx_f - tx)
    sol, *_ = np.linalg.lstsq(A, field_integral(tx, ty, q, tx_f), rcond=None)
    c = np.zeros((5, 10), np.float64)
    j = 0
    for i in range(5):
        n = len(km_of(i))
        c[i, :n] = sol[j:j + n]
        j += n
    return c.astype(np.float32)


def qop_of(c: np.ndarray, tx, ty, tx_f, ty_f, polarity: int = 1):
    """Eq. pt_kick with the fitted field integral, in binary64 (for checks)."""
    c = np.asarray(c, np.float64)
    ds = tx_f - tx
    ci = [sum(c[i, j] * tx ** k * ty ** m for j, (k, m) in enumerate(km_of(i))) for i in range(5)]
    F = ci[0] + ds * (ci[1] + ds * (ci[2] + ds * (ci[3] + ds * ci[4])))
    sf = tx_f / np.sqrt(1.0 + tx_f * tx_f + ty_f * ty_f)
    si = tx / np.sqrt(1.0 + tx * tx + ty * ty)
    return (sf - si) / (polarity * F)
